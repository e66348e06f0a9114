"""GPU parity of vector OMT on 3-D grids (Appendix A's discretization with a third
direction, the iteration of Section 7.2) against the FP64 oracle, through the C ABI.

* fixed iteration counts from zero on grids that span several 32 x 8 tiles, z chunks and
  a ragged tail (n = 2, 3, 7, 16, 33, 45), every norm pair, k = 1 and 3: relative L2 <=
  1e-3 on phi and u, relative <= 1e-4 on the primal objective;
* one iteration from a GPU state at n = 64 and at the 128^3 benchmark size: every element
  within 1e-5 of the state's scale (one FP32 iteration against FP64);
* warm start, convergence to 1e-5 in both, ghost faces, the step-size rule and the errors.

The parity cases use O(1) cell masses (the densities scaled to mean cell mass 1), so that
the flux is active from the first iterations: with total mass 1 on a large grid the
potential needs many iterations before |grad phi| exceeds 1 and the shrink lets flux
through.
"""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")

K3 = S.COMPLETE_K3


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(_dev())


def _f64(x):
    return x.astype(np.float32).astype(np.float64)


def _gpu(r0, r1, edges, alpha, **kw):
    sol = V.solve3d(_t(r0), _t(r1), edges, alpha, **kw)
    torch.cuda.synchronize()
    return sol


def _np(sol):
    u = sol.u.cpu().numpy().astype(np.float64)
    return dict(ux=u[0], uy=u[1], uz=u[2], w=sol.w.cpu().numpy().astype(np.float64),
                phi=sol.phi.cpu().numpy().astype(np.float64))


NORMS = [(V.U_L12, V.W_L1), (V.U_L2, V.W_L2), (V.U_L1, V.W_L1), (V.U_L12, V.W_L2)]


def _unit_cells(r0, r1):
    s = r0.size
    return r0 * s, r1 * s


@pytest.mark.parametrize("n", [2, 3, 7, 16, 33, 45])
@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("norms", NORMS)
def test_fixed_iterations_match_oracle(n, k, norms):
    if k == 1 and norms[1] != V.W_L1:
        pytest.skip("no edges at k = 1")
    un, wn = norms
    edges = K3 if k == 3 else []
    r0, r1 = _unit_cells(*S.blob_pair3(n, k, seed=20 + n))
    iters = 200
    g = _gpu(r0, r1, edges, 0.7, u_norm=un, w_norm=wn, max_iters=iters, check_every=50)
    r = g.result
    assert r["iters"] == iters and r["status"] == 0 and r["variant"] == 0     # per-thread-load form
    o = oracle.vomt3_solve(_f64(r0), _f64(r1), edges, 0.7, tau=r["tau"], mu=r["mu"], nu=r["nu"], u_norm=un,
                           w_norm=wn, max_iters=iters, check_every=50)
    G = _np(g)
    uo = np.stack([o["ux"], o["uy"], o["uz"]])
    assert np.abs(uo).max() > 0 and o["metrics"]["primal"] > 0      # the flux is active
    assert _rel(G["phi"], o["phi"]) <= 1e-3
    ug = np.stack([G["ux"], G["uy"], G["uz"]])
    assert _rel(ug, uo) <= 1e-3
    if edges:
        assert _rel(G["w"], o["w"]) <= 1e-3
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-4)
    assert r["dual"] == pytest.approx(o["metrics"]["dual"], rel=1e-3, abs=1e-6)
    assert r["rel_res"] == pytest.approx(o["metrics"]["rel_res"], rel=1e-2)


@pytest.mark.parametrize("n,k,zc", [(40, 3, 0), (44, 3, 5), (44, 1, 1), (48, 2, 7), (44, 4, 0), (52, 3, 52),
                                    (44, 5, 0), (40, 6, 3)])
@pytest.mark.parametrize("norms", NORMS)
def test_tma_form_matches_oracle(n, k, zc, norms):
    """The TMA form (n a multiple of 4, n >= 40, k <= 6; k = 6 with the complete graph's 15
    edges does not fit and takes a path graph here): ragged 32 x 8 tiles, z chunks of
    1 (every chunk ends on a phi-only plane), 5, 7, the default and the whole column, so the
    stage ring wraps at every offset."""
    un, wn = norms
    if k == 1 and wn != V.W_L1:
        pytest.skip("no edges at k = 1")
    edges = S.complete_graph(k) if k <= 5 else [(c, c + 1) for c in range(k - 1)]
    r0, r1 = _unit_cells(*S.blob_pair3(n, k, seed=60 + n + k))
    iters = 100
    g = _gpu(r0, r1, edges, 0.7, u_norm=un, w_norm=wn, max_iters=iters, check_every=50, zc=zc)
    r = g.result
    assert r["iters"] == iters and r["status"] == 0 and r["variant"] == 1
    if zc:
        assert r["blocks"] == -(-n // 32) * -(-n // 8) * -(-n // zc)
    o = oracle.vomt3_solve(_f64(r0), _f64(r1), edges, 0.7, tau=r["tau"], mu=r["mu"], nu=r["nu"], u_norm=un,
                           w_norm=wn, max_iters=iters, check_every=50)
    G = _np(g)
    uo = np.stack([o["ux"], o["uy"], o["uz"]])
    assert np.abs(uo).max() > 0
    assert _rel(G["phi"], o["phi"]) <= 1e-3
    assert _rel(np.stack([G["ux"], G["uy"], G["uz"]]), uo) <= 1e-3
    if edges:
        assert _rel(G["w"], o["w"]) <= 1e-3
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-4)


def test_z_chunks_agree():
    """TMA runs with z chunks of 1, 3, 16 and 64 planes give the same iterate to rounding
    (a chunk's first plane recomputes the z flux that the march otherwise carries)."""
    n, k = 64, 3
    r0, r1 = _unit_cells(*S.blob_pair3(n, k, seed=77))
    outs = [_np(_gpu(r0, r1, K3, 1.0, max_iters=50, check_every=50, zc=zc)) for zc in (1, 3, 16, 64)]
    for o in outs[1:]:
        for key in o:
            scale = max(np.abs(outs[0][key]).max(), 1e-30)
            assert np.abs(o[key] - outs[0][key]).max() <= 1e-5 * scale, key


def test_default_step_sizes_follow_the_3d_rule():
    n = 9
    r0, r1 = S.blob_pair3(n, 3, seed=5)
    r = _gpu(r0, r1, K3, 1.0, max_iters=1, check_every=1).result
    assert r["tau"] == 1.0
    assert r["mu"] == pytest.approx(1.0 / (48.0 * r["tau"] * (n - 1) ** 2), rel=1e-12)
    mu, nu, tau, lmax = V.step_sizes(n, 3, K3)
    assert r["nu"] == pytest.approx(nu, rel=1e-12)
    r = _gpu(r0[:1] / r0[:1].sum(), r1[:1] / r1[:1].sum(), [], 1.0, max_iters=1, check_every=1).result
    assert r["mu"] == pytest.approx(1.0 / (24.0 * (n - 1) ** 2), rel=1e-12)


@pytest.mark.parametrize("n", [64, 66, 128])
def test_one_iteration_from_gpu_state_matches_oracle(n):
    """At 128^3 x 3 channels (the benchmark's launch configuration), at 64^3 (both TMA) and
    at 66^3 (per-thread form): run the GPU some iterations, then one more iteration from
    that state on both sides."""
    k = 3
    r0, r1 = _unit_cells(*S.blob_pair3(n, k, seed=40 + n))
    g = _gpu(r0, r1, K3, 1.0, max_iters=60, check_every=60)
    state = _np(g)
    assert np.abs(state["uz"]).max() > 0 and np.abs(state["w"]).max() > 0
    init = (g.u.clone(), g.w.clone(), g.phi.clone())
    g1 = _gpu(r0, r1, K3, 1.0, max_iters=1, check_every=1, init=init)
    r = g1.result
    assert r["variant"] == (1 if n % 4 == 0 else 0)
    o = oracle.vomt3_solve(_f64(r0), _f64(r1), K3, 1.0, tau=r["tau"], mu=r["mu"], nu=r["nu"], max_iters=1,
                           check_every=1, init=state)
    G = _np(g1)
    for key in ("phi", "ux", "uy", "uz", "w"):
        scale = max(np.abs(o[key]).max(), 1e-30)
        err = np.abs(G[key] - o[key]).max() / scale
        assert err <= 1e-5, (key, err)
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-5)
    assert r["fp_resid"] == pytest.approx(o["metrics"]["fp_resid"], rel=5e-2)


def test_ghost_faces_stay_zero_and_phi_mean_zero():
    n = 12
    r0, r1 = _unit_cells(*S.blob_pair3(n, 3, seed=3))
    G = _np(_gpu(r0, r1, K3, 1.0, max_iters=300, check_every=100))
    assert np.all(G["ux"][..., -1] == 0) and np.all(G["uy"][..., -1, :] == 0) and np.all(G["uz"][:, -1] == 0)
    assert abs(G["phi"].sum()) <= 1e-4 * np.abs(G["phi"]).sum()


def test_warm_start_continues_the_run():
    n = 40
    r0, r1 = _unit_cells(*S.blob_pair3(n, 3, seed=8))
    full = _gpu(r0, r1, K3, 1.0, max_iters=200, check_every=100)
    half = _gpu(r0, r1, K3, 1.0, max_iters=100, check_every=100)
    cont = _gpu(r0, r1, K3, 1.0, max_iters=100, check_every=100, init=(half.u, half.w, half.phi))
    a, b = _np(full), _np(cont)
    for key in a:
        np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-6 * max(np.abs(a[key]).max(), 1e-30))


def test_converges_with_the_oracle():
    """Both reach gap and residual 1e-5; their objectives agree to the tolerance."""
    n = 8
    r0, r1 = S.blob_pair3(n, 3, seed=11)
    kw = dict(max_iters=400000, check_every=200, tol_gap=1e-5, tol_res=1e-5)
    g = _gpu(r0, r1, K3, 1.0, **kw).result
    assert g["status"] == 0 and g["rel_gap"] <= 1e-5 and g["rel_res"] <= 1e-5
    o = oracle.vomt3_solve(_f64(r0), _f64(r1), K3, 1.0, tau=g["tau"], mu=g["mu"], nu=g["nu"],
                           **dict(kw, tol_gap=1e-9, tol_res=1e-9))
    assert g["primal"] == pytest.approx(o["metrics"]["primal"], rel=5e-5)


def test_z_constant_volume_costs_the_2d_optimum_on_gpu():
    """A density constant in z costs the 2-D optimum of one slice (GPU 3-D vs GPU 2-D)."""
    n = 8
    r0, r1 = S.blob_pair(n, 3, seed=12)
    kw = dict(tau=3.0, max_iters=400000, check_every=200, tol_gap=1e-5, tol_res=1e-5)
    d = _dev()
    two = V.solve(torch.from_numpy(r0.astype(np.float32)).to(d), torch.from_numpy(r1.astype(np.float32)).to(d),
                  K3, 1.0, **kw).result
    r0_3 = np.repeat(r0[:, None], n, axis=1) / n
    r1_3 = np.repeat(r1[:, None], n, axis=1) / n
    three = _gpu(r0_3, r1_3, K3, 1.0, **kw).result
    assert three["primal"] == pytest.approx(two["primal"], rel=3e-5)


def test_errors():
    n = 6
    r0, r1 = S.blob_pair3(n, 3, seed=2)
    with pytest.raises(V.VomtError):
        _gpu(r0, r1 * 1.01, K3, 1.0, max_iters=1)
    bad = r0.copy()
    bad[0, 0, 0, 0] = -1.0
    with pytest.raises(V.VomtError):
        _gpu(bad, r1, K3, 1.0, max_iters=1)
    with pytest.raises(V.VomtError):
        _gpu(r0, r1, K3, 1.0, max_iters=1, u_norm=V.U_NUC)
    with pytest.raises(V.VomtError):
        _gpu(r0, r1, K3, 1.0, max_iters=1, mu=1.0 / (8.0 * (n - 1) ** 2))   # breaks the 3-D rule
    with pytest.raises(ValueError):
        V.solve3d(_t(r0[:, 0]), _t(r1[:, 0]), K3, 1.0)
    # beyond the 3-D size limit (n <= 1024): refused before any allocation
    big = torch.zeros((1, 2, 2, 2), device=_dev())
    import ctypes
    from paper_1712_10279_gb300 import _native
    p = V._params(None, None, None, V.U_L12, V.W_L1, 1, 1, 0.0, 0.0, False, "stream")
    g = _native.GraphArg(1, [], None)
    rc = _native.load().vomt_solve3d(_native.context(0), 1025, big.data_ptr(), big.data_ptr(), g.ref, 1.0,
                                     ctypes.byref(p), big.data_ptr(), None, big.data_ptr(),
                                     ctypes.byref(_native.Result()), None)
    assert rc < 0
