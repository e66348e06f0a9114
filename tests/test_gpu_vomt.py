"""GPU parity of the vector-OMT solver (Section 7.2) against the FP64 oracle,
called through the C ABI.  Tolerances: relative L2 <= 1e-3 on phi and u and
relative <= 1e-4 on the primal objective at a fixed iteration count."""
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


def _gpu(r0, r1, edges, alpha, **kw):
    d = _dev()
    sol = V.solve(torch.from_numpy(r0.astype(np.float32)).to(d), torch.from_numpy(r1.astype(np.float32)).to(d),
                  edges, alpha, **kw)
    torch.cuda.synchronize()
    return sol


def _oracle(r0, r1, edges, alpha, **kw):
    return oracle.vomt_solve(r0.astype(np.float32).astype(np.float64), r1.astype(np.float32).astype(np.float64),
                             edges, alpha, **kw)


def _compare(sol, ref, tol_field=1e-3, tol_obj=1e-4, k=None):
    phi = sol.phi.cpu().numpy().astype(np.float64)
    u = sol.u.cpu().numpy().astype(np.float64)
    ru = np.stack([ref["ux"], ref["uy"]])
    e_phi, e_u = _rel(phi, ref["phi"]), _rel(u, ru)
    e_p = abs(sol.result["primal"] - ref["metrics"]["primal"]) / max(abs(ref["metrics"]["primal"]), 1e-300)
    assert e_phi <= tol_field, ("phi", e_phi)
    assert e_u <= tol_field, ("u", e_u)
    assert e_p <= tol_obj, ("primal", e_p)
    if ref["w"].size:
        assert _rel(sol.w.cpu().numpy().astype(np.float64), ref["w"]) <= 10 * tol_field
    return e_phi, e_u, e_p


ENGINES = ["stream", "resident"]


@pytest.mark.parametrize("engine", ENGINES)
def test_parity_blob_32_k3_2000_iterations(engine):
    r0, r1 = S.blob_pair(32, 3, seed=1001)
    sol = _gpu(r0, r1, K3, 1.0, max_iters=2000, check_every=100, engine=engine)
    assert sol.result["engine"] == engine
    ref = _oracle(r0, r1, K3, 1.0, max_iters=2000, check_every=100, history=True)
    assert sol.result["iters"] == 2000 and sol.result["checks"] == 20
    errs = _compare(sol, ref)
    print("32x32 k=3 2000 it: rel err phi %.2e u %.2e P %.2e" % errs)
    # every check row agrees with the oracle's
    h = V.history()
    assert h.shape == (20, 8)
    np.testing.assert_allclose(h[:, 6], ref["history"][:, 6])
    np.testing.assert_allclose(h[:, 0], ref["history"][:, 0], rtol=1e-4)
    np.testing.assert_allclose(h[:, 3], ref["history"][:, 3], rtol=2e-2)
    np.testing.assert_allclose(h[:, 2], ref["history"][:, 2], rtol=5e-2, atol=1e-5)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n", [2, 3, 5, 33, 47, 70, 130])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_parity_sizes_and_channels(n, k, engine):
    rng = np.random.default_rng(100 * n + k)
    edges = S.random_connected_graph(rng, k, 0.6)
    r0, r1 = S.blob_pair(n, k, seed=10 * n + k) if n >= 5 else (rng.uniform(0.1, 1, (k, n, n)), rng.uniform(0.1, 1, (k, n, n)))
    r0 = r0 / r0.sum(); r1 = r1 / r1.sum()
    sol = _gpu(r0, r1, edges, 0.7, max_iters=300, check_every=60, engine=engine)
    assert sol.result["engine"] == engine
    ref = _oracle(r0, r1, edges, 0.7, max_iters=300, check_every=60)
    _compare(sol, ref)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("u_norm,w_norm", [(0, 1), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_parity_norms(u_norm, w_norm, engine):
    r0, r1 = S.blob_pair(40, 3, seed=77)
    sol = _gpu(r0, r1, K3, 2.0, u_norm=u_norm, w_norm=w_norm, max_iters=500, check_every=100, engine=engine)
    ref = _oracle(r0, r1, K3, 2.0, u_norm=u_norm, w_norm=w_norm, max_iters=500, check_every=100)
    _compare(sol, ref)


def test_parity_edge_costs_and_tau():
    r0, r1 = S.blob_pair(36, 4, seed=5)
    edges = [(0, 1), (1, 2), (2, 3), (0, 3)]
    cost = [1.0, 0.5, 2.0, 1.5]
    sol = _gpu(r0, r1, edges, 1.0, cost=cost, tau=4.0, max_iters=400, check_every=100)
    ref = _oracle(r0, r1, edges, 1.0, cost=cost, tau=4.0, max_iters=400, check_every=100)
    _compare(sol, ref)


@pytest.mark.parametrize("engine", ENGINES)
def test_one_step_from_gpu_state_at_256(engine):
    """At the full 256 x 256 colour-image size, in the launch configuration the benchmark
    uses: one GPU iteration from a mid-run GPU state against one FP64 oracle iteration from
    the same state."""
    r0, r1 = S.color_image_pair(256, 3, seed=1002)
    mid = _gpu(r0, r1, K3, 1.0, max_iters=300, check_every=100, engine=engine)
    nxt = _gpu(r0, r1, K3, 1.0, max_iters=1, check_every=1, init=(mid.u, mid.w, mid.phi), engine=engine)
    assert mid.result["engine"] == engine and nxt.result["engine"] == engine
    u0 = mid.u.cpu().numpy().astype(np.float64)
    init = dict(ux=u0[0], uy=u0[1], w=mid.w.cpu().numpy().astype(np.float64),
                phi=mid.phi.cpu().numpy().astype(np.float64))
    ref = _oracle(r0, r1, K3, 1.0, max_iters=1, check_every=1, init=init)
    u1 = nxt.u.cpu().numpy().astype(np.float64)
    assert _rel(u1, np.stack([ref["ux"], ref["uy"]])) < 1e-5
    assert _rel(nxt.w.cpu().numpy().astype(np.float64), ref["w"]) < 1e-5
    dphi_g = nxt.phi.cpu().numpy().astype(np.float64) - init["phi"]
    dphi_o = ref["phi"] - init["phi"]
    assert _rel(dphi_g, dphi_o) < 2e-2
    assert _rel(nxt.phi.cpu().numpy().astype(np.float64), ref["phi"]) < 1e-6


@pytest.mark.parametrize("engine", ENGINES)
def test_tolerance_stop_matches_oracle(engine):
    r0, r1 = S.blob_pair(32, 3, seed=1001)
    kw = dict(max_iters=20000, check_every=100, tol_gap=1e-3, tol_res=1e-3)
    sol = _gpu(r0, r1, K3, 1.0, engine=engine, **kw)
    ref = _oracle(r0, r1, K3, 1.0, **kw)
    assert sol.result["status"] == 0
    assert abs(sol.result["iters"] - ref["iters"]) <= 100
    assert sol.result["rel_gap"] <= 1e-3 and sol.result["rel_res"] <= 1e-3


@pytest.mark.parametrize("engine", ENGINES)
def test_invariants_on_gpu(engine):
    r0, r1 = S.color_image_pair(128, 3, seed=3)
    sol = _gpu(r0, r1, K3, 1.0, max_iters=1000, check_every=250, engine=engine)
    u = sol.u.cpu().numpy()
    assert np.all(u[0, :, :, -1] == 0) and np.all(u[1, :, -1, :] == 0)   # ghost cells stay zero
    phi = sol.phi.cpu().numpy().astype(np.float64)
    assert abs(phi.sum()) < 1e-4 * np.abs(phi).sum()                     # Sum phi stays ~0
    h = V.history()
    assert np.all(np.diff(h[:, 4]) <= 1e-6 * h[0, 4])                    # R non-increasing


def test_host_api_matches_device_api():
    r0, r1 = S.blob_pair(48, 3, seed=9)
    dsol = _gpu(r0, r1, K3, 1.0, max_iters=250, check_every=50)
    hsol = V.solve_host(r0.astype(np.float32), r1.astype(np.float32), K3, 1.0, max_iters=250, check_every=50)
    np.testing.assert_array_equal(hsol.phi, dsol.phi.cpu().numpy())
    np.testing.assert_array_equal(hsol.u, dsol.u.cpu().numpy())
    assert hsol.result["primal"] == dsol.result["primal"]


def test_input_errors():
    r0, r1 = S.blob_pair(16, 3, seed=2)
    with pytest.raises(V.VomtError) as e:
        _gpu(r0, 1.01 * r1, K3, 1.0, max_iters=5)
    assert e.value.status == -2
    bad = r1.copy(); bad[0, 3, 3] = -1e-3; bad[1, 2, 2] += 1e-3
    with pytest.raises(V.VomtError) as e:
        _gpu(r0, bad, K3, 1.0, max_iters=5)
    assert e.value.status == -3
    bad = r1.copy(); bad[0, 0, 0] = np.nan
    with pytest.raises(V.VomtError) as e:
        _gpu(r0, bad, K3, 1.0, max_iters=5)
    assert e.value.status == -7
    with pytest.raises(V.VomtError) as e:
        _gpu(r0, r1, K3, 1.0, max_iters=5, mu=1.0, nu=1.0)
    assert e.value.status == -6
    with pytest.raises(V.VomtError) as e:
        _gpu(r0, r1, K3, -1.0, max_iters=5)
    assert e.value.status == -1


@pytest.mark.parametrize("engine", ENGINES)
def test_zero_iterations_and_identical_densities(engine):
    r0, _ = S.blob_pair(40, 3, seed=4)
    sol = _gpu(r0, r0, K3, 1.0, max_iters=0, engine=engine)
    assert sol.result["iters"] == 0 and sol.result["primal"] == 0.0
    sol = _gpu(r0, r0, K3, 1.0, max_iters=50, check_every=10, engine=engine)
    assert sol.result["primal"] == 0.0 and float(sol.phi.abs().max()) == 0.0


def test_auto_engine_choice():
    r0, r1 = S.blob_pair(64, 3, seed=12)
    sol = _gpu(r0, r1, K3, 1.0, max_iters=10)
    assert sol.result["engine"] == "resident"
    r0, r1 = S.blob_pair(600, 1, seed=13)
    sol = _gpu(r0, r1, [], 1.0, max_iters=10)
    assert sol.result["engine"] == "stream"


def test_resident_matches_stream_closely_at_256():
    r0, r1 = S.color_image_pair(256, 3, seed=1002)
    a = _gpu(r0, r1, K3, 1.0, max_iters=3000, check_every=100, engine="stream")
    b = _gpu(r0, r1, K3, 1.0, max_iters=3000, check_every=100, engine="resident")
    assert _rel(b.phi.cpu().numpy().astype(np.float64), a.phi.cpu().numpy().astype(np.float64)) < 1e-5
    assert _rel(b.u.cpu().numpy().astype(np.float64), a.u.cpu().numpy().astype(np.float64)) < 1e-4
    assert abs(a.result["primal"] - b.result["primal"]) <= 1e-5 * a.result["primal"]


@pytest.mark.parametrize("n,k", [(190, 3), (200, 2), (176, 4), (160, 1)])
def test_resident_two_point_384_thread_form_matches_oracle(n, k):
    """Sizes whose default tile plan puts two points on each of at most 384 threads (the
    384-thread form of the resident kernel, ring widths 4 and 5, ragged tiles): iterates and
    the check history equal the oracle's at a fixed iteration count."""
    rng = np.random.default_rng(3 * n + k)
    edges = S.random_connected_graph(rng, k, 0.6)
    r0, r1 = S.blob_pair(n, k, seed=n + 11 * k)
    sol = _gpu(r0, r1, edges, 0.7, max_iters=150, check_every=50, engine="resident")
    assert sol.result["engine"] == "resident" and sol.result["iters"] == 150
    ref = _oracle(r0, r1, edges, 0.7, max_iters=150, check_every=50, history=True)
    _compare(sol, ref)
    h = V.history()
    np.testing.assert_allclose(h[:, 0], ref["history"][:, 0], rtol=1e-4)


@pytest.mark.parametrize("halo", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("n,k", [(64, 3), (130, 2), (256, 3), (97, 5)])
def test_resident_halo_widths_match_oracle(halo, n, k):
    """Temporal blocking: every ring width gives the same iterates (up to FP32 rounding)."""
    rng = np.random.default_rng(n + 10 * k + halo)
    edges = S.random_connected_graph(rng, k, 0.6)
    r0, r1 = S.blob_pair(n, k, seed=n * 7 + k)
    sol = _gpu(r0, r1, edges, 1.3, max_iters=210, check_every=70, engine="resident", halo=halo)
    ref = _oracle(r0, r1, edges, 1.3, max_iters=210, check_every=70, history=True)
    _compare(sol, ref)
    h = V.history()
    np.testing.assert_allclose(h[:, 0], ref["history"][:, 0], rtol=1e-4)
    np.testing.assert_allclose(h[:, 4], ref["history"][:, 4], rtol=5e-2)


@pytest.mark.parametrize("n,k,edges", [(1024, 3, K3), (1028, 3, K3), (1436, 2, [(0, 1)]), (2048, 1, []),
                                       (1024, 1, []), (772, 3, K3)])
def test_tma_streaming_step_matches_oracle(n, k, edges):
    """Grids whose iterate is at least 16 MB over at least 304 tiles, with n a multiple of 4,
    take the TMA form of the streaming step (64 x 16 tiles; 1028, 1436 and 772 leave ragged
    tiles in x and y).  Cell masses
    of order one (equal totals), so that the flux moves within the few iterations run: a few
    iterations from zero, then one from the GPU state, against the FP64 oracle."""
    rng = np.random.default_rng(n)
    r0 = rng.uniform(0.2, 1.0, (k, n, n)); r0 /= r0.mean()
    r1 = rng.uniform(0.2, 1.0, (k, n, n)); r1 /= r1.mean()
    r0 = r0.astype(np.float32); r1 = r1.astype(np.float32)
    kw = dict(max_iters=4, check_every=2, tau=3.0)
    sol = _gpu(r0, r1, edges, 1.0, engine="stream", **kw)
    assert sol.result["blocks"] == ((n + 63) // 64) * ((n + 15) // 16)      # the TMA step ran
    assert np.abs(sol.u.cpu().numpy()).max() > 0                            # the flux moved
    ref = _oracle(r0, r1, edges, 1.0, **kw)
    _compare(sol, ref, k=k)
    nxt = _gpu(r0, r1, edges, 1.0, max_iters=1, check_every=1, engine="stream", tau=3.0,
               init=(sol.u, sol.w, sol.phi))
    u0 = sol.u.cpu().numpy().astype(np.float64)
    init = dict(ux=u0[0], uy=u0[1], w=sol.w.cpu().numpy().astype(np.float64),
                phi=sol.phi.cpu().numpy().astype(np.float64))
    ref1 = _oracle(r0, r1, edges, 1.0, max_iters=1, check_every=1, tau=3.0, init=init)
    assert _rel(nxt.phi.cpu().numpy().astype(np.float64), ref1["phi"]) < 1e-6
    u1 = nxt.u.cpu().numpy().astype(np.float64)
    assert _rel(u1, np.stack([ref1["ux"], ref1["uy"]])) < 1e-5
