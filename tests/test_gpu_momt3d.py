"""GPU parity of matrix OMT on 3-D grids (momt_solve3d: the iteration of Section 7.3 with a
third direction) against the FP64 oracle (full k x k matrices), through the C ABI.

* fixed iteration counts from zero, k = 2 (compact K = 3) and k = 3 (K = 6), each in the TMA
  form (n a multiple of 4, n >= 40) and the per-thread form, every norm pair including the
  nuclear norms, ragged tiles and z chunks: relative L2 <= 1e-3 on Phi, U and W, relative
  <= 1e-4 on the primal objective;
* one iteration from a GPU state at 48^3 (k = 2 and 3, TMA) and 26^3 (k = 3, per-thread form):
  every element within 1e-5 of the state's scale;
* the isotropic density moved along z converges to (mass x shift) / sqrt(k);
* errors.
Densities: ``synthetic.tensor_field_pair3`` rescaled to mean trace 1 per cell (O(1) masses, so
that U and W are active within the tested iterations).
"""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(_dev())


def _f64(x):
    return x.astype(np.float32).astype(np.float64)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _pair(n, k, seed):
    a, b = S.tensor_field_pair3(n, k, seed=seed)
    return a * n ** 3, b * n ** 3


def _gpu(L0, L1, L, alpha, **kw):
    sol = V.momt_solve3d(_t(L0), _t(L1), L, alpha, **kw)
    torch.cuda.synchronize()
    U = sol.U.cpu().numpy().astype(np.float64)
    n = U.shape[-1]
    return dict(Ux=U[0], Uy=U[1], Uz=U[2], W=sol.W.cpu().numpy().astype(np.float64).reshape(-1, n, n, n),
                Phi=sol.Phi.cpu().numpy().astype(np.float64)), sol.result


NORMS = [(V.U_L2, V.W_L1), (V.U_L1, V.W_L2), (V.U_NUC, V.W_L1), (V.U_L2, V.W_NUC), (V.U_NUC, V.W_NUC)]


@pytest.mark.parametrize("n,k,zc,variant", [(5, 2, 0, 0), (12, 3, 0, 0), (44, 2, 7, 1), (40, 2, 0, 1),
                                            (13, 3, 4, 0), (44, 3, 5, 1), (40, 3, 0, 1)])
@pytest.mark.parametrize("norms", NORMS)
def test_fixed_iterations_match_oracle(n, k, zc, variant, norms):
    un, wn = norms
    L0, L1 = _pair(n, k, seed=30 + n + k)
    L = S.random_L(k, 3, seed=31 + k)
    iters = 150 if n <= 13 else 40
    G, r = _gpu(L0, L1, L, 0.7, u_norm=un, w_norm=wn, max_iters=iters, check_every=30, zc=zc)
    assert r["iters"] == iters and r["status"] == 0 and r["variant"] == variant
    o = oracle.momt3_solve(_f64(L0), _f64(L1), L, 0.7, tau=r["tau"], mu=r["mu"], nu=r["nu"], u_norm=un,
                           w_norm=wn, max_iters=iters, check_every=30)
    Uo = np.stack([o["Ux"], o["Uy"], o["Uz"]])
    assert np.abs(Uo).max() > 0 and np.abs(o["W"]).max() > 0
    assert _rel(G["Phi"], o["Phi"]) <= 1e-3
    assert _rel(np.stack([G["Ux"], G["Uy"], G["Uz"]]), Uo) <= 1e-3
    assert _rel(G["W"], o["W"]) <= 1e-3
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-4)
    assert r["dual"] == pytest.approx(o["metrics"]["dual"], rel=1e-3, abs=1e-6)


@pytest.mark.parametrize("n,k", [(48, 2), (48, 3), (26, 3)])
def test_one_iteration_from_gpu_state_matches_oracle(n, k):
    L0, L1 = _pair(n, k, seed=50 + n)
    L = S.random_L(k, 3, seed=51)
    d0, d1 = _t(L0), _t(L1)
    sol = V.momt_solve3d(d0, d1, L, 1.0, max_iters=40, check_every=40)
    torch.cuda.synchronize()
    U = sol.U.cpu().numpy().astype(np.float64)
    state = dict(Ux=U[0], Uy=U[1], Uz=U[2], W=sol.W.cpu().numpy().astype(np.float64).reshape(-1, n, n, n),
                 Phi=sol.Phi.cpu().numpy().astype(np.float64))
    G, r = _gpu(L0, L1, L, 1.0, max_iters=1, check_every=1, init=(sol.U.clone(), sol.W.clone(), sol.Phi.clone()))
    assert r["variant"] == (1 if n % 4 == 0 else 0)
    o = oracle.momt3_solve(_f64(L0), _f64(L1), L, 1.0, tau=r["tau"], mu=r["mu"], nu=r["nu"], max_iters=1,
                           check_every=1, init=state)
    for key in ("Phi", "Ux", "Uy", "Uz", "W"):
        scale = max(np.abs(o[key]).max(), 1e-30)
        err = np.abs(G[key] - o[key]).max() / scale
        assert err <= 1e-5, (key, err)
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-5)


def test_isotropic_density_moved_along_z_on_gpu():
    n, k, s = 6, 3, 2
    rng = np.random.default_rng(2)
    rho = np.zeros((n, n, n))
    rho[0:3, 1:5, 1:5] = rng.uniform(0.5, 1.0, (3, 4, 4))
    rho /= rho.sum()
    moved = np.zeros_like(rho)
    moved[s:] = rho[:n - s]

    def iso(r):
        M = np.zeros((k * k,) + r.shape)
        for a in range(k):
            M[a * k + a] = r / k
        return M

    L = S.random_L(k, 3, seed=12)
    _, r = _gpu(iso(rho), iso(moved), L, 1.0, tau=10.0, max_iters=200000, check_every=200, tol_gap=1e-5,
                tol_res=1e-5)
    assert r["status"] == 0
    assert r["primal"] == pytest.approx((s / (n - 1)) / np.sqrt(k), rel=5e-5)


def test_errors():
    n, k = 6, 3
    L0, L1 = _pair(n, k, seed=1)
    L = S.random_L(k, 3, seed=2)
    with pytest.raises(V.VomtError):
        _gpu(L0, L1 * 1.01, L, 1.0, max_iters=1)
    with pytest.raises(V.VomtError):
        _gpu(L0, L1, L, 1.0, max_iters=1, mu=1.0 / (8.0 * (n - 1) ** 2))    # breaks the 3-D rule
    bad = L0.copy()
    bad[1] += 0.5                                                           # not symmetric
    with pytest.raises(V.VomtError):
        _gpu(bad, L1, L, 1.0, max_iters=1)
    with pytest.raises(ValueError):
        V.momt_solve3d(_t(L0[:, 0]), _t(L1[:, 0]), L, 1.0)
