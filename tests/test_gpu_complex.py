"""GPU parity of complex Hermitian matrix OMT (momt_solve_complex: Section 4's complex setting,
the Section 7.3 iteration) against the complex FP64 oracle, through the C ABI, for 2 x 2 and
3 x 3 fields, the Frobenius norms ||U||_2, ||W||_2 and the entrywise ||U||_1, ||W||_1 (sums of
the entries' moduli).

* fixed iteration counts from zero, n = 5, 17, 33, N = 2 and 3, both engines: relative L2
  <= 1e-3 on Phi, U and W, relative <= 1e-4 on the primal objective;
* one iteration from a GPU state at 128^2 (both engines): every element within 1e-5 of the
  state's scale;
* real symmetric inputs give the real matrix path's iterates (||U||_2, ||W||_2);
* conjugating the densities and L by a unitary leaves the GPU cost unchanged;
* errors.
Densities: ``synthetic.hermitian_field_pair`` rescaled to mean trace 1 per cell (O(1) masses).
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
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64)).to(_dev())


def _c(x):
    return x.astype(np.complex64).astype(np.complex128)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _pair(n, seed):
    a, b = S.hermitian_field_pair(n, 2, seed=seed)
    return a * n * n, b * n * n


def _gpu(A0, A1, L, alpha, **kw):
    sol = V.momt_solve_complex(_t(A0), _t(A1), L, alpha, **kw)
    torch.cuda.synchronize()
    U = sol.U.cpu().numpy().astype(np.complex128)
    n = U.shape[-1]
    return dict(Ux=U[0], Uy=U[1], W=sol.W.cpu().numpy().astype(np.complex128).reshape(-1, n, n),
                Phi=sol.Phi.cpu().numpy().astype(np.complex128)), sol.result, sol


@pytest.mark.parametrize("engine", ["resident", "stream"])
@pytest.mark.parametrize("n,N", [(5, 2), (17, 3), (33, 2)])
def test_fixed_iterations_match_oracle(engine, n, N):
    A0, A1 = _pair(n, seed=40 + n)
    L = S.random_hermitian_L(2, N, seed=41 + N)
    iters = 200
    G, r, _ = _gpu(A0, A1, L, 0.7, max_iters=iters, check_every=50, engine=engine)
    assert r["iters"] == iters and r["status"] == 0 and r["engine"] == engine
    o = oracle.zmomt_solve(_c(A0), _c(A1), L, 0.7, tau=r["tau"], mu=r["mu"], nu=r["nu"], max_iters=iters,
                           check_every=50)
    assert np.abs(o["Ux"]).max() > 0 and np.abs(o["W"]).max() > 0 and np.abs(o["W"].imag).max() > 0
    assert _rel(G["Phi"], o["Phi"]) <= 1e-3
    assert _rel(np.stack([G["Ux"], G["Uy"]]), np.stack([o["Ux"], o["Uy"]])) <= 1e-3
    assert _rel(G["W"], o["W"]) <= 1e-3
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-4)
    assert r["dual"] == pytest.approx(o["metrics"]["dual"], rel=1e-3, abs=1e-6)


@pytest.mark.parametrize("engine", ["resident", "stream"])
def test_one_iteration_from_gpu_state_at_128(engine):
    n, N = 128, 3
    A0, A1 = _pair(n, seed=7)
    L = S.random_hermitian_L(2, N, seed=8)
    G0, r0, sol = _gpu(A0, A1, L, 1.0, max_iters=100, check_every=100, engine=engine)
    G, r, _ = _gpu(A0, A1, L, 1.0, max_iters=1, check_every=1, engine=engine,
                   init=(sol.U.clone(), sol.W.clone(), sol.Phi.clone()))
    o = oracle.zmomt_solve(_c(A0), _c(A1), L, 1.0, tau=r["tau"], mu=r["mu"], nu=r["nu"], max_iters=1,
                           check_every=1, init=G0)
    for key in ("Phi", "Ux", "Uy", "W"):
        scale = max(np.abs(o[key]).max(), 1e-30)
        err = np.abs(G[key] - o[key]).max() / scale
        assert err <= 1e-5, (key, err)
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-5)


def test_real_inputs_give_the_real_path():
    n = 20
    L0, L1 = S.tensor_field_pair(n, 2, seed=9)
    L0, L1 = L0 * n * n, L1 * n * n
    L = S.random_L(2, 3, seed=10)
    G, r, _ = _gpu(L0.astype(np.complex128), L1.astype(np.complex128), L.astype(np.complex128), 0.5,
                   max_iters=300, check_every=100)
    d = _dev()
    real = V.momt_solve(torch.from_numpy(L0.astype(np.float32)).to(d), torch.from_numpy(L1.astype(np.float32)).to(d),
                        L, 0.5, u_norm=V.U_L2, w_norm=V.W_L2, max_iters=300, check_every=100)
    torch.cuda.synchronize()
    Ur = real.U.cpu().numpy().astype(np.float64)
    assert np.abs(G["Phi"].imag).max() <= 1e-6 * np.abs(G["Phi"]).max()
    assert _rel(G["Phi"].real, real.Phi.cpu().numpy().astype(np.float64)) <= 1e-4
    assert _rel(np.stack([G["Ux"], G["Uy"]]).real, Ur) <= 1e-4
    assert r["primal"] == pytest.approx(real.result["primal"], rel=1e-5)


def test_unitary_conjugation_leaves_the_cost():
    n, N = 16, 3
    rng = np.random.default_rng(5)
    A0, A1 = _pair(n, seed=6)
    L = S.random_hermitian_L(2, N, seed=7)
    q, rr = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))
    Vu = q * (np.diag(rr) / np.abs(np.diag(rr)))

    def conj(F):
        M = F.reshape(2, 2, -1)
        return np.einsum("ab,bcp,dc->adp", Vu, M, Vu.conj()).reshape(F.shape)

    _, ra, _ = _gpu(A0, A1, L, 0.8, max_iters=400, check_every=100)
    LV = np.einsum("ab,sbc,dc->sad", Vu, L, Vu.conj())
    _, rb, _ = _gpu(conj(A0), conj(A1), LV, 0.8, max_iters=400, check_every=100)
    assert rb["nu"] == pytest.approx(ra["nu"], rel=1e-6)
    assert rb["primal"] == pytest.approx(ra["primal"], rel=1e-4)
    assert rb["dual"] == pytest.approx(ra["dual"], rel=1e-4, abs=1e-6)


@pytest.mark.parametrize("k,n,N", [(3, 5, 2), (3, 17, 3), (3, 12, 4), (2, 17, 3)])
@pytest.mark.parametrize("norms", [(V.U_L2, V.W_L2), (V.U_L1, V.W_L1), (V.U_L2, V.W_L1), (V.U_L1, V.W_L2)])
def test_fixed_iterations_3x3_and_entrywise_match_oracle(k, n, N, norms):
    """3 x 3 fields (nine real coordinates per point, the resident engine) and the entrywise
    norms, whose shrink scales each complex entry by its modulus, against the oracle."""
    un, wn = norms
    if k == 2 and norms == (V.U_L2, V.W_L2):
        pytest.skip("covered by test_fixed_iterations_match_oracle")
    A0, A1 = S.hermitian_field_pair(n, k, seed=70 + n + k)
    A0, A1 = A0 * n * n, A1 * n * n
    L = S.random_hermitian_L(k, N, seed=71 + N)
    iters = 200
    G, r, _ = _gpu(A0, A1, L, 0.7, max_iters=iters, check_every=50, u_norm=un, w_norm=wn)
    assert r["iters"] == iters and r["status"] == 0 and r["engine"] == "resident"
    o = oracle.zmomt_solve(_c(A0), _c(A1), L, 0.7, tau=r["tau"], mu=r["mu"], nu=r["nu"], max_iters=iters,
                           check_every=50, u_norm=un, w_norm=wn)
    assert np.abs(o["Ux"]).max() > 0 and np.abs(o["W"]).max() > 0 and np.abs(o["W"].imag).max() > 0
    assert _rel(G["Phi"], o["Phi"]) <= 1e-3
    assert _rel(np.stack([G["Ux"], G["Uy"]]), np.stack([o["Ux"], o["Uy"]])) <= 1e-3
    assert _rel(G["W"], o["W"]) <= 1e-3
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-4)
    assert r["dual"] == pytest.approx(o["metrics"]["dual"], rel=1e-3, abs=1e-6)
    assert r["rel_res"] == pytest.approx(o["metrics"]["rel_res"], rel=1e-3)
    assert r["dual_infeas"] == pytest.approx(o["metrics"]["dual_infeas"], rel=1e-3, abs=1e-6)


def test_one_iteration_from_gpu_state_3x3_entrywise_at_64():
    n, N, k = 64, 3, 3
    A0, A1 = S.hermitian_field_pair(n, k, seed=17)
    A0, A1 = A0 * n * n, A1 * n * n
    L = S.random_hermitian_L(k, N, seed=18)
    kw = dict(u_norm=V.U_L1, w_norm=V.W_L1)
    G0, r0, sol = _gpu(A0, A1, L, 1.0, max_iters=100, check_every=100, **kw)
    G, r, _ = _gpu(A0, A1, L, 1.0, max_iters=1, check_every=1, init=(sol.U.clone(), sol.W.clone(), sol.Phi.clone()),
                   **kw)
    o = oracle.zmomt_solve(_c(A0), _c(A1), L, 1.0, tau=r["tau"], mu=r["mu"], nu=r["nu"], max_iters=1,
                           check_every=1, init=G0, **kw)
    for key in ("Phi", "Ux", "Uy", "W"):
        scale = max(np.abs(o[key]).max(), 1e-30)
        err = np.abs(G[key] - o[key]).max() / scale
        assert err <= 1e-5, (key, err)
    assert r["primal"] == pytest.approx(o["metrics"]["primal"], rel=1e-5)


@pytest.mark.parametrize("k", [2, 3])
def test_entrywise_real_inputs_give_the_real_entrywise_path(k):
    """On real inputs the modulus of an entry is its absolute value: the complex entrywise
    solve equals the real matrix path with ||U||_1, ||W||_1."""
    n = 20
    L0, L1 = S.tensor_field_pair(n, k, seed=19 + k)
    L0, L1 = L0 * n * n, L1 * n * n
    L = S.random_L(k, 3, seed=20)
    G, r, _ = _gpu(L0.astype(np.complex128), L1.astype(np.complex128), L.astype(np.complex128), 0.5,
                   max_iters=300, check_every=100, u_norm=V.U_L1, w_norm=V.W_L1)
    d = _dev()
    real = V.momt_solve(torch.from_numpy(L0.astype(np.float32)).to(d), torch.from_numpy(L1.astype(np.float32)).to(d),
                        L, 0.5, u_norm=V.U_L1, w_norm=V.W_L1, max_iters=300, check_every=100)
    torch.cuda.synchronize()
    assert np.abs(G["Phi"].imag).max() <= 1e-6 * np.abs(G["Phi"]).max()
    assert _rel(G["Phi"].real, real.Phi.cpu().numpy().astype(np.float64)) <= 1e-4
    assert _rel(np.stack([G["Ux"], G["Uy"]]).real, real.U.cpu().numpy().astype(np.float64)) <= 1e-4
    assert r["primal"] == pytest.approx(real.result["primal"], rel=1e-5)


def test_errors():
    n = 6
    A0, A1 = _pair(n, seed=1)
    L = S.random_hermitian_L(2, 2, seed=2)
    with pytest.raises(V.VomtError):
        _gpu(A0, A1 * 1.01, L, 1.0, max_iters=1)
    bad = A0.copy()
    bad[1] += 0.5                                        # not Hermitian
    with pytest.raises(V.VomtError):
        _gpu(bad, A1, L, 1.0, max_iters=1)
    with pytest.raises(V.VomtError):
        _gpu(A0, A1, S.random_hermitian_L(2, 10, seed=3), 1.0, max_iters=1)     # 2 x 2: N > 9
    a3, b3 = S.hermitian_field_pair(n, 3, seed=4)
    with pytest.raises(V.VomtError):
        _gpu(a3, b3, S.random_hermitian_L(3, 5, seed=5), 1.0, max_iters=1)   # 3 x 3: N > 4
    with pytest.raises(V.VomtError) as ex:                                   # 3 x 3: resident engine only
        _gpu(a3, b3, S.random_hermitian_L(3, 2, seed=5), 1.0, max_iters=1, engine="stream")
    assert ex.value.status == -1
    with pytest.raises(V.VomtError) as ex:                                   # entrywise: resident engine only
        _gpu(A0, A1, L, 1.0, max_iters=1, engine="stream", u_norm=V.U_L1, w_norm=V.W_L1)
    assert ex.value.status == -1
    with pytest.raises(V.VomtError):
        _gpu(A0, A1, L, 1.0, max_iters=1, u_norm=V.U_NUC)                    # no nuclear norm here
    Lnh = L.copy()
    Lnh[0, 0, 1] += 0.3                                  # L not Hermitian
    with pytest.raises(V.VomtError):
        _gpu(A0, A1, Lnh, 1.0, max_iters=1)
    # one L: its commutant on Hermitian matrices is span{I, L}, larger than span{I}
    with pytest.raises(V.VomtError) as ex:
        _gpu(A0, A1, L[:1], 1.0, max_iters=1)
    assert ex.value.status == -5                          # VOMT_ERR_L_KERNEL
