"""GPU parity of the matrix-OMT solver (Section 7.3) against the FP64 oracle, which
iterates on full k x k matrices while the GPU uses compact symmetric / skew storage
with weighted inner products.  Tolerances as for vector OMT: relative L2 <= 1e-3 on
Phi and U, relative <= 1e-4 on the primal objective, at a fixed iteration count."""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")

ENGINES = ["stream", "resident"]


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _run(T0, T1, L, alpha, **kw):
    d = _dev()
    sol = V.momt_solve(torch.from_numpy(T0.astype(np.float32)).to(d), torch.from_numpy(T1.astype(np.float32)).to(d),
                       L, alpha, **kw)
    torch.cuda.synchronize()
    kw.pop("engine", None)
    kw.pop("halo", None)
    if "init" in kw:
        U, W, P = (x.cpu().numpy().astype(np.float64) for x in kw["init"])
        kw["init"] = dict(Ux=U[0], Uy=U[1], W=W.reshape(-1, *W.shape[2:]), Phi=P)
    ref = oracle.momt_solve(T0.astype(np.float32).astype(np.float64), T1.astype(np.float32).astype(np.float64),
                            L, alpha, **kw)
    return sol, ref


def _compare(sol, ref, tol=1e-3, tol_obj=1e-4):
    Phi = sol.Phi.cpu().numpy().astype(np.float64)
    U = sol.U.cpu().numpy().astype(np.float64)
    W = sol.W.cpu().numpy().astype(np.float64)
    e_phi = _rel(Phi, ref["Phi"])
    e_u = _rel(U, np.stack([ref["Ux"], ref["Uy"]]))
    e_w = _rel(W.reshape(ref["W"].shape), ref["W"])
    P_ref = ref["metrics"]["primal"]
    assert P_ref > 0.0, "test case too short: no flux yet"
    e_p = abs(sol.result["primal"] - P_ref) / abs(P_ref)
    assert e_phi <= tol and e_u <= tol and e_w <= 10 * tol and e_p <= tol_obj, (e_phi, e_u, e_w, e_p)
    # structure: symmetric Phi and U, skew W
    k = int(round(np.sqrt(Phi.shape[0])))
    P4 = Phi.reshape(k, k, *Phi.shape[1:])
    assert np.array_equal(P4, P4.transpose(1, 0, 2, 3))
    W5 = W.reshape(W.shape[0], k, k, *W.shape[2:])
    assert np.array_equal(W5, -W5.transpose(0, 2, 1, 3, 4))
    return e_phi, e_u, e_p


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("which", ["paper", "random3"])
def test_matrix_parity_3x3(engine, which):
    L = S.paper_L() if which == "paper" else S.random_L(3, 3, seed=1003)
    T0, T1 = S.tensor_field_pair(32, 3, seed=1003)
    sol, ref = _run(T0, T1, L, 1.0, max_iters=600, check_every=150, engine=engine)
    assert sol.result["engine"] == engine and sol.result["iters"] == 600
    _compare(sol, ref)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("n", [3, 17, 45])
def test_matrix_parity_2x2_and_sizes(engine, n):
    L = S.random_L(2, 2, seed=n)
    T0, T1 = S.tensor_field_pair(n, 2, seed=n + 1)
    sol, ref = _run(T0, T1, L, 0.8, max_iters=300 if n < 40 else 3000, check_every=100, engine=engine)
    _compare(sol, ref)


@pytest.mark.parametrize("u_norm,w_norm", [(1, 1), (2, 0), (2, 1)])
def test_matrix_parity_norms(u_norm, w_norm):
    L = S.random_L(3, 2, seed=5)
    T0, T1 = S.tensor_field_pair(24, 3, seed=6)
    sol, ref = _run(T0, T1, L, 2.0, u_norm=u_norm, w_norm=w_norm, max_iters=400, check_every=100)
    _compare(sol, ref)


def test_matrix_one_step_at_128_dti_config():
    """The 128 x 128 tensor-field configuration (N = 3 random L, tau = 30): one GPU iteration
    from a mid-run GPU state against one FP64 oracle iteration from the same state."""
    L = S.random_L(3, 3, seed=1003)
    T0, T1 = S.tensor_field_pair(128, 3, seed=1003)
    d = _dev()
    t0 = torch.from_numpy(T0.astype(np.float32)).to(d)
    t1 = torch.from_numpy(T1.astype(np.float32)).to(d)
    mid = V.momt_solve(t0, t1, L, 1.0, max_iters=200, check_every=100)
    nxt = V.momt_solve(t0, t1, L, 1.0, max_iters=1, check_every=1, init=(mid.U, mid.W, mid.Phi))
    torch.cuda.synchronize()
    U, W, P = (x.cpu().numpy().astype(np.float64) for x in (mid.U, mid.W, mid.Phi))
    init = dict(Ux=U[0], Uy=U[1], W=W.reshape(-1, 128, 128), Phi=P)
    ref = oracle.momt_solve(T0.astype(np.float32).astype(np.float64), T1.astype(np.float32).astype(np.float64),
                            L, 1.0, max_iters=1, check_every=1, init=init)
    U1 = nxt.U.cpu().numpy().astype(np.float64)
    assert _rel(U1, np.stack([ref["Ux"], ref["Uy"]])) < 1e-5
    assert _rel(nxt.W.cpu().numpy().astype(np.float64).reshape(ref["W"].shape), ref["W"]) < 1e-4
    dP = nxt.Phi.cpu().numpy().astype(np.float64) - P
    assert _rel(dP, ref["Phi"] - P) < 2e-2


def test_matrix_isotropic_shift_closed_form_on_gpu():
    """Lam = rho I/k moved s cells: M = mass * s * h / sqrt(k) under ||U||_2, for any alpha."""
    n, k, s = 12, 3, 2
    b0, b1 = S.shifted_blob_pair(n, 1, s, sigma=1.0, margin=2)
    def iso(r):
        M = np.zeros((k * k, n, n))
        for a in range(k):
            M[a * k + a] = r / k
        return M
    d = _dev()
    sol = V.momt_solve(torch.from_numpy(iso(b0[0]).astype(np.float32)).to(d),
                       torch.from_numpy(iso(b1[0]).astype(np.float32)).to(d), S.paper_L(), 1.0, tau=10.0,
                       max_iters=100000, check_every=500, tol_gap=2e-5, tol_res=2e-5)
    exact = (s / (n - 1)) / np.sqrt(k)
    assert sol.result["status"] == 0
    assert sol.result["primal"] == pytest.approx(exact, rel=1e-4)


def test_matrix_input_errors():
    d = _dev()
    T0, T1 = S.tensor_field_pair(16, 3, seed=2)
    t0 = torch.from_numpy(T0.astype(np.float32)).to(d)
    with pytest.raises(V.VomtError) as e:
        V.momt_solve(t0, 1.01 * torch.from_numpy(T1.astype(np.float32)).to(d), S.paper_L(), 1.0, max_iters=5)
    assert e.value.status == -2
    with pytest.raises(V.VomtError) as e:
        V.momt_solve(t0, torch.from_numpy(T1.astype(np.float32)).to(d), np.diag([1.0, 1.0, 0])[None], 1.0,
                     max_iters=5)
    assert e.value.status == -5
    asym = T1.copy(); asym[1] += 0.1 * np.abs(T1).max()
    with pytest.raises(V.VomtError) as e:
        V.momt_solve(t0, torch.from_numpy(asym.astype(np.float32)).to(d), S.paper_L(), 1.0, max_iters=5)
    assert e.value.status in (-1, -2)


# ---- nuclear norms (Section 6.2: ||U||_{1,nuc}, ||W||_{1,nuc}; shrink of Appendix B)
@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("u_norm,w_norm", [(oracle.U_NUC, oracle.W_L1), (oracle.U_NUC, oracle.W_NUC),
                                           (oracle.U_L2, oracle.W_NUC)])
def test_matrix_parity_nuclear_norms(engine, k, u_norm, w_norm):
    L = S.random_L(k, 3 if k == 3 else 2, seed=40 + k)
    T0, T1 = S.tensor_field_pair(29, k, seed=41 + k)
    sol, ref = _run(T0, T1, L, 0.7, max_iters=900, check_every=300, engine=engine, u_norm=u_norm, w_norm=w_norm)
    assert sol.result["engine"] == engine
    _compare(sol, ref)
    m = ref["metrics"]
    assert sol.result["dual_infeas"] == pytest.approx(m["dual_infeas"], rel=1e-3, abs=1e-6)


@pytest.mark.parametrize("engine", ENGINES)
def test_matrix_nuclear_parity_at_tiny_scale(engine):
    """Scaling both densities by s and tau by 1/s scales mu and nu by s (Section 7.3's rules),
    so the exact iterates are s U, s W and the same Phi.  At s = 2^-40 the 3 x 3 entries of the
    nuclear shrink sit near 1e-20, where squares of squares underflow in FP32; the GPU must
    still match the FP64 oracle run on the same scaled problem."""
    k, s = 3, 2.0 ** -40
    L = S.random_L(k, 3, seed=43)
    T0, T1 = S.tensor_field_pair(29, k, seed=44)
    sol, ref = _run(T0 * s, T1 * s, L, 0.7, tau=30.0 / s, max_iters=900, check_every=300, engine=engine,
                    u_norm=oracle.U_NUC, w_norm=oracle.W_NUC)
    _compare(sol, ref)
    big, _ = _run(T0, T1, L, 0.7, tau=30.0, max_iters=900, check_every=300, engine=engine, u_norm=oracle.U_NUC,
                  w_norm=oracle.W_NUC)
    assert _rel(sol.U.cpu().numpy() / s, big.U.cpu().numpy()) <= 1e-4
    assert sol.result["primal"] / s == pytest.approx(big.result["primal"], rel=1e-4)


@pytest.mark.parametrize("engine", ENGINES)
def test_matrix_nuclear_isotropic_shift_on_gpu(engine):
    """||U||_{1,nuc}: an isotropic density moved s cells costs mass x shift (within the
    tolerance reached)."""
    n, k, s = 12, 3, 2
    b0, b1 = S.shifted_blob_pair(n, 1, s, sigma=1.0, margin=2)
    iso = lambda r: np.stack([(r / k if a == b else 0.0 * r) for a in range(k) for b in range(k)])
    L = S.paper_L()
    sol, _ = _run(iso(b0[0]), iso(b1[0]), L, 1.0, tau=10.0, max_iters=100000, check_every=200, tol_gap=1e-5,
                  tol_res=1e-5, engine=engine, u_norm=oracle.U_NUC)
    assert sol.result["status"] == 0
    assert sol.result["primal"] == pytest.approx(s / (n - 1), rel=3e-5)
