"""Pins of the complex Hermitian matrix-OMT oracle (Section 4 in its complex setting: Hermitian
densities, Hermitian L_l, skew-Hermitian W, the Hilbert-Schmidt product Re tr(X Y*); the
iteration of Section 7.3 with the Frobenius norms ||U||_2, ||W||_2).

* real symmetric inputs with real L: the iterates equal the real oracle's (||U||_2, ||W||_2)
  element by element, with zero imaginary parts, and lambda_max(-Delta_L) agrees;
* unitary equivariance: conjugating the densities and every L_l by one unitary V conjugates
  every iterate by V (a dropped conjugate or transpose anywhere breaks it);
* grad_L maps Hermitian to skew-Hermitian and is minus the adjoint of div_L in Re tr(X Y*);
  lambda_max(-Delta_L) equals the largest eigenvalue of the Kronecker form
  sum_s (L_s^2 (x) I - 2 L_s (x) L_s^T + I (x) (L_s^2)^T), built here independently;
* a pure reshape rho A -> rho V A V* at the same place costs alpha x mass x g, g the
  least Frobenius norm of W with div_L W = A - B (least squares on the real representation);
* the iteration keeps Phi, U Hermitian and W skew-Hermitian, and R non-increasing.
"""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S


def _rand_unitary(rng, k):
    q, r = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _conj_field(V, F):
    """V F(x) V* per point for [k*k, n, n] planes (or [N*k*k, n, n] blocks of k*k)."""
    k = V.shape[0]
    blocks = F.shape[0] // (k * k)
    M = F.reshape(blocks, k, k, -1)
    return np.einsum("ab,sbcp,dc->sadp", V, M, V.conj()).reshape(F.shape)


def _herm_err(F, k, sign=1):
    M = F.reshape(-1, k, k, F.shape[-2] * F.shape[-1])
    return np.abs(M - sign * M.conj().transpose(0, 2, 1, 3)).max()


@pytest.mark.parametrize("k", [2, 3])
def test_real_inputs_equal_the_real_oracle(k):
    n = 7
    L0, L1 = S.tensor_field_pair(n, k, seed=5 + k)
    L = S.random_L(k, 3, seed=6)
    lr = oracle.quantum_lmax(L)
    assert oracle.zquantum_lmax(L.astype(np.complex128)) == pytest.approx(lr, rel=1e-12)
    kw = dict(tau=10.0, mu=1.0 / (32.0 * 10.0 * (n - 1) ** 2), nu=1.0 / (4.0 * 10.0 * lr), max_iters=400,
              check_every=100)
    r = oracle.momt_solve(L0, L1, L, 0.8, u_norm=oracle.U_L2, w_norm=oracle.W_L2, **kw)
    z = oracle.zmomt_solve(L0.astype(np.complex128), L1.astype(np.complex128), L.astype(np.complex128), 0.8,
                           **kw)
    for key in ("Ux", "Uy", "W", "Phi"):
        assert np.all(z[key].imag == 0.0)
        np.testing.assert_allclose(z[key].real, r[key], rtol=0, atol=1e-12 * max(np.abs(r[key]).max(), 1e-30))
    assert z["metrics"]["primal"] == pytest.approx(r["metrics"]["primal"], rel=1e-12)
    assert z["metrics"]["fp_resid"] == pytest.approx(r["metrics"]["fp_resid"], rel=1e-9)


@pytest.mark.parametrize("k", [2, 3])
def test_unitary_equivariance(k):
    n = 6
    rng = np.random.default_rng(11)
    A0, A1 = S.hermitian_field_pair(n, k, seed=12)
    L = S.random_hermitian_L(k, 3, seed=13)
    V = _rand_unitary(rng, k)
    kw = dict(tau=10.0, max_iters=300, check_every=100)
    a = oracle.zmomt_solve(A0, A1, L, 0.6, **kw)
    LV = np.einsum("ab,sbc,dc->sad", V, L, V.conj())
    b = oracle.zmomt_solve(_conj_field(V, A0), _conj_field(V, A1), LV, 0.6, **kw)
    assert b["nu"] == pytest.approx(a["nu"], rel=1e-10)
    for key in ("Ux", "Uy", "W", "Phi"):
        expect = _conj_field(V, a[key])
        assert np.abs(b[key] - expect).max() <= 1e-10 * max(np.abs(expect).max(), 1e-30), key
    assert b["metrics"]["primal"] == pytest.approx(a["metrics"]["primal"], rel=1e-10)


def test_quantum_operators_in_the_complex_setting():
    rng = np.random.default_rng(3)
    for k in (2, 3):
        L = S.random_hermitian_L(k, 2, seed=4 + k)
        G = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
        X = (G + G.conj().T) / 2
        Z = oracle.zgrad_L_point(X, L)
        assert np.abs(Z + Z.conj().transpose(0, 2, 1)).max() < 1e-13        # skew-Hermitian
        Y = rng.standard_normal((2, k, k)) + 1j * rng.standard_normal((2, k, k))
        lhs = np.sum((Z * Y.conj()).real)
        rhs = -np.sum((X * oracle.zdiv_L_point(Y, L).conj()).real)
        assert lhs == pytest.approx(rhs, rel=1e-12)
        I = np.eye(k)
        M = sum(np.kron(Ls @ Ls, I) - 2 * np.kron(Ls, Ls.T) + np.kron(I, (Ls @ Ls).T) for Ls in L)
        assert oracle.zquantum_lmax(L) == pytest.approx(np.linalg.eigvalsh(M).max(), rel=1e-10)


def _least_norm_g(delta, L):
    """min ||W||_F over W in (C^{k x k})^N with div_L W = delta, on the real representation."""
    N, k = L.shape[0], L.shape[1]
    cols = []
    for s in range(N):
        for q in range(k * k):
            for unit in (1.0, 1j):
                Z = np.zeros((N, k, k), np.complex128)
                Z.reshape(N, -1)[s, q] = unit
                Y = sum(-L[t] @ Z[t] + Z[t] @ L[t] for t in range(N))
                cols.append(np.concatenate([Y.real.ravel(), Y.imag.ravel()]))
    A = np.array(cols).T
    d = np.concatenate([delta.real.ravel(), delta.imag.ravel()])
    x = np.linalg.lstsq(A, d, rcond=None)[0]
    assert np.linalg.norm(A @ x - d) < 1e-10 * np.linalg.norm(d)
    return np.linalg.norm(x)


def test_pure_reshape_costs_alpha_times_least_norm():
    n, k = 5, 2
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.3, 1.0, (n, n)); rho /= rho.sum()
    L = S.random_hermitian_L(k, 2, seed=22)
    A = np.diag([0.7, 0.3]).astype(np.complex128)
    V = _rand_unitary(rng, k)
    B = V @ A @ V.conj().T
    Lam0 = A.reshape(k * k, 1, 1) * rho[None]
    Lam1 = B.reshape(k * k, 1, 1) * rho[None]
    g = _least_norm_g(A - B, L)
    for alpha in (0.2, 1.0):
        o = oracle.zmomt_solve(Lam0, Lam1, L, alpha, tau=10.0, max_iters=200000, check_every=200, tol_gap=1e-9,
                               tol_res=1e-9)
        assert o["metrics"]["primal"] == pytest.approx(alpha * g, rel=1e-6)
        assert o["metrics"]["dual"] == pytest.approx(alpha * g, rel=1e-6)


def test_iteration_keeps_structure():
    n, k = 6, 2
    A0, A1 = S.hermitian_field_pair(n, k, seed=31)
    L = S.random_hermitian_L(k, 3, seed=32)
    o = oracle.zmomt_solve(A0, A1, L, 1.0, max_iters=600, check_every=100, history=True)
    for key in ("Ux", "Uy", "Phi"):
        assert _herm_err(o[key], k) <= 1e-12 * max(np.abs(o[key]).max(), 1e-30)
    assert _herm_err(o["W"], k, sign=-1) <= 1e-12 * max(np.abs(o["W"]).max(), 1e-30)
    assert np.all(o["Ux"][..., -1] == 0) and np.all(o["Uy"][:, -1, :] == 0)
    R = o["history"][:, 4]
    assert np.all(np.diff(R) <= 1e-12 * R[0])


# ---------------------------------------------------------------- the entrywise ||.||_1
@pytest.mark.parametrize("k", [2, 3])
def test_entrywise_norm_with_real_inputs_equals_the_real_oracle(k):
    """||U||_1, ||W||_1 as sums of entry moduli: on real symmetric inputs with real L the
    modulus of an entry is its absolute value, so the iterates must equal the real oracle's
    entrywise-norm iteration (which the LP and closed-form pins fix) element by element."""
    n = 7
    L0, L1 = S.tensor_field_pair(n, k, seed=40 + k)
    L0, L1 = L0 * n * n, L1 * n * n
    L = S.random_L(k, 3, seed=41)
    kw = dict(tau=10.0, max_iters=300, check_every=100)
    r = oracle.momt_solve(L0, L1, L, 0.7, u_norm=oracle.U_L1, w_norm=oracle.W_L1, **kw)
    z = oracle.zmomt_solve(L0.astype(np.complex128), L1.astype(np.complex128), L.astype(np.complex128), 0.7,
                           u_norm=oracle.U_L1, w_norm=oracle.W_L1, **kw)
    for key in ("Ux", "Uy", "W", "Phi"):
        assert np.all(z[key].imag == 0.0)
        np.testing.assert_allclose(z[key].real, r[key], rtol=0, atol=1e-12 * max(np.abs(r[key]).max(), 1e-30))
    for m in ("primal", "dual", "rel_res", "dual_infeas"):
        assert z["metrics"][m] == pytest.approx(r["metrics"][m], rel=1e-10, abs=1e-14), m


@pytest.mark.parametrize("k", [2, 3])
def test_entrywise_norm_diagonal_unitary_equivariance(k):
    """A diagonal unitary D = diag(exp(i theta_a)) multiplies entry (a, b) by
    exp(i (theta_a - theta_b)) and keeps every modulus, so conjugating the densities and
    the L_l by D conjugates every iterate by D.  A shrink that treated the real and
    imaginary parts separately, or a Frobenius shrink, would break this."""
    n = 6
    rng = np.random.default_rng(50 + k)
    A0, A1 = S.hermitian_field_pair(n, k, seed=51)
    A0, A1 = A0 * n * n, A1 * n * n
    L = S.random_hermitian_L(k, 3, seed=52)
    D = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, k)))
    kw = dict(tau=10.0, max_iters=300, check_every=100, u_norm=oracle.U_L1, w_norm=oracle.W_L1)
    a = oracle.zmomt_solve(A0, A1, L, 0.6, **kw)
    LD = np.einsum("ab,sbc,dc->sad", D, L, D.conj())
    b = oracle.zmomt_solve(_conj_field(D, A0), _conj_field(D, A1), LD, 0.6, **kw)
    for key in ("Ux", "Uy", "W", "Phi"):
        expect = _conj_field(D, a[key])
        assert np.abs(b[key] - expect).max() <= 1e-10 * max(np.abs(expect).max(), 1e-30), key
    assert b["metrics"]["primal"] == pytest.approx(a["metrics"]["primal"], rel=1e-10)
    # the entrywise norm is not invariant under a general unitary: the iterates then differ
    V = _rand_unitary(rng, k)
    LV = np.einsum("ab,sbc,dc->sad", V, L, V.conj())
    c = oracle.zmomt_solve(_conj_field(V, A0), _conj_field(V, A1), LV, 0.6, **kw)
    expect = _conj_field(V, a["Phi"])
    assert np.abs(c["Phi"] - expect).max() > 1e-6 * np.abs(expect).max()


def test_entrywise_metrics_and_structure():
    """With ||.||_1 the iteration keeps U, Phi Hermitian and W skew-Hermitian (an entry and
    its mirror have equal moduli, so the entrywise shrink keeps the pairing), R does not
    increase, and the reported primal is the summed entry moduli of U plus alpha times those
    of W."""
    n, k = 6, 3
    A0, A1 = S.hermitian_field_pair(n, k, seed=61)
    A0, A1 = A0 * n * n, A1 * n * n
    L = S.random_hermitian_L(k, 2, seed=62)
    alpha = 0.8
    o = oracle.zmomt_solve(A0, A1, L, alpha, max_iters=400, check_every=50, history=True, u_norm=oracle.U_L1,
                           w_norm=oracle.W_L1)
    for key in ("Ux", "Uy", "Phi"):
        assert _herm_err(o[key], k) <= 1e-12 * max(np.abs(o[key]).max(), 1e-30)
    assert _herm_err(o["W"], k, sign=-1) <= 1e-12 * max(np.abs(o["W"]).max(), 1e-30)
    R = o["history"][:, 4]
    assert np.all(np.diff(R) <= 1e-12 * R[0])
    P = np.abs(o["Ux"]).sum() + np.abs(o["Uy"]).sum() + alpha * np.abs(o["W"]).sum()
    assert o["metrics"]["primal"] == pytest.approx(P, rel=1e-12)
    assert np.abs(o["W"]).max() > 0.0
