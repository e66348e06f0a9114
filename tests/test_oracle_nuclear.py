"""Pins of the oracle's nuclear-norm pieces (Section 6.2 norms ||U||_{1,nuc}, ||W||_{1,nuc};
shrink_nuc of Appendix B) and of matrix OMT under those norms.

* shrink_nuc: soft-thresholded singular values on diagonal matrices; the uniform scaling
  max(0, 1 - t / theta) of a 3 x 3 skew matrix (both nonzero singular values are theta);
  unitary invariance; the proximal optimality of the result against random perturbations;
  the Lemma of Appendix B (symmetric in, symmetric out; skew in, skew out).
* nuclear and spectral norms are dual: <X, Y> <= ||X||_nuc ||Y||_2, with equality at the
  polar factor.
* matrix OMT with ||U||_{1,nuc}: an isotropic density moved s cells costs mass x shift
  (the nuclear norm of f I / k is |f|);
* with ||W||_{1,nuc}: a pure reshape costs alpha x min sum_s ||W_s||_nuc subject to
  div_L W = Lam0 - Lam1, the latter solved here independently as a second-order cone
  program (scipy SLSQP on the epigraph form) from the commutators written out.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_L():
    vals = []
    with open(os.path.join(GOLDEN, "dti_L.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#") or line.startswith("L"):
                continue
            vals.append([float(x) for x in line.split()])
    return np.array(vals).reshape(2, 3, 3)


def _rand_orth(rng, k):
    q, r = np.linalg.qr(rng.standard_normal((k, k)))
    return q * np.sign(np.diag(r))


def test_shrink_nuc_on_diagonal_matrices():
    for d in ([3.0, -1.0, 0.5], [0.2, -0.1], [-2.0, 4.0, -0.3]):
        X = np.diag(d)
        t = 0.7
        expect = np.diag(np.sign(d) * np.maximum(np.abs(d) - t, 0.0))
        np.testing.assert_allclose(oracle.shrink_nuc(X, t), expect, atol=1e-12)
        assert oracle.nuc_norm(X) == pytest.approx(np.abs(d).sum(), rel=1e-12)
        assert oracle.spectral_norm(X) == pytest.approx(np.abs(d).max(), rel=1e-12)


def test_shrink_nuc_of_skew_matrices():
    rng = np.random.default_rng(1)
    for _ in range(5):
        a, b, c = rng.standard_normal(3)
        X = np.array([[0, a, b], [-a, 0, c], [-b, -c, 0]])
        th = np.sqrt(a * a + b * b + c * c)
        for t in (0.3 * th, 1.5 * th):
            np.testing.assert_allclose(oracle.shrink_nuc(X, t), max(0.0, 1 - t / th) * X, atol=1e-7 * th)
        assert oracle.nuc_norm(X) == pytest.approx(2 * th, rel=1e-7)
        X2 = np.array([[0, a], [-a, 0]])
        np.testing.assert_allclose(oracle.shrink_nuc(X2, 0.5 * abs(a)), X2 * 0.5, atol=1e-10 * abs(a))


def test_shrink_nuc_unitary_invariance_and_lemma():
    rng = np.random.default_rng(2)
    for k in (2, 3):
        for _ in range(5):
            X = rng.standard_normal((k, k))
            Q1, Q2 = _rand_orth(rng, k), _rand_orth(rng, k)
            t = 0.4
            np.testing.assert_allclose(oracle.shrink_nuc(Q1 @ X @ Q2.T, t), Q1 @ oracle.shrink_nuc(X, t) @ Q2.T,
                                       atol=1e-7)
            Sym = X + X.T
            Sk = X - X.T
            Z = oracle.shrink_nuc(Sym, t)
            np.testing.assert_allclose(Z, Z.T, atol=1e-8)
            Z = oracle.shrink_nuc(Sk, t)
            np.testing.assert_allclose(Z, -Z.T, atol=1e-8)


def test_shrink_nuc_is_the_proximal_point():
    rng = np.random.default_rng(3)
    for k in (2, 3):
        for _ in range(4):
            X = rng.standard_normal((k, k))
            t = 0.5
            Z = oracle.shrink_nuc(X, t)

            def obj(Y):
                return t * np.linalg.svd(Y, compute_uv=False).sum() + 0.5 * np.sum((Y - X) ** 2)

            f0 = obj(Z)
            for _ in range(200):
                D = rng.standard_normal((k, k)) * 10 ** rng.uniform(-4, -1)
                assert obj(Z + D) >= f0 - 1e-10


def test_nuclear_and_spectral_norms_are_dual():
    rng = np.random.default_rng(4)
    for _ in range(10):
        X, Y = rng.standard_normal((3, 3)), rng.standard_normal((3, 3))
        assert np.sum(X * Y) <= oracle.nuc_norm(X) * oracle.spectral_norm(Y) * (1 + 1e-12)
        U, s, Vt = np.linalg.svd(X)
        assert np.sum(X * (U @ Vt)) == pytest.approx(oracle.nuc_norm(X), rel=1e-7)
        assert oracle.spectral_norm(U @ Vt) == pytest.approx(1.0, rel=1e-7)


def _iso(rho, k):
    M = np.zeros((k * k,) + rho.shape)
    for a in range(k):
        M[a * k + a] = rho / k
    return M


def test_matrix_nuclear_isotropic_shift_costs_mass_times_shift():
    n, k, s = 10, 3, 2
    b0, b1 = S.shifted_blob_pair(n, 1, s, sigma=1.0, margin=2)
    L = _read_L()
    exact = s / (n - 1)
    for w_norm in (oracle.W_L1, oracle.W_NUC):
        o = oracle.momt_solve(_iso(b0[0], k), _iso(b1[0], k), L, alpha=1.0, tau=10.0, u_norm=oracle.U_NUC,
                              w_norm=w_norm, max_iters=200000, check_every=200, tol_gap=1e-8, tol_res=1e-8)
        assert o["metrics"]["primal"] == pytest.approx(exact, rel=1e-5)
        assert o["metrics"]["dual"] == pytest.approx(exact, rel=1e-5)


def _g_L_nuc(delta, L):
    """min sum_s ||W_s||_nuc over skew W_s with sum_s (-L_s W_s + W_s L_s) = delta; for 3 x 3
    skew W_s = [[0, a, b], [-a, 0, c], [-b, -c, 0]], ||W_s||_nuc = 2 ||(a, b, c)||_2, so this is
    a second-order cone program, solved in epigraph form: min 2 sum t_s, t_s^2 >= |w_s|^2."""
    from scipy.optimize import minimize
    N = L.shape[0]

    def skew(v):
        a, b, c = v
        return np.array([[0, a, b], [-a, 0, c], [-b, -c, 0]])

    cols = []
    for s in range(N):
        for q in range(3):
            e = np.zeros(3); e[q] = 1.0
            W = skew(e)
            cols.append((-L[s] @ W + W @ L[s]).ravel())
    A = np.array(cols).T                       # 9 x 3N
    # equality constraints on an orthonormal basis of the range of A (the rows of A are dependent)
    U_, sv, _ = np.linalg.svd(A, full_matrices=False)
    Q = U_[:, sv > 1e-10 * sv[0]]
    d = delta.ravel()
    assert np.linalg.norm(d - Q @ (Q.T @ d)) < 1e-12 * np.linalg.norm(d)    # delta is reachable
    QA, Qd = Q.T @ A, Q.T @ d
    x0 = np.concatenate([np.linalg.lstsq(A, d, rcond=None)[0], np.ones(N)])
    cons = [dict(type="eq", fun=lambda x: QA @ x[:3 * N] - Qd)]
    for s in range(N):
        cons.append(dict(type="ineq", fun=lambda x, s=s: x[3 * N + s] ** 2 - np.sum(x[3 * s:3 * s + 3] ** 2)))
        cons.append(dict(type="ineq", fun=lambda x, s=s: x[3 * N + s]))
    x0[3 * N:] = [np.linalg.norm(x0[3 * s:3 * s + 3]) + 1e-3 for s in range(N)]
    res = minimize(lambda x: 2 * np.sum(x[3 * N:]), x0, constraints=cons, method="SLSQP",
                   options=dict(maxiter=2000, ftol=1e-14))
    assert res.success, res.message
    return res.fun


def test_matrix_nuclear_pure_reshape_matches_cone_program():
    """Lam0 = rho A, Lam1 = rho B at the same place, ||W||_{1,nuc}: M = alpha mass g(A - B)."""
    n, k = 6, 3
    L = _read_L()
    rng = np.random.default_rng(10)
    rho = rng.uniform(0.3, 1.0, (n, n)); rho /= rho.sum()
    A = np.diag([0.6, 0.3, 0.1]); th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    B = R @ A @ R.T
    Lam0 = (A.reshape(9, 1, 1) * rho[None]); Lam1 = (B.reshape(9, 1, 1) * rho[None])
    g = _g_L_nuc(A - B, L)
    for alpha in (0.1, 0.5):
        o = oracle.momt_solve(Lam0, Lam1, L, alpha=alpha, tau=10.0, u_norm=oracle.U_NUC, w_norm=oracle.W_NUC,
                              max_iters=200000, check_every=200, tol_gap=1e-9, tol_res=1e-9)
        assert o["metrics"]["primal"] == pytest.approx(alpha * g, rel=1e-5)
        assert o["metrics"]["dual"] == pytest.approx(alpha * g, rel=1e-5)
