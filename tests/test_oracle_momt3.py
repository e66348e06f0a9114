"""Pins of the 3-D matrix-OMT oracle (Sections 4-5 and the iteration of Section 7.3 on an
n x n x n grid, the discretization of Appendix A with a third direction).

* k = 1: the matrix problem is scalar OMT (grad_L of a 1 x 1 matrix vanishes), so the
  iterates equal those of the independent 3-D vector oracle with k = 1, element by element;
* an isotropic density rho I / k moved s planes along z costs (mass x shift) / sqrt(k) under
  ||U||_2 and mass x shift under ||U||_{1,nuc}, for two alphas (the z operators carry it);
* a pure reshape at the same place costs alpha x mass x g_L(A - B), g_L by linear
  programming from the commutators written out;
* a z-constant volume costs the 2-D matrix oracle's optimum of one slice;
* the iteration keeps U_d and Phi symmetric and W skew, the ghost faces zero, and the
  fixed-point residual non-increasing.
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


def _iso(rho, k):
    M = np.zeros((k * k,) + rho.shape)
    for a in range(k):
        M[a * k + a] = rho / k
    return M


def test_k1_matrix_iterates_equal_the_scalar_3d_oracle():
    n = 5
    rng = np.random.default_rng(1)
    r0 = rng.uniform(0.2, 1.0, (1, n, n, n)); r0 /= r0.sum()
    r1 = rng.uniform(0.2, 1.0, (1, n, n, n)); r1 /= r1.sum()
    L = np.array([[[0.7]], [[-0.2]]])
    mu, tau = 1.0 / (48.0 * (n - 1) ** 2), 1.0
    m = oracle.momt3_solve(r0, r1, L, 1.0, tau=tau, mu=mu, nu=1.0, u_norm=oracle.U_L2, max_iters=300,
                           check_every=100)
    v = oracle.vomt3_solve(r0, r1, [], 1.0, tau=tau, mu=mu, nu=0.0, u_norm=oracle.U_L2, max_iters=300,
                           check_every=100)
    for a, b in (("Ux", "ux"), ("Uy", "uy"), ("Uz", "uz"), ("Phi", "phi")):
        np.testing.assert_allclose(m[a], v[b], rtol=0, atol=1e-13 * max(np.abs(v[b]).max(), 1e-30))
    assert np.all(m["W"] == 0.0)
    assert m["metrics"]["primal"] == pytest.approx(v["metrics"]["primal"], rel=1e-12)


@pytest.mark.parametrize("u_norm", ["l2", "nuc"])
def test_isotropic_density_moved_along_z(u_norm):
    n, k, s = 6, 3, 2
    rng = np.random.default_rng(2)
    rho = np.zeros((n, n, n))
    rho[0:3, 1:5, 1:5] = rng.uniform(0.5, 1.0, (3, 4, 4))
    rho /= rho.sum()
    moved = np.zeros_like(rho)
    moved[s:] = rho[:n - s]
    L = _read_L()
    un = oracle.U_L2 if u_norm == "l2" else oracle.U_NUC
    exact = (s / (n - 1)) / (np.sqrt(k) if u_norm == "l2" else 1.0)
    for alpha in (0.3, 3.0):
        o = oracle.momt3_solve(_iso(rho, k), _iso(moved, k), L, alpha=alpha, tau=10.0, u_norm=un,
                               max_iters=200000, check_every=200, tol_gap=1e-8, tol_res=1e-8)
        assert o["metrics"]["primal"] == pytest.approx(exact, rel=1e-5)
        assert o["metrics"]["dual"] == pytest.approx(exact, rel=1e-5)


def _g_L(delta, L):
    """min ||W||_1 s.t. div_L W = delta over W in (R^{k x k})^N, by LP (the commutators of
    Section 4.1 written out per entry)."""
    from scipy.optimize import linprog
    N, k = L.shape[0], L.shape[1]
    cols = []
    for s in range(N):
        for q in range(k * k):
            Z = np.zeros((N, k, k)); Z.reshape(N, k * k)[s, q] = 1.0
            Y = sum(-L[t] @ Z[t] + Z[t] @ L[t] for t in range(N))
            cols.append(Y.ravel())
    A = np.array(cols).T
    res = linprog(np.ones(2 * A.shape[1]), A_eq=np.hstack([A, -A]), b_eq=delta.ravel(),
                  bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


def test_pure_reshape_costs_alpha_times_g_L():
    n, k = 4, 3
    L = _read_L()
    rng = np.random.default_rng(10)
    rho = rng.uniform(0.3, 1.0, (n, n, n)); rho /= rho.sum()
    A = np.diag([0.6, 0.3, 0.1]); th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    B = R @ A @ R.T
    Lam0 = A.reshape(9, 1, 1, 1) * rho[None]
    Lam1 = B.reshape(9, 1, 1, 1) * rho[None]
    g = _g_L(A - B, L)
    for alpha in (0.1, 1.0):
        o = oracle.momt3_solve(Lam0, Lam1, L, alpha=alpha, tau=10.0, max_iters=200000, check_every=200,
                               tol_gap=1e-9, tol_res=1e-9)
        assert o["metrics"]["primal"] == pytest.approx(alpha * g, rel=1e-6)
        assert o["metrics"]["dual"] == pytest.approx(alpha * g, rel=1e-6)


def test_z_constant_volume_costs_the_2d_matrix_optimum():
    n = 6
    L0, L1 = S.tensor_field_pair(n, 3, seed=21)
    L = _read_L()
    kw = dict(tau=10.0, max_iters=400000, check_every=200, tol_gap=1e-9, tol_res=1e-9)
    two = oracle.momt_solve(L0, L1, L, 1.0, **kw)
    three = oracle.momt3_solve(np.repeat(L0[:, None], n, axis=1) / n, np.repeat(L1[:, None], n, axis=1) / n, L,
                               1.0, **kw)
    assert three["metrics"]["primal"] == pytest.approx(two["metrics"]["primal"], rel=1e-6)


def test_iteration_keeps_structure_3d():
    n, k = 5, 3
    L = S.random_L(3, 3, seed=12)
    L0, L1 = S.tensor_field_pair(n, k, seed=13)
    Lam0 = np.repeat(L0[:, None], n, axis=1) * np.linspace(0.5, 1.5, n)[None, :, None, None]
    Lam1 = np.repeat(L1[:, None], n, axis=1)
    Lam0 *= np.trace(Lam1.reshape(k, k, -1)).sum() / np.trace(Lam0.reshape(k, k, -1)).sum()
    o = oracle.momt3_solve(Lam0, Lam1, L, 1.0, max_iters=600, check_every=100, history=True)
    for d in ("Ux", "Uy", "Uz", "Phi"):
        M = o[d].reshape(k, k, -1)
        assert np.abs(M - M.transpose(1, 0, 2)).max() <= 1e-12 * max(np.abs(M).max(), 1e-30)
    Wm = o["W"].reshape(3, k, k, -1)
    assert np.abs(Wm + Wm.transpose(0, 2, 1, 3)).max() <= 1e-12 * max(np.abs(Wm).max(), 1e-30)
    assert np.all(o["Ux"][..., -1] == 0) and np.all(o["Uy"][..., -1, :] == 0) and np.all(o["Uz"][:, -1] == 0)
    Rh = o["history"][:, 4]
    assert np.all(np.diff(Rh) <= 1e-12 * Rh[0])
