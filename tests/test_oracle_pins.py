"""Pins for the FP64 oracle: each test checks it against something the paper or
the mathematics fixes independently of the oracle's own code (a printed worked
example, a closed form, an invariant, a textbook special case, an LP solve or
brute force on a tiny input)."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
K3 = S.COMPLETE_K3


def _read_golden_matrix(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#") or line.startswith("edges:"):
                continue
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


# ------------------------------------------------------------------ Section 3.1
def test_incidence_matches_figure1_example():
    D = _read_golden_matrix("incidence_fig1.txt")
    edges = [(0, 1), (0, 2), (1, 2), (0, 3), (2, 3)]
    np.testing.assert_array_equal(oracle.incidence(4, edges), D)
    # orientation does not depend on the order the pair is given in
    np.testing.assert_array_equal(oracle.incidence(4, [(b, a) for a, b in edges]), D)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 7])
def test_graph_laplacian_lmax_closed_forms(k):
    # complete graph K_k: Laplacian spectrum {0, k (k-1 times)}
    assert oracle.graph_lmax(k, S.complete_graph(k)) == pytest.approx(k, rel=1e-12)
    # path P_k: 2 - 2 cos(pi j / k), j = 0..k-1
    path = [(a, a + 1) for a in range(k - 1)]
    assert oracle.graph_lmax(k, path) == pytest.approx(2 - 2 * np.cos(np.pi * (k - 1) / k), rel=1e-12)
    # star S_k: {0, 1 (k-2 times), k}
    star = [(0, a) for a in range(1, k)]
    assert oracle.graph_lmax(k, star) == pytest.approx(k, rel=1e-12)
    # edge costs c scale the weights 1/c^2
    assert oracle.graph_lmax(k, S.complete_graph(k), cost=2.0) == pytest.approx(k / 4.0, rel=1e-12)


def test_jacobi_matches_lapack():
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 5, 9):
        A = rng.standard_normal((m, m))
        A = A + A.T
        np.testing.assert_allclose(oracle.jacobi_eigvals(A), np.linalg.eigvalsh(A), rtol=0, atol=1e-12)


def test_graph_div_is_minus_adjoint_of_graph_grad():
    rng = np.random.default_rng(1)
    k, n = 5, 4
    edges = [(0, 1), (1, 2), (0, 3), (2, 4), (3, 4), (1, 4)]
    cost = rng.uniform(0.5, 2.0, len(edges))
    phi = rng.standard_normal((k, n, n))
    y = rng.standard_normal((len(edges), n, n))
    lhs = np.sum(oracle.grad_G(phi, edges, cost) * y)
    rhs = -np.sum(phi * oracle.div_G(y, k, edges, cost))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # grad_G vanishes on constants shared by all channels, and Sum_c div_G = 0
    assert np.abs(oracle.grad_G(np.ones((k, n, n)), edges, cost)).max() == 0.0
    assert np.abs(oracle.div_G(y, k, edges, cost).sum(axis=0)).max() < 1e-13


# ------------------------------------------------------------------ Appendix A
def test_spatial_gradient_of_linear_field_and_ghosts():
    n = 7
    h = 1.0 / (n - 1)
    jj, ii = np.mgrid[0:n, 0:n].astype(float)
    phi = (2.5 * ii * h - 1.5 * jj * h)[None]
    gx, gy = oracle.grad(phi)
    np.testing.assert_allclose(gx[0, :, :-1], 2.5, rtol=1e-12)
    np.testing.assert_allclose(gy[0, :-1, :], -1.5, rtol=1e-12)
    assert np.all(gx[0, :, -1] == 0) and np.all(gy[0, -1, :] == 0)


def test_divergence_of_uniform_flux_is_boundary_only():
    n = 6
    ux = np.zeros((1, n, n)); uy = np.zeros((1, n, n))
    ux[0, :, :-1] = 0.3          # uniform x-flux on real entries, ghosts zero
    d = oracle.div(ux, uy)[0] / (n - 1)
    np.testing.assert_allclose(d[:, 0], 0.3)
    np.testing.assert_allclose(d[:, 1:-1], 0.0, atol=1e-15)
    np.testing.assert_allclose(d[:, -1], -0.3)
    assert abs(oracle.div(ux, uy).sum()) < 1e-13   # zero-flux boundary conserves mass


def test_spatial_div_is_minus_transpose_of_grad():
    rng = np.random.default_rng(2)
    k, n = 3, 9
    phi = rng.standard_normal((k, n, n))
    ux = rng.standard_normal((k, n, n)); uy = rng.standard_normal((k, n, n))
    ux[:, :, -1] = 0; uy[:, -1, :] = 0
    gx, gy = oracle.grad(phi)
    lhs = np.sum(gx * ux + gy * uy)
    rhs = -np.sum(phi * oracle.div(ux, uy))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_spatial_laplacian_bound():
    # lambda_max(-Delta_x) for the Neumann grid is (4 - 4 cos(pi (n-1)/n))/h^2 < 8/h^2
    n = 9
    N = n * n
    M = np.zeros((N, N))
    for q in range(N):
        e = np.zeros((1, n, n)); e.flat[q] = 1.0
        gx, gy = oracle.grad(e)
        M[:, q] = -oracle.div(gx, gy).ravel()
    lm = np.linalg.eigvalsh(0.5 * (M + M.T)).max()
    h = 1.0 / (n - 1)
    # 1D Neumann path Laplacian: 2 - 2cos(pi p/n); the 2D grid adds one per direction
    assert lm == pytest.approx(2 * (2 - 2 * np.cos(np.pi * (n - 1) / n)) / h ** 2, rel=1e-9)
    assert lm < 8.0 / h ** 2


# ------------------------------------------------------------------ Section 4.1
def _read_L():
    vals = []
    with open(os.path.join(GOLDEN, "dti_L.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#") or line.startswith("L"):
                continue
            vals.append([float(x) for x in line.split()])
    return np.array(vals).reshape(2, 3, 3)


def test_quantum_div_is_minus_adjoint_and_maps_sym_to_skew():
    rng = np.random.default_rng(3)
    L = S.random_L(3, 3, seed=5)
    n = 3
    X = rng.standard_normal((9, n, n))
    Z = rng.standard_normal((27, n, n))
    lhs = np.sum(oracle.grad_L(X, L) * Z)
    rhs = -np.sum(X * oracle.div_L(Z, L))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # symmetric X -> skew gradient; skew Z -> symmetric divergence
    Xs = X.reshape(3, 3, n, n); Xs = (Xs + Xs.transpose(1, 0, 2, 3)).reshape(9, n, n)
    G = oracle.grad_L(Xs, L).reshape(3, 3, 3, n, n)
    np.testing.assert_allclose(G, -G.transpose(0, 2, 1, 3, 4), atol=1e-14)
    Zs = Z.reshape(3, 3, 3, n, n); Zs = (Zs - Zs.transpose(0, 2, 1, 3, 4)).reshape(27, n, n)
    Y = oracle.div_L(Zs, L).reshape(3, 3, n, n)
    np.testing.assert_allclose(Y, Y.transpose(1, 0, 2, 3), atol=1e-14)


def test_quantum_laplacian_matrix_matches_operator():
    """The k^2 x k^2 matrix of Section 7.3 equals -div_L grad_L applied column by column."""
    for L in (_read_L(), S.random_L(3, 3, seed=11)):
        M = oracle.neg_quantum_laplacian(L)
        cols = []
        for q in range(9):
            E = np.zeros((9, 1, 1)); E[q] = 1.0
            cols.append(-oracle.div_L(oracle.grad_L(E, L), L).ravel())
        np.testing.assert_allclose(M, np.array(cols).T, atol=1e-13)
        assert oracle.quantum_lmax(L) == pytest.approx(np.linalg.eigvalsh(M).max(), rel=1e-12)


def test_quantum_kernel_assumption():
    # the paper's L_1, L_2 satisfy ker grad_L = span{I} on symmetric matrices
    assert oracle.quantum_sym_gap(_read_L()) > 1e-3
    # a single diagonal L with a repeated eigenvalue does not (E_01 + E_10 commutes with it)
    assert abs(oracle.quantum_sym_gap(np.diag([1.0, 1.0, 0.0])[None])) < 1e-12
    # the identity is always in the kernel
    I = np.eye(3).reshape(9, 1, 1)
    assert np.abs(oracle.grad_L(I, _read_L())).max() < 1e-15


# ------------------------------------------------------------------ Appendix B
def test_shrinks_satisfy_prox_optimality():
    rng = np.random.default_rng(4)
    for _ in range(200):
        m = int(rng.integers(1, 7))
        x = rng.standard_normal(m) * rng.uniform(0.1, 3)
        t = rng.uniform(0.05, 2.0)
        z = oracle.shrink2(x, t)
        if np.linalg.norm(z) > 0:
            # 0 = t z/||z|| + z - x
            np.testing.assert_allclose(t * z / np.linalg.norm(z) + z - x, 0, atol=1e-12)
        else:
            assert np.linalg.norm(x) <= t + 1e-15
        s = oracle.shrink1(x[0], t)
        if s != 0:
            assert t * np.sign(s) + s - x[0] == pytest.approx(0, abs=1e-12)
        else:
            assert abs(x[0]) <= t
    # brute force: the shrink minimises t||z|| + 0.5||z - x||^2
    from scipy.optimize import minimize
    x = np.array([0.7, -1.3, 0.4]); t = 0.5
    f = lambda z: t * np.linalg.norm(z) + 0.5 * np.sum((z - x) ** 2)
    z = oracle.shrink2(x, t)
    best = minimize(f, x, method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-14, maxiter=20000))
    assert f(z) <= best.fun + 1e-10
    # boundary cases: ||x|| = t and x = 0 give 0 without dividing by zero
    np.testing.assert_array_equal(oracle.shrink2(np.array([0.6, 0.8]), 1.0), 0.0)
    np.testing.assert_array_equal(oracle.shrink2(np.zeros(3), 0.1), 0.0)


# ------------------------------------------------------------------ Sections 7.1-7.2
def test_step_size_rules():
    mu, nu = oracle.step_sizes(32, 1.0, oracle.graph_lmax(3, K3), True)
    assert mu == 1.0 / (32 * 31 ** 2) and nu == pytest.approx(1.0 / 12.0, rel=1e-15)
    mu1, _ = oracle.step_sizes(32, 2.0, 0.0, False)
    assert mu1 == 1.0 / (16 * 2.0 * 31 ** 2)
    # both rules satisfy the PDHG condition 1 > tau mu lmax(-Dx) + tau nu lmax(-DG) using 8(n-1)^2
    assert 1.0 > 1.0 * mu * 8 * 31 ** 2 + 1.0 * nu * 3.0
    assert 1.0 > 2.0 * mu1 * 8 * 31 ** 2


def test_single_channel_vector_iteration_is_scalar_box():
    rng = np.random.default_rng(6)
    n = 10
    r0 = rng.uniform(0.1, 1, (1, n, n)); r0 /= r0.sum()
    r1 = rng.uniform(0.1, 1, (1, n, n)); r1 /= r1.sum()
    v = oracle.vomt_solve(r0, r1, [], alpha=1.0, tau=2.0, max_iters=57, check_every=57)
    s = oracle.somt_run(r0[0], r1[0], tau=2.0, iters=57)
    assert v["mu"] == s["mu"]
    np.testing.assert_array_equal(v["phi"][0], s["phi"])
    np.testing.assert_array_equal(v["ux"][0], s["ux"])
    np.testing.assert_array_equal(v["uy"][0], s["uy"])


def test_one_dimensional_closed_form():
    """Densities constant in y: the optimal cost is Delta x * Sum |F0 - F1| (cumulative masses)."""
    rng = np.random.default_rng(7)
    n = 10
    a = rng.uniform(0.2, 1.0, n); b = rng.uniform(0.2, 1.0, n)
    r0 = np.tile(a, (n, 1))[None]; r0 /= r0.sum()
    r1 = np.tile(b, (n, 1))[None]; r1 /= r1.sum()
    F = np.cumsum(r0[0] - r1[0], axis=1)
    exact = (1.0 / (n - 1)) * np.abs(F).sum()
    o = oracle.vomt_solve(r0, r1, [], tau=10.0, max_iters=300000, check_every=200, tol_gap=1e-9, tol_res=1e-9)
    m = o["metrics"]
    assert m["primal"] == pytest.approx(exact, rel=2e-6)
    assert m["dual"] == pytest.approx(exact, rel=2e-6)


@pytest.mark.parametrize("alpha", [0.1, 1.0, 10.0])
def test_shifted_blob_costs_mass_times_shift(alpha):
    n, k, s = 12, 3, 2
    r0, r1 = S.shifted_blob_pair(n, k, s, sigma=1.0, margin=2)
    exact = s / (n - 1)                  # unit mass moved s cells of width 1/(n-1)
    o = oracle.vomt_solve(r0, r1, K3, alpha=alpha, tau=10.0, max_iters=200000, check_every=100,
                          tol_gap=1e-8, tol_res=1e-8)
    m = o["metrics"]
    assert m["dual"] <= exact * (1 + 1e-6) + m["dual_infeas"] * 10   # weak duality (up to infeasibility)
    assert m["primal"] == pytest.approx(exact, rel=5e-6)
    assert m["dual"] == pytest.approx(exact, rel=5e-6)


@pytest.mark.parametrize("alpha", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("w_norm", [oracle.W_L1, oracle.W_L2])
def test_pure_recolor_closed_form(alpha, w_norm):
    """rho e_p -> rho e_q on K3 (c = 1): alpha * mass * (shortest path) for ||w||_1 and
    alpha * mass * sqrt(delta^T L_G^+ delta) = alpha sqrt(2/3) for ||w||_2."""
    rng = np.random.default_rng(8)
    n, k = 8, 3
    rho = rng.uniform(0.2, 1.0, (n, n)); rho /= rho.sum()
    r0 = np.zeros((k, n, n)); r1 = np.zeros((k, n, n))
    r0[0] = rho; r1[2] = rho
    exact = alpha * (1.0 if w_norm == oracle.W_L1 else np.sqrt(2.0 / 3.0))
    o = oracle.vomt_solve(r0, r1, K3, alpha=alpha, tau=3.0, w_norm=w_norm, max_iters=20000,
                          check_every=50, tol_gap=1e-10, tol_res=1e-10)
    m = o["metrics"]
    assert m["primal"] == pytest.approx(exact, rel=1e-8)
    assert m["dual"] == pytest.approx(exact, rel=1e-8)
    # dV/dalpha = Sum ||w*|| = exact / alpha
    _, _, ga = oracle.envelope_grad(o["phi"], o["w"], w_norm)
    assert ga == pytest.approx(exact / alpha, rel=1e-7)
    # a longer path costs more: with edge {0,2} removed the path 0-1-2 has length 2
    o2 = oracle.vomt_solve(r0, r1, [(0, 1), (1, 2)], alpha=alpha, tau=3.0, w_norm=oracle.W_L1,
                           max_iters=40000, check_every=50, tol_gap=1e-10, tol_res=1e-10)
    assert o2["metrics"]["primal"] == pytest.approx(2 * alpha, rel=1e-7)


def _assemble_constraint(k, n, edges):
    """Sparse matrix of u, w -> div_x u + div_G w (Appendix A, Section 3.1), assembled entry by
    entry from the definitions, over the real (non-ghost) unknowns only.  Returns the matrix,
    the variable keys in column order and the row index function."""
    from scipy.sparse import lil_matrix
    ih = n - 1.0
    var = {}
    for c in range(k):
        for j in range(n):
            for i in range(n - 1):
                var[("x", c, j, i)] = len(var)
    for c in range(k):
        for j in range(n - 1):
            for i in range(n):
                var[("y", c, j, i)] = len(var)
    for e in range(len(edges)):
        for j in range(n):
            for i in range(n):
                var[("w", e, j, i)] = len(var)
    A = lil_matrix((k * n * n, len(var)))
    row = lambda c, j, i: (c * n + j) * n + i
    for (t, c, j, i), v in var.items():
        if t == "x":       # u_x,ij enters div at (i,j) with +1/h and at (i+1,j) with -1/h
            entries = [(row(c, j, i), ih), (row(c, j, i + 1), -ih)]
        elif t == "y":
            entries = [(row(c, j, i), ih), (row(c, j + 1, i), -ih)]
        else:
            a, b = edges[c]
            lo, hi = min(a, b), max(a, b)
            entries = [(row(lo, j, i), -1.0), (row(hi, j, i), 1.0)]   # div_G w = -D w
        for r, val in entries:
            A[r, v] += val
    return A.tocsr(), list(var.keys())


def _lp_value(r0, r1, edges, alpha):
    """min Sum|u_x| + Sum|u_y| + alpha Sum|w| s.t. div_x u + div_G w = rho0 - rho1, by HiGHS."""
    from scipy.optimize import linprog
    from scipy.sparse import hstack
    k, n = r0.shape[0], r0.shape[-1]
    A, keys = _assemble_constraint(k, n, edges)
    cost = np.array([alpha if key[0] == "w" else 1.0 for key in keys])
    res = linprog(np.concatenate([cost, cost]), A_eq=hstack([A, -A]).tocsr(), b_eq=(r0 - r1).ravel(),
                  bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


def test_iteration_matches_generic_pdhg():
    """Section 6.1 states PDHG for L(x, y, z) = f(x) + g(y) + <Ax + By, z> - h(z).  With
    f = ||.||_1, g = alpha ||.||_1, h(z) = <rho0 - rho1, z> and A, B the assembled sparse
    divergence operators, its iterates must equal the oracle's V-OMT iterates (||u||_1, ||w||_1)."""
    n, k, T = 5, 3, 60
    r0, r1 = S.blob_pair(n, k, seed=61)
    alpha, tau = 0.7, 2.0
    A, keys = _assemble_constraint(k, n, K3)
    isw = np.array([key[0] == "w" for key in keys])
    o = oracle.vomt_solve(r0, r1, K3, alpha=alpha, tau=tau, u_norm=oracle.U_L1, w_norm=oracle.W_L1,
                          max_iters=T, check_every=T)
    mu, nu = o["mu"], o["nu"]
    Ax, By = A[:, ~isw], A[:, isw]
    x = np.zeros((~isw).sum()); y = np.zeros(isw.sum()); z = np.zeros(k * n * n)
    soft = lambda v, t: np.sign(v) * np.maximum(np.abs(v) - t, 0.0)
    for _ in range(T):
        # x-step: argmin ||x||_1 + <Ax, z> + |x - x^k|^2/(2 mu) = soft(x^k - mu A^T z^k, mu)
        xn = soft(x - mu * (Ax.T @ z), mu)
        yn = soft(y - nu * (By.T @ z), alpha * nu)
        # z-step: argmax <A xbar + B ybar, z> - <rho0 - rho1, z> - |z - z^k|^2/(2 tau)
        z = z + tau * (Ax @ (2 * xn - x) + By @ (2 * yn - y) - (r0 - r1).ravel())
        x, y = xn, yn
    np.testing.assert_allclose(o["phi"].ravel(), z, rtol=0, atol=1e-12 * np.abs(z).max())
    ux = np.array([o["ux"][c, j, i] if t == "x" else o["uy"][c, j, i] if t == "y" else o["w"][c, j, i]
                   for (t, c, j, i) in keys])
    np.testing.assert_allclose(ux[~isw], x, rtol=0, atol=1e-12 * np.abs(x).max())
    np.testing.assert_allclose(ux[isw], y, rtol=0, atol=1e-12 * max(np.abs(y).max(), 1e-300))


@pytest.mark.parametrize("alpha", [0.3, 2.0])
def test_l1_norms_match_linear_program(alpha):
    n, k = 5, 3
    r0, r1 = S.blob_pair(n, k, seed=21)
    lp = _lp_value(r0, r1, K3, alpha)
    o = oracle.vomt_solve(r0, r1, K3, alpha=alpha, tau=3.0, u_norm=oracle.U_L1, w_norm=oracle.W_L1,
                          max_iters=400000, check_every=100, tol_gap=1e-10, tol_res=1e-10)
    assert o["metrics"]["primal"] == pytest.approx(lp, rel=1e-7)
    assert o["metrics"]["dual"] == pytest.approx(lp, rel=1e-7)


def test_iteration_invariants():
    n, k = 16, 3
    r0, r1 = S.blob_pair(n, k, seed=31)
    o = oracle.vomt_solve(r0, r1, K3, alpha=1.0, max_iters=400, check_every=1, history=True)
    h = o["history"]
    R = h[:, 4]
    assert np.all(R >= -1e-18)
    assert np.all(np.diff(R) <= 1e-12 * R[0])        # fixed-point residual is monotone (Section 6.1)
    assert abs(o["phi"].sum()) < 1e-12                 # Sum phi stays 0: Sum div = Sum div_G = Sum b = 0
    assert np.all(o["ux"][:, :, -1] == 0) and np.all(o["uy"][:, -1, :] == 0)   # ghost cells
    div = oracle.div(o["ux"], o["uy"])
    assert np.abs(div.sum(axis=(1, 2))).max() < 1e-14  # zero-flux: no mass leaves a channel in space
    # longer runs drive gap and residual down (strong duality, Section 3.3)
    o2 = oracle.vomt_solve(r0, r1, K3, alpha=1.0, tau=10.0, max_iters=20000, check_every=1000, history=True)
    assert o2["history"][-1, 2] < 1e-3 and o2["history"][-1, 3] < 1e-3
    assert o2["history"][-1, 3] < o2["history"][0, 3]


def test_metric_axioms():
    n, k = 7, 3
    rng = np.random.default_rng(9)
    dens = []
    for _ in range(3):
        d = rng.uniform(0.05, 1.0, (k, n, n)); dens.append(d / d.sum())
    V = {}
    kw = dict(alpha=1.0, tau=3.0, max_iters=400000, check_every=200, tol_gap=1e-8, tol_res=1e-8)
    for a in range(3):
        for b in range(3):
            if a != b:
                V[a, b] = oracle.vomt_solve(dens[a], dens[b], K3, **kw)["metrics"]["primal"]
    for a in range(3):
        for b in range(3):
            if a < b:
                assert V[a, b] == pytest.approx(V[b, a], rel=1e-5)
    for a, b, c in [(0, 1, 2), (1, 2, 0), (2, 0, 1)]:
        assert V[a, c] <= V[a, b] + V[b, c] + 1e-6
    same = oracle.vomt_solve(dens[0], dens[0], K3, max_iters=50, check_every=50)
    assert same["metrics"]["primal"] == 0.0


# ------------------------------------------------------------------ Section 7.3
def _iso(rho, k):
    M = np.zeros((k * k,) + rho.shape)
    for a in range(k):
        M[a * k + a] = rho / k
    return M


def test_matrix_isotropic_shift_closed_form():
    """Lam = rho I / k moved s cells: M = S(rho0, rho1)/sqrt(k) under ||U||_2 (any alpha)."""
    n, k, s = 10, 3, 2
    b0, b1 = S.shifted_blob_pair(n, 1, s, sigma=1.0, margin=2)
    L = _read_L()
    exact = (s / (n - 1)) / np.sqrt(k)
    for alpha in (0.3, 3.0):
        o = oracle.momt_solve(_iso(b0[0], k), _iso(b1[0], k), L, alpha=alpha, tau=10.0,
                              max_iters=200000, check_every=200, tol_gap=1e-8, tol_res=1e-8)
        assert o["metrics"]["primal"] == pytest.approx(exact, rel=1e-5)
        assert o["metrics"]["dual"] == pytest.approx(exact, rel=1e-5)


def _g_L(delta, L):
    """min ||W||_1 s.t. div_L W = delta over W in (R^{k x k})^N, by LP (Section 4.1 operator
    written out per entry)."""
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


def test_matrix_pure_reshape_is_linear_in_alpha():
    """Lam0 = rho A, Lam1 = rho B at the same place: M = alpha * mass * g_L(A - B)."""
    n, k = 6, 3
    L = _read_L()
    rng = np.random.default_rng(10)
    rho = rng.uniform(0.3, 1.0, (n, n)); rho /= rho.sum()
    A = np.diag([0.6, 0.3, 0.1]); th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    B = R @ A @ R.T
    Lam0 = (A.reshape(9, 1, 1) * rho[None]); Lam1 = (B.reshape(9, 1, 1) * rho[None])
    g = _g_L(A - B, L)
    for alpha in (0.1, 1.0):
        o = oracle.momt_solve(Lam0, Lam1, L, alpha=alpha, tau=10.0, max_iters=200000, check_every=200,
                              tol_gap=1e-9, tol_res=1e-9)
        assert o["metrics"]["primal"] == pytest.approx(alpha * g, rel=1e-6)
        assert o["metrics"]["dual"] == pytest.approx(alpha * g, rel=1e-6)


def test_table2_pattern_is_consistent_with_closed_forms():
    """Table 2: the moved-ellipsoid column does not depend on alpha and the reshaped-ellipsoid
    column is proportional to alpha, as the two closed forms above predict."""
    T = _read_golden_matrix("table2_pattern.txt")
    alpha, m01, m02 = T[:, 0], T[:, 1], T[:, 2]
    assert np.ptp(m02) == 0.0
    np.testing.assert_allclose(m01 / alpha, 0.27, rtol=0.01)


def test_matrix_iteration_keeps_structure():
    n, k = 8, 3
    L = S.random_L(3, 3, seed=12)
    T0, T1 = S.tensor_field_pair(n, k, seed=13)
    o = oracle.momt_solve(T0, T1, L, alpha=1.0, max_iters=200, check_every=1, history=True)
    P = o["Phi"].reshape(3, 3, n, n)
    np.testing.assert_allclose(P, P.transpose(1, 0, 2, 3), atol=1e-15)
    W = o["W"].reshape(3, 3, 3, n, n)
    np.testing.assert_allclose(W, -W.transpose(0, 2, 1, 3, 4), atol=1e-15)
    R = o["history"][:, 4]
    assert np.all(np.diff(R) <= 1e-12 * R[0])
    assert abs(np.trace(P).sum()) < 1e-13


# ------------------------------------------------------------------ gradients
def _J(r0, r1, alpha, T):
    o = oracle.vomt_solve(r0, r1, K3, alpha=alpha, tau=3.0, max_iters=T, check_every=T)
    return o["metrics"]["primal"]


def test_unrolled_gradient_matches_finite_differences():
    n, k, T = 6, 3, 40
    r0, r1 = S.blob_pair(n, k, seed=41)
    J, g1, g0, ga = oracle.unrolled_grad(r0, r1, K3, 1.0, T, tau=3.0)
    assert J == pytest.approx(_J(r0, r1, 1.0, T), rel=1e-14)
    h = 1e-7
    ok = 0
    dirs = S.mass_preserving_directions(r1, 8, seed=42)
    for d in dirs:
        fd = (_J(r0, r1 + h * d, 1.0, T) - _J(r0, r1 - h * d, 1.0, T)) / (2 * h)
        ok += abs(fd - np.sum(g1 * d)) <= 1e-5 * (abs(fd) + 1e-12)
    assert ok >= 7
    for d in S.mass_preserving_directions(r0, 4, seed=43):
        fd = (_J(r0 + h * d, r1, 1.0, T) - _J(r0 - h * d, r1, 1.0, T)) / (2 * h)
        assert np.sum(g0 * d) == pytest.approx(fd, rel=1e-5, abs=1e-12)
    fda = (_J(r0, r1, 1.0 + 1e-6, T) - _J(r0, r1, 1.0 - 1e-6, T)) / 2e-6
    assert ga == pytest.approx(fda, rel=1e-5)


def test_envelope_gradient_matches_finite_differences():
    n, k = 6, 3
    r0, r1 = S.blob_pair(n, k, seed=51)
    kw = dict(alpha=1.0, tau=3.0, max_iters=600000, check_every=200, tol_gap=1e-11, tol_res=1e-11)
    o = oracle.vomt_solve(r0, r1, K3, **kw)
    g1, g0, ga = oracle.envelope_grad(o["phi"], o["w"])
    assert abs(g1.sum()) < 1e-12
    h = 1e-4
    agree = 0
    dirs = S.mass_preserving_directions(r1, 6, seed=52)
    for d in dirs:
        Vp = oracle.vomt_solve(r0, r1 + h * d, K3, **kw)["metrics"]["primal"]
        Vm = oracle.vomt_solve(r0, r1 - h * d, K3, **kw)["metrics"]["primal"]
        fd = (Vp - Vm) / (2 * h)
        agree += abs(fd - np.sum(g1 * d)) <= 1e-3 * abs(fd) + 1e-9
    assert agree >= 5
