"""Pins for two of the oracle's convergence measures that the iteration itself never uses:
the fixed-point residual R of Section 6.1 and the dual infeasibility of the dual problem
(eq. (vomt-dual) of Section 3.3 and its matrix analogue of Section 4).

R is checked against the squared norm of the last step in the PDHG metric
    M = [[I/mu, 0, -A^T], [0, I/nu, -B^T], [-A, -B, I/tau]]
with A (spatial divergence) and B (graph or quantum divergence) assembled here as sparse
matrices entry by entry from Appendix A, Section 3.1 and Section 4.1, independently of the
oracle's operator code.  The y-block weight is 1/nu: Section 6.1 prints 1/mu there, a
typo (the metric above is the one in which PDHG is a proximal-point method), so a wrong
weight fails these tests.

The dual infeasibility max_x max(||grad phi||_{u*} - 1, ||grad_G phi||_{w*} - alpha, 0) is
checked on potentials whose gradients are known in closed form: piecewise-linear ramps
(spatial term) and channel offsets constant in space (graph term), for the dual of every
u-norm (per-channel Euclidean maximum, joint Euclidean, entrywise maximum) and w-norm
(maximum modulus, Euclidean).
"""
import numpy as np
import pytest
from scipy import sparse

import oracle
from paper_1712_10279_gb300 import synthetic as S


# ------------------------------------------------------------------ assembled operators
def _div1d(n):
    """n x n backward difference of Appendix A for one axis, times 1/h: flux entry i
    (i < n-1, the face between cells i and i+1) enters cell i with +1/h and cell i+1 with
    -1/h; entry n-1 is the ghost face and enters nothing."""
    ih = n - 1.0
    D = sparse.lil_matrix((n, n))
    for i in range(n - 1):
        D[i, i] += ih
        D[i + 1, i] -= ih
    return D.tocsr()


def _spatial_div_2d(n, planes):
    """[ux; uy] (planes x n x n each, x fastest) -> div, as a sparse matrix."""
    I = sparse.identity(n, format="csr")
    dx = sparse.kron(I, _div1d(n))          # acts on the x index (fastest)
    dy = sparse.kron(_div1d(n), I)
    Ip = sparse.identity(planes, format="csr")
    return sparse.hstack([sparse.kron(Ip, dx), sparse.kron(Ip, dy)]).tocsr()


def _spatial_div_3d(n, planes):
    I = sparse.identity(n, format="csr")
    d = _div1d(n)
    dx = sparse.kron(I, sparse.kron(I, d))
    dy = sparse.kron(I, sparse.kron(d, I))
    dz = sparse.kron(d, sparse.kron(I, I))
    Ip = sparse.identity(planes, format="csr")
    return sparse.hstack([sparse.kron(Ip, dx), sparse.kron(Ip, dy), sparse.kron(Ip, dz)]).tocsr()


def _graph_div(k, edges, cost, npts):
    """w ([l][points]) -> div_G w = -D diag(1/c) w ([k][points]); D has +1 at the smaller
    node and -1 at the larger node of each edge (Section 3.1)."""
    l = len(edges)
    Dc = np.zeros((k, l))
    for e, (a, b) in enumerate(edges):
        lo, hi = min(a, b), max(a, b)
        Dc[lo, e] = 1.0 / cost[e]
        Dc[hi, e] = -1.0 / cost[e]
    return sparse.kron(sparse.csr_matrix(-Dc), sparse.identity(npts, format="csr")).tocsr()


def _quantum_div_point(L):
    """Z = (Z_s)_s (row-major k x k each) -> sum_s (Z_s L_s - L_s Z_s) (Section 4.1) as a
    k^2 x N k^2 matrix: for row-major vec, vec(L Z) = (L kron I) vec Z and
    vec(Z L) = (I kron L^T) vec Z."""
    N, k = L.shape[0], L.shape[1]
    I = np.eye(k)
    return np.hstack([-np.kron(L[s], I) + np.kron(I, L[s].T) for s in range(N)])


def _metric_norm2(dx, dy, dz, A, B, mu, nu, tau):
    """Delta^T M Delta with M = [[I/mu, 0, -A^T], [0, I/nu, -B^T], [-A, -B, I/tau]]
    assembled as one sparse block matrix (complex blocks use the real inner product)."""
    nx, ny, nz = dx.size, dy.size, dz.size
    blocks = [[sparse.identity(nx) / mu, None, -A.conj().T],
              [None, sparse.identity(ny) / nu if ny else None, -B.conj().T if ny else None],
              [-A, -B if ny else None, sparse.identity(nz) / tau]]
    if not ny:
        blocks = [[blocks[0][0], blocks[0][2]], [blocks[2][0], blocks[2][2]]]
        s = np.concatenate([dx, dz])
    else:
        s = np.concatenate([dx, dy, dz])
    M = sparse.bmat(blocks, format="csr")
    return float(np.real(np.vdot(s, M @ s)))


def _last_step(solve, init, **kw):
    """One more iteration from the state `init` with a check after it: the check's R is
    computed from the new state and `init`."""
    o = solve(init=init, max_iters=1, check_every=1, history=True, **kw)
    return o, o["history"][-1]


# ------------------------------------------------------------------ R, vector OMT (2-D)
@pytest.mark.parametrize("u_norm", [oracle.U_L12, oracle.U_L2, oracle.U_L1])
@pytest.mark.parametrize("w_norm", [oracle.W_L1, oracle.W_L2])
def test_fixed_point_residual_is_pdhg_metric_norm(u_norm, w_norm):
    n, k = 6, 3
    edges = [(0, 1), (0, 2), (1, 2)]
    cost = np.array([1.0, 1.7, 0.6])
    r0, r1 = S.blob_pair(n, k, seed=71)
    r0, r1 = r0 * n * n, r1 * n * n          # unit mean mass: the flux and w move within a few steps
    kw = dict(edges=edges, alpha=0.4, tau=2.0, cost=cost, u_norm=u_norm, w_norm=w_norm)
    mid = oracle.vomt_solve(r0, r1, max_iters=17, check_every=17, **kw)
    st = {x: mid[x] for x in ("ux", "uy", "w", "phi")}
    o, row = _last_step(lambda **a: oracle.vomt_solve(r0, r1, **a), st, **kw)
    assert np.abs(o["w"] - st["w"]).max() > 0.0          # the w block takes part
    A = _spatial_div_2d(n, k)
    B = _graph_div(k, edges, cost, n * n)
    dx = np.concatenate([(o["ux"] - st["ux"]).ravel(), (o["uy"] - st["uy"]).ravel()])
    dy = (o["w"] - st["w"]).ravel()
    dz = (o["phi"] - st["phi"]).ravel()
    ref = _metric_norm2(dx, dy, dz, A, B, o["mu"], o["nu"], o["tau"])
    assert ref > 0.0
    assert row[4] == pytest.approx(ref, rel=1e-11)
    # the same number from the metrics entry point, given both states
    met = oracle.vomt_metrics(o, st, r0, r1, edges, kw["alpha"], o["mu"], o["nu"], o["tau"], cost=cost,
                              u_norm=u_norm, w_norm=w_norm)
    assert met[4] == pytest.approx(ref, rel=1e-11)
    # the printed weight 1/mu on the y block would give a different number
    wrong = ref - (dy @ dy) / o["nu"] + (dy @ dy) / o["mu"]
    assert abs(wrong - ref) > 1e-3 * ref


def test_fixed_point_residual_without_edges():
    """k = 1 (no graph): M reduces to [[I/mu, -A^T], [-A, I/tau]] (the S-OMT metric)."""
    n = 7
    r0, r1 = S.blob_pair(n, 1, seed=72)
    r0, r1 = r0 * n * n, r1 * n * n
    kw = dict(edges=[], alpha=1.0, tau=1.5)
    mid = oracle.vomt_solve(r0, r1, max_iters=9, check_every=9, **kw)
    st = {x: mid[x] for x in ("ux", "uy", "w", "phi")}
    o, row = _last_step(lambda **a: oracle.vomt_solve(r0, r1, **a), st, **kw)
    A = _spatial_div_2d(n, 1)
    dx = np.concatenate([(o["ux"] - st["ux"]).ravel(), (o["uy"] - st["uy"]).ravel()])
    dz = (o["phi"] - st["phi"]).ravel()
    ref = _metric_norm2(dx, np.zeros(0), dz, A, None, o["mu"], 1.0, o["tau"])
    assert row[4] == pytest.approx(ref, rel=1e-11)


# ------------------------------------------------------------------ R, matrix OMT (2-D)
@pytest.mark.parametrize("u_norm,w_norm", [(oracle.U_L2, oracle.W_L1), (oracle.U_NUC, oracle.W_L2),
                                           (oracle.U_L1, oracle.W_NUC)])
def test_matrix_fixed_point_residual_is_pdhg_metric_norm(u_norm, w_norm):
    n, k = 5, 3
    L0, L1 = S.tensor_field_pair(n, k, seed=73)
    L0, L1 = L0 * n * n, L1 * n * n
    L = S.random_L(k, 2, seed=73)
    kw = dict(L=L, alpha=0.5, tau=5.0, u_norm=u_norm, w_norm=w_norm)
    mid = oracle.momt_solve(L0, L1, max_iters=13, check_every=13, **kw)
    st = {x: mid[x] for x in ("Ux", "Uy", "W", "Phi")}
    o, row = _last_step(lambda **a: oracle.momt_solve(L0, L1, **a), st, **kw)
    assert np.abs(o["W"] - st["W"]).max() > 0.0
    kk = k * k
    A = _spatial_div_2d(n, kk)
    B = sparse.kron(sparse.csr_matrix(_quantum_div_point(L)), sparse.identity(n * n)).tocsr()
    # W planes are [s][entry][points]: column s*kk + q of the point matrix, point-major blocks
    dx = np.concatenate([(o["Ux"] - st["Ux"]).ravel(), (o["Uy"] - st["Uy"]).ravel()])
    dy = (o["W"] - st["W"]).ravel()
    dz = (o["Phi"] - st["Phi"]).ravel()
    ref = _metric_norm2(dx, dy, dz, A, B, o["mu"], o["nu"], o["tau"])
    assert row[4] == pytest.approx(ref, rel=1e-11)
    met = oracle.momt_metrics(o, st, L0, L1, L, kw["alpha"], o["mu"], o["nu"], o["tau"],
                              u_norm=u_norm, w_norm=w_norm)
    assert met[4] == pytest.approx(ref, rel=1e-11)


# ------------------------------------------------------------------ R, 3-D grids
def test_volume_fixed_point_residual_is_pdhg_metric_norm():
    n, k = 4, 3
    edges = [(0, 1), (0, 2), (1, 2)]
    r0, r1 = S.blob_pair3(n, k, seed=74)
    r0, r1 = r0 * n ** 3, r1 * n ** 3
    kw = dict(edges=edges, alpha=0.3, tau=2.0)
    mid = oracle.vomt3_solve(r0, r1, max_iters=11, check_every=11, **kw)
    st = {x: mid[x] for x in ("ux", "uy", "uz", "w", "phi")}
    o, row = _last_step(lambda **a: oracle.vomt3_solve(r0, r1, **a), st, **kw)
    A = _spatial_div_3d(n, k)
    B = _graph_div(k, edges, np.ones(3), n ** 3)
    dx = np.concatenate([(o[c] - st[c]).ravel() for c in ("ux", "uy", "uz")])
    dy = (o["w"] - st["w"]).ravel()
    dz = (o["phi"] - st["phi"]).ravel()
    ref = _metric_norm2(dx, dy, dz, A, B, o["mu"], o["nu"], o["tau"])
    assert row[4] == pytest.approx(ref, rel=1e-11)


def test_matrix_volume_fixed_point_residual_is_pdhg_metric_norm():
    n, k = 4, 2
    L0, L1 = S.tensor_field_pair3(n, k, seed=75)
    L0, L1 = L0 * n ** 3, L1 * n ** 3
    L = S.random_L(k, 3, seed=75)
    kw = dict(L=L, alpha=0.5, tau=4.0)
    mid = oracle.momt3_solve(L0, L1, max_iters=9, check_every=9, **kw)
    st = {x: mid[x] for x in ("Ux", "Uy", "Uz", "W", "Phi")}
    o, row = _last_step(lambda **a: oracle.momt3_solve(L0, L1, **a), st, **kw)
    A = _spatial_div_3d(n, k * k)
    B = sparse.kron(sparse.csr_matrix(_quantum_div_point(L)), sparse.identity(n ** 3)).tocsr()
    dx = np.concatenate([(o[c] - st[c]).ravel() for c in ("Ux", "Uy", "Uz")])
    dy = (o["W"] - st["W"]).ravel()
    dz = (o["Phi"] - st["Phi"]).ravel()
    ref = _metric_norm2(dx, dy, dz, A, B, o["mu"], o["nu"], o["tau"])
    assert row[4] == pytest.approx(ref, rel=1e-11)


def test_complex_fixed_point_residual_is_pdhg_metric_norm():
    """Complex Hermitian fields: the metric uses the real inner product Re <x, y> of
    Section 4's Hilbert-Schmidt geometry; div_L is complex linear, so its matrix is the
    complex analogue of the real one."""
    n, k = 4, 2
    L0, L1 = S.hermitian_field_pair(n, k, seed=76)
    L0, L1 = L0 * n * n, L1 * n * n
    L = S.random_hermitian_L(k, 2, seed=76)
    kw = dict(L=L, alpha=0.5, tau=4.0)
    mid = oracle.zmomt_solve(L0, L1, max_iters=7, check_every=7, **kw)
    st = {x: mid[x] for x in ("Ux", "Uy", "W", "Phi")}
    o, row = _last_step(lambda **a: oracle.zmomt_solve(L0, L1, **a), st, **kw)
    kk = k * k
    A = _spatial_div_2d(n, kk).astype(np.complex128)
    B = sparse.kron(sparse.csr_matrix(_quantum_div_point(np.asarray(L))), sparse.identity(n * n)).tocsr()
    dx = np.concatenate([(o["Ux"] - st["Ux"]).ravel(), (o["Uy"] - st["Uy"]).ravel()])
    dy = (o["W"] - st["W"]).ravel()
    dz = (o["Phi"] - st["Phi"]).ravel()
    ref = _metric_norm2(dx, dy, dz, A, B, o["mu"], o["nu"], o["tau"])
    assert row[4] == pytest.approx(ref, rel=1e-11)


# ------------------------------------------------------------------ dual infeasibility
def _zero_state(k, l, n):
    return dict(ux=np.zeros((k, n, n)), uy=np.zeros((k, n, n)), w=np.zeros((l, n, n)))


def _ramp(n, k, a, b, a2=None):
    """phi_c(x, y) = a_c x + b_c y on the grid x = i h, y = j h (h = 1/(n-1)); with a2 the
    x-slope is a2_c on the cells right of the middle (a kink in x)."""
    h = 1.0 / (n - 1)
    i = np.arange(n)
    phi = np.zeros((k, n, n))
    for c in range(k):
        if a2 is None:
            fx = a[c] * i * h
        else:
            m = n // 2
            fx = np.where(i <= m, a[c] * i * h, a[c] * m * h + a2[c] * (i - m) * h)
        phi[c] = fx[None, :] + b[c] * (i * h)[:, None]
    return phi


@pytest.mark.parametrize("u_norm", [oracle.U_L12, oracle.U_L2, oracle.U_L1])
def test_dual_infeasibility_of_spatial_ramps(u_norm):
    """A linear phi_c = a_c x + b_c y has grad phi_c = (a_c, b_c) at every cell that has both
    forward neighbours; the dual norms of Section 6.2's u-norms at such a point are
    max_c |(a_c, b_c)|_2 (||u||_{1,2}), |(a, b)|_2 over all channels (||u||_2) and
    max_c max(|a_c|, |b_c|) (||u||_1).  alpha is large, so the graph term stays inactive."""
    n, k = 9, 3
    a = np.array([1.5, -0.4, 0.9])
    b = np.array([0.7, 1.3, -1.1])
    phi = _ramp(n, k, a, b)
    st = dict(_zero_state(k, 3, n), phi=phi)
    z = np.zeros((k, n, n))
    expect = {oracle.U_L12: np.max(np.hypot(a, b)),
              oracle.U_L2: np.sqrt(np.sum(a * a + b * b)),
              oracle.U_L1: np.max(np.maximum(np.abs(a), np.abs(b)))}[u_norm]
    met = oracle.vomt_metrics(st, None, z, z, S.COMPLETE_K3, 1e6, 1.0, 1.0, 1.0, u_norm=u_norm)
    assert met[5] == pytest.approx(max(expect - 1.0, 0.0), rel=1e-12, abs=1e-13)
    # a kinked ramp: the maximum over points, not a sum or a mean, decides
    a2 = np.array([2.5, 0.1, -0.2])
    phi2 = _ramp(n, k, a, b, a2=a2)
    st2 = dict(st, phi=phi2)
    steep = {oracle.U_L12: np.max(np.hypot(a2, b)),
             oracle.U_L2: np.sqrt(np.sum(a2 * a2 + b * b)),
             oracle.U_L1: np.max(np.maximum(np.abs(a2), np.abs(b)))}[u_norm]
    met2 = oracle.vomt_metrics(st2, None, z, z, S.COMPLETE_K3, 1e6, 1.0, 1.0, 1.0, u_norm=u_norm)
    assert met2[5] == pytest.approx(max(expect, steep) - 1.0, rel=1e-12)
    # inside the dual ball: zero
    met3 = oracle.vomt_metrics(dict(st, phi=_ramp(n, k, 0.3 * a / np.abs(a).max(), 0.3 * b / np.abs(b).max())),
                               None, z, z, S.COMPLETE_K3, 1e6, 1.0, 1.0, 1.0, u_norm=u_norm)
    assert met3[5] == 0.0


@pytest.mark.parametrize("w_norm", [oracle.W_L1, oracle.W_L2])
def test_dual_infeasibility_of_channel_offsets(w_norm):
    """phi_c = o_c constant in space: grad phi = 0, and grad_G phi on edge e = (p < q) is
    (o_p - o_q) / c_e at every point (Section 3.1), so the graph term is
    max_e |(o_p - o_q)/c_e| - alpha (||w||_1, dual max-modulus) or
    |((o_p - o_q)/c_e)_e|_2 - alpha (||w||_2)."""
    n, k = 6, 4
    edges = [(0, 1), (1, 2), (2, 3), (0, 3), (1, 3)]
    cost = np.array([1.0, 0.5, 2.0, 1.3, 0.8])
    o_c = np.array([0.3, -0.9, 1.4, 0.2])
    phi = np.broadcast_to(o_c[:, None, None], (k, n, n)).copy()
    st = dict(_zero_state(k, len(edges), n), phi=phi)
    z = np.zeros((k, n, n))
    g = np.array([(o_c[min(p, q)] - o_c[max(p, q)]) / cost[e] for e, (p, q) in enumerate(edges)])
    dual = np.abs(g).max() if w_norm == oracle.W_L1 else np.linalg.norm(g)
    for alpha in (0.25, 0.9 * dual, 2.0 * dual):
        met = oracle.vomt_metrics(st, None, z, z, edges, alpha, 1.0, 1.0, 1.0, cost=cost, w_norm=w_norm)
        assert met[5] == pytest.approx(max(dual - alpha, 0.0), rel=1e-12, abs=1e-15)


def test_dual_infeasibility_takes_the_larger_term():
    """Both terms active: the measure is the larger excess, spatial or graph."""
    n, k = 8, 3
    a = np.array([1.2, 0.0, 0.0])
    b = np.zeros(3)
    phi = _ramp(n, k, a, b) + np.array([0.0, 0.5, -0.5])[:, None, None]
    st = dict(_zero_state(k, 3, n), phi=phi)
    z = np.zeros((k, n, n))
    # spatial excess 0.2; graph values phi_p - phi_q range over the grid, the largest |.| is
    # on edge (1, 2): 1.0 everywhere, and on edge (0, 2) 0.5 + 1.2 x at most 1.7 (x = 1)
    for alpha, expect in ((1.0, 0.7), (1.6, 0.2), (1.45, 0.25)):
        met = oracle.vomt_metrics(st, None, z, z, S.COMPLETE_K3, alpha, 1.0, 1.0, 1.0)
        assert met[5] == pytest.approx(expect, rel=1e-12)


def _sym(rng, k):
    X = rng.normal(size=(k, k))
    return X + X.T


@pytest.mark.parametrize("u_norm", [oracle.U_L2, oracle.U_L1, oracle.U_NUC])
def test_matrix_dual_infeasibility_of_spatial_ramps(u_norm):
    """Phi = A x + B y with symmetric A, B has grad Phi = (A, B) at interior cells; the dual
    norms (Section 6.2) are |(A, B)|_F (||U||_2), the largest entry modulus (||U||_1) and
    max(spectral A, spectral B) (||U||_{1,nuc})."""
    n, k = 6, 3
    rng = np.random.default_rng(5)
    A, B = _sym(rng, k), _sym(rng, k)
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    Phi = (A.reshape(k * k, 1, 1) * x[None, None, :] + B.reshape(k * k, 1, 1) * x[None, :, None])
    st = dict(Ux=np.zeros((k * k, n, n)), Uy=np.zeros((k * k, n, n)), W=np.zeros((2 * k * k, n, n)), Phi=Phi)
    L = S.random_L(k, 2, seed=5)
    z = np.zeros((k * k, n, n))
    expect = {oracle.U_L2: np.sqrt(np.sum(A * A) + np.sum(B * B)),
              oracle.U_L1: max(np.abs(A).max(), np.abs(B).max()),
              oracle.U_NUC: max(np.linalg.norm(A, 2), np.linalg.norm(B, 2))}[u_norm]
    met = oracle.momt_metrics(st, None, z, z, L, 1e6, 1.0, 1.0, 1.0, u_norm=u_norm)
    assert met[5] == pytest.approx(expect - 1.0, rel=1e-10)


@pytest.mark.parametrize("w_norm", [oracle.W_L1, oracle.W_L2, oracle.W_NUC])
def test_matrix_dual_infeasibility_of_constant_field(w_norm):
    """A constant symmetric Phi = C has grad Phi = 0 and grad_L Phi = (L_s C - C L_s)_s at every
    cell (Section 4.1); the dual norms are the largest entry modulus (||W||_1), the joint
    Frobenius norm (||W||_2) and max_s spectral(.) (||W||_{1,nuc})."""
    n, k = 5, 3
    rng = np.random.default_rng(6)
    C = _sym(rng, k)
    L = S.random_L(k, 3, seed=6)
    G = [L[s] @ C - C @ L[s] for s in range(3)]
    dual = {oracle.W_L1: max(np.abs(g).max() for g in G),
            oracle.W_L2: np.sqrt(sum(np.sum(g * g) for g in G)),
            oracle.W_NUC: max(np.linalg.norm(g, 2) for g in G)}[w_norm]
    Phi = np.broadcast_to(C.reshape(k * k, 1, 1), (k * k, n, n)).copy()
    st = dict(Ux=np.zeros((k * k, n, n)), Uy=np.zeros((k * k, n, n)), W=np.zeros((3 * k * k, n, n)), Phi=Phi)
    z = np.zeros((k * k, n, n))
    for alpha in (0.5 * dual, 0.95 * dual, 1.5 * dual):
        met = oracle.momt_metrics(st, None, z, z, L, alpha, 1.0, 1.0, 1.0, u_norm=oracle.U_L2, w_norm=w_norm)
        assert met[5] == pytest.approx(max(dual - alpha, 0.0), rel=1e-10, abs=1e-14)
