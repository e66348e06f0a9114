"""Pins of the quadratically regularised oracle (the paper's concluding section):
objective sum_x ||u||_u + alpha ||w||_w + eps (||u||_2^2 + ||w||_2^2), Euclidean norms in
the regulariser.  Each check is independent of the oracle's own arithmetic:

* one iteration from a random state satisfies the optimality conditions of the two
  proximal steps (checked with a numpy gradient written here);
* densities constant in y (k = 1): the unique regularised optimum is the 1-D flux, so
  the cost is sum (|F| h + eps (F h)^2) in closed form;
* the duality gap with the regularised dual closes, and two different starting points
  reach the same (unique) solution;
* eps = 0 reproduces the plain iteration bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

K3 = S.COMPLETE_K3


def _grad(phi):
    """Forward differences times (n - 1), zero in the ghost row / column (Appendix A)."""
    n = phi.shape[-1]
    gx = np.zeros_like(phi)
    gy = np.zeros_like(phi)
    gx[..., :, :-1] = (phi[..., :, 1:] - phi[..., :, :-1]) * (n - 1)
    gy[..., :-1, :] = (phi[..., 1:, :] - phi[..., :-1, :]) * (n - 1)
    return gx, gy


@pytest.mark.parametrize("eps", [0.5, 20.0])
def test_one_step_satisfies_regularised_prox_conditions(eps):
    rng = np.random.default_rng(3)
    n, k = 7, 3
    r0, r1 = S.blob_pair(n, k, seed=8)
    init = dict(ux=rng.normal(0, 1e-2, (k, n, n)), uy=rng.normal(0, 1e-2, (k, n, n)),
                w=rng.normal(0, 1e-2, (3, n, n)), phi=rng.normal(0, 1.0, (k, n, n)))
    init["ux"][:, :, -1] = 0.0
    init["uy"][:, -1, :] = 0.0
    alpha = 0.7
    o = oracle.vomt_solve(r0, r1, K3, alpha, tau=1.0, max_iters=1, check_every=1, init=init, eps=eps)
    mu, nu = o["mu"], o["nu"]
    gx, gy = _grad(init["phi"])
    # u: per channel 2-vector z minimising mu ||z|| + mu eps ||z||^2 + |z - v|^2 / 2
    vx, vy = init["ux"] + mu * gx, init["uy"] + mu * gy
    zx, zy = o["ux"], o["uy"]
    nz = np.hypot(zx, zy)
    nv = np.hypot(vx, vy)
    on = nz > 0
    assert np.all(nv[~on] <= mu * (1 + 1e-12))
    rx = mu * zx[on] / nz[on] + 2 * mu * eps * zx[on] + zx[on] - vx[on]
    ry = mu * zy[on] / nz[on] + 2 * mu * eps * zy[on] + zy[on] - vy[on]
    assert np.abs(rx).max() < 1e-12 and np.abs(ry).max() < 1e-12
    assert on.sum() > 10
    # w (||.||_1): entrywise, nu alpha sign(z) + 2 nu eps z + z - v = 0, or |v| <= nu alpha at z = 0
    D = np.array([[1, 1, 0], [-1, 0, 1], [0, -1, -1]], dtype=float)   # K3 incidence, edges (0,1),(0,2),(1,2)
    gG = np.einsum("ce,cij->eij", D, init["phi"])
    v = init["w"] + nu * gG
    z = o["w"]
    on = z != 0
    assert np.all(np.abs(v[~on]) <= nu * alpha * (1 + 1e-12))
    r = nu * alpha * np.sign(z[on]) + 2 * nu * eps * z[on] + z[on] - v[on]
    assert np.abs(r).max() < 1e-12 and on.sum() > 10


@pytest.mark.parametrize("eps", [0.0, 1.0, 10.0])
def test_regularised_one_dimensional_closed_form(eps):
    """k = 1, densities constant in y: for eps > 0 the optimum is unique and is the 1-D flux
    u_x = F h, u_y = 0 (for a fixed column sum, sum_j |t_j| + eps t_j^2 is least when all t_j
    are equal), so P = sum (|F| h + eps (F h)^2)."""
    rng = np.random.default_rng(17)
    n = 10
    a = rng.uniform(0.2, 1.0, n); b = rng.uniform(0.2, 1.0, n)
    r0 = np.tile(a, (n, 1))[None]; r0 /= r0.sum()
    r1 = np.tile(b, (n, 1))[None]; r1 /= r1.sum()
    F = np.cumsum(r0[0] - r1[0], axis=1)
    h = 1.0 / (n - 1)
    exact = np.sum(np.abs(F) * h + eps * (F * h) ** 2)
    o = oracle.vomt_solve(r0, r1, [], tau=10.0, max_iters=400000, check_every=200, tol_gap=1e-10, tol_res=1e-10,
                          eps=eps)
    m = o["metrics"]
    assert m["primal"] == pytest.approx(exact, rel=2e-6)
    assert m["dual"] == pytest.approx(exact, rel=2e-6)
    if eps > 0:
        np.testing.assert_allclose(o["ux"][0][:, :-1], (F * h)[:, :-1], rtol=0, atol=1e-6 * np.abs(F * h).max())
        assert np.abs(o["uy"]).max() < 1e-6 * np.abs(F * h).max()


def test_regularised_gap_closes_and_solution_is_unique():
    n = 12
    r0, r1 = S.blob_pair(n, 3, seed=21)
    kw = dict(tau=3.0, max_iters=300000, check_every=200, tol_gap=1e-9, tol_res=1e-9, eps=2.0)
    a = oracle.vomt_solve(r0, r1, K3, 1.0, **kw)
    rng = np.random.default_rng(5)
    init = dict(ux=rng.normal(0, 1e-2, (3, n, n)), uy=rng.normal(0, 1e-2, (3, n, n)),
                w=rng.normal(0, 1e-2, (3, n, n)), phi=rng.normal(0, 1.0, (3, n, n)))
    init["ux"][:, :, -1] = 0.0
    init["uy"][:, -1, :] = 0.0
    b = oracle.vomt_solve(r0, r1, K3, 1.0, init=init, **kw)
    for o in (a, b):
        assert o["metrics"]["converged"] == 1.0
        assert o["metrics"]["rel_gap"] <= 1e-9
    assert a["metrics"]["primal"] == pytest.approx(b["metrics"]["primal"], rel=1e-8)
    scale = np.abs(a["ux"]).max()
    for f in ("ux", "uy", "w"):
        np.testing.assert_allclose(a[f], b[f], rtol=0, atol=1e-5 * scale)
    # the regularised cost exceeds the plain optimum by at most eps times the plain solution's
    # squared norm, and is at least the plain optimum
    p0 = oracle.vomt_solve(r0, r1, K3, 1.0, tau=3.0, max_iters=300000, check_every=200, tol_gap=1e-9, tol_res=1e-9)
    q0 = sum(np.sum(p0[f] ** 2) for f in ("ux", "uy", "w"))
    assert p0["metrics"]["primal"] * (1 - 1e-6) <= a["metrics"]["primal"] <= p0["metrics"]["primal"] + 2.0 * q0 * (1 + 1e-6)


def test_eps_zero_is_the_plain_iteration():
    r0, r1 = S.blob_pair(9, 3, seed=2)
    a = oracle.vomt_solve(r0, r1, K3, 1.0, max_iters=300, check_every=100)
    b = oracle.vomt_solve(r0, r1, K3, 1.0, max_iters=300, check_every=100, eps=0.0)
    for f in ("ux", "uy", "w", "phi"):
        np.testing.assert_array_equal(a[f], b[f])
