"""Pins of the 3-D oracle (the discretization of Appendix A with a third direction).

* the 3-D divergence is minus the adjoint of the 3-D gradient (ghost entries zero), and
  the gradient of a linear field is its slope away from the ghosts;
* densities that vary along x only cost h sum |F0 - F1| over every (y, z) line;
* a density moved s cells in x costs mass x shift for every alpha (k = 3, K3);
* densities constant in z cost exactly the 2-D optimum of one slice (a 3-D flux summed over
  z is a 2-D flux of no larger cost, and the z-constant 2-D solution is feasible), computed
  by the independent 2-D oracle;
* iteration invariants: ghosts stay zero, the fixed-point residual does not increase.
"""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

K3 = S.COMPLETE_K3


def test_div3_is_minus_adjoint_of_grad3():
    rng = np.random.default_rng(0)
    n, k = 5, 2
    phi = rng.standard_normal((k, n, n, n))
    ux, uy, uz = (rng.standard_normal((k, n, n, n)) for _ in range(3))
    ux[..., -1] = 0.0
    uy[..., -1, :] = 0.0
    uz[:, -1] = 0.0
    gx, gy, gz = oracle.grad3(phi)
    lhs = np.sum(gx * ux) + np.sum(gy * uy) + np.sum(gz * uz)
    rhs = -np.sum(phi * oracle.div3(ux, uy, uz))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_grad3_of_linear_field():
    n = 6
    h = 1.0 / (n - 1)
    z, y, x = np.meshgrid(*(np.arange(n) * h,) * 3, indexing="ij")
    phi = (0.3 * x - 1.2 * y + 2.0 * z)[None]
    gx, gy, gz = oracle.grad3(phi)
    np.testing.assert_allclose(gx[0][..., :-1], 0.3, rtol=1e-12)
    np.testing.assert_allclose(gy[0][:, :-1, :], -1.2, rtol=1e-12)
    np.testing.assert_allclose(gz[0][:-1], 2.0, rtol=1e-12)
    assert np.all(gx[0][..., -1] == 0) and np.all(gy[0][:, -1, :] == 0) and np.all(gz[0][-1] == 0)


def test_one_dimensional_closed_form_3d():
    rng = np.random.default_rng(7)
    n = 7
    a = rng.uniform(0.2, 1.0, n); b = rng.uniform(0.2, 1.0, n)
    r0 = np.broadcast_to(a, (n, n, n)).copy()[None]; r0 /= r0.sum()
    r1 = np.broadcast_to(b, (n, n, n)).copy()[None]; r1 /= r1.sum()
    F = np.cumsum(r0[0] - r1[0], axis=-1)
    exact = (1.0 / (n - 1)) * np.abs(F).sum()
    o = oracle.vomt3_solve(r0, r1, [], tau=10.0, max_iters=300000, check_every=200, tol_gap=1e-9, tol_res=1e-9)
    assert o["metrics"]["primal"] == pytest.approx(exact, rel=2e-6)
    assert o["metrics"]["dual"] == pytest.approx(exact, rel=2e-6)


@pytest.mark.parametrize("alpha", [0.3, 3.0])
def test_shifted_density_costs_mass_times_shift_3d(alpha):
    n, s = 8, 2
    rng = np.random.default_rng(3)
    base = np.zeros((3, n, n, n))
    base[:, 2:6, 2:6, 1:4] = rng.uniform(0.5, 1.0, (3, 4, 4, 3))
    base /= base.sum()
    moved = np.zeros_like(base)
    moved[..., s:] = base[..., :n - s]
    o = oracle.vomt3_solve(base, moved, K3, alpha, tau=10.0, max_iters=300000, check_every=200, tol_gap=1e-8,
                           tol_res=1e-8)
    assert o["metrics"]["primal"] == pytest.approx(s / (n - 1), rel=5e-6)


def test_z_constant_densities_cost_the_2d_optimum():
    n = 8
    r0, r1 = S.blob_pair(n, 3, seed=12)
    kw = dict(tau=3.0, max_iters=400000, check_every=200, tol_gap=1e-9, tol_res=1e-9)
    two = oracle.vomt_solve(r0, r1, K3, 1.0, **kw)
    r0_3 = np.repeat(r0[:, None], n, axis=1) / n
    r1_3 = np.repeat(r1[:, None], n, axis=1) / n
    three = oracle.vomt3_solve(r0_3, r1_3, K3, 1.0, **kw)
    assert three["metrics"]["primal"] == pytest.approx(two["metrics"]["primal"], rel=1e-6)


def test_iteration_invariants_3d():
    n = 6
    rng = np.random.default_rng(4)
    r0 = rng.uniform(0.2, 1.0, (3, n, n, n)); r0 /= r0.sum()
    r1 = rng.uniform(0.2, 1.0, (3, n, n, n)); r1 /= r1.sum()
    o = oracle.vomt3_solve(r0, r1, K3, 1.0, max_iters=2000, check_every=100, history=True)
    assert np.all(o["ux"][..., -1] == 0) and np.all(o["uy"][..., -1, :] == 0) and np.all(o["uz"][:, -1] == 0)
    R = o["history"][:, 4]
    assert np.all(np.diff(R) <= 1e-12 * R[0])
    assert abs(o["phi"].sum()) < 1e-9 * np.abs(o["phi"]).sum()
