"""GPU gradients of the transport cost against the FP64 oracle.

Envelope gradient (vomt_backward): the kernel equals the oracle's envelope
formula on the same converged iterate, and its directional derivatives agree
with central finite differences of the oracle's converged cost.  Unrolled
gradient (vomt_unrolled_grad): against the oracle's reverse-mode gradient of the
same T-iteration map, and against central finite differences of that map."""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")
A = pytest.importorskip("paper_1712_10279_gb300.autograd")

K3 = S.COMPLETE_K3


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _t(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(_dev())


def test_envelope_kernel_matches_oracle_formula():
    r0, r1 = S.blob_pair(24, 3, seed=31)
    sol = V.solve(_t(r0), _t(r1), K3, 1.0, max_iters=3000, check_every=500)
    rho0 = _t(r0).requires_grad_(True)
    rho1 = _t(r1).requires_grad_(True)
    alpha = torch.tensor(1.0, device=_dev(), dtype=torch.float64, requires_grad=True)
    cost = A.transport_cost(rho0, rho1, K3, alpha, max_iters=3000, check_every=500)
    (2.5 * cost).backward()
    assert float(cost) == pytest.approx(sol.result["primal"], rel=1e-12)
    g1, g0, ga = oracle.envelope_grad(sol.phi.cpu().numpy().astype(np.float64), sol.w.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(rho1.grad.cpu().numpy(), 2.5 * g1, rtol=0, atol=1e-6 * np.abs(g1).max())
    np.testing.assert_allclose(rho0.grad.cpu().numpy(), 2.5 * g0, rtol=0, atol=1e-6 * np.abs(g0).max())
    assert float(alpha.grad) == pytest.approx(2.5 * ga, rel=1e-5)
    assert abs(float(rho1.grad.double().sum())) < 1e-4 * float(rho1.grad.abs().sum())


def test_envelope_dalpha_recolor_closed_form():
    """rho e_0 -> rho e_2 on K3: V = alpha * mass, so dV/dalpha = 1."""
    n = 10
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.2, 1.0, (n, n)); rho /= rho.sum()
    r0 = np.zeros((3, n, n)); r1 = np.zeros((3, n, n)); r0[0] = rho; r1[2] = rho
    alpha = torch.tensor(0.7, device=_dev(), dtype=torch.float64, requires_grad=True)
    cost = A.transport_cost(_t(r0), _t(r1), K3, alpha, tau=3.0, max_iters=20000, check_every=100,
                            tol_gap=1e-6, tol_res=1e-6)
    cost.backward()
    assert float(cost) == pytest.approx(0.7, rel=1e-4)
    assert float(alpha.grad) == pytest.approx(1.0, rel=1e-4)


def test_envelope_directional_derivatives_match_finite_differences():
    """32 mass-preserving directions (the differentiable configuration's count); central
    differences (h = 1e-4) of the FP64 oracle's optimal value, each perturbed solve warm-started
    from the unperturbed optimum and run to gap 1e-11.  V is piecewise linear in rho1 where the
    optimal phi is not unique, so a few directions may sit on a kink."""
    n = 8
    r0, r1 = S.blob_pair(n, 3, seed=51)
    rho1 = _t(r1).requires_grad_(True)
    cost = A.transport_cost(_t(r0), rho1, K3, 1.0, tau=3.0, max_iters=200000, check_every=500, tol_gap=2e-6,
                            tol_res=2e-6)
    cost.backward()
    g = rho1.grad.cpu().numpy().astype(np.float64)
    kw = dict(alpha=1.0, tau=3.0, max_iters=600000, check_every=200, tol_gap=1e-11, tol_res=1e-11)
    base = oracle.vomt_solve(r0, r1, K3, **kw)
    init = {x: base[x] for x in ("ux", "uy", "w", "phi")}
    h = 1e-4
    agree = 0
    dirs = S.mass_preserving_directions(r1, 32, seed=52)
    for d in dirs:
        Vp = oracle.vomt_solve(r0, r1 + h * d, K3, init=init, **kw)["metrics"]["primal"]
        Vm = oracle.vomt_solve(r0, r1 - h * d, K3, init=init, **kw)["metrics"]["primal"]
        fd = (Vp - Vm) / (2 * h)
        agree += abs(fd - np.sum(g * d)) <= 1e-2 * abs(fd) + 1e-7
    assert agree >= 28, agree


def test_batched_forward_backward():
    d = _dev()
    B, n = 4, 20
    pairs = [S.blob_pair(n, 3, seed=60 + q) for q in range(B)]
    r0 = torch.stack([_t(p[0]) for p in pairs])
    r1 = torch.stack([_t(p[1]) for p in pairs]).requires_grad_(True)
    costs = A.transport_cost(r0, r1, K3, 1.0, engine="batched", max_iters=800, check_every=200)
    costs.sum().backward()
    for q in range(B):
        sol = V.solve(r0[q], r1[q].detach(), K3, 1.0, max_iters=800, check_every=200, engine="stream")
        assert float(costs[q]) == pytest.approx(sol.result["primal"], rel=1e-6)
        g1, _, _ = oracle.envelope_grad(sol.phi.cpu().numpy().astype(np.float64), sol.w.cpu().numpy().astype(np.float64))
        assert _rel(r1.grad[q].cpu().numpy(), g1) < 1e-4
    assert d.type == "cuda"


def _kink_margin(r0, r1, T, tau, w_norm, alpha=1.0):
    """Smallest relative distance |arg - threshold| / threshold over the T iterations of the
    oracle's map from zero, over every shrink of Appendix B the iteration applies (per-channel
    ||(u_x, u_y) + mu grad phi|| against mu, and |w + nu grad_G phi| or its norm against alpha nu).
    The unrolled map is smooth wherever this stays away from 0."""
    k, n = r0.shape[0], r0.shape[-1]
    o = oracle.vomt_solve(r0, r1, K3, alpha, tau=tau, max_iters=1, check_every=1)
    mu, nu = o["mu"], o["nu"]
    st = dict(ux=np.zeros((k, n, n)), uy=np.zeros((k, n, n)), w=np.zeros((3, n, n)), phi=np.zeros((k, n, n)))
    m = np.inf
    for _ in range(T):
        gx, gy = oracle.grad(st["phi"])
        s = np.hypot(st["ux"] + mu * gx, st["uy"] + mu * gy)
        m = min(m, float(np.min(np.abs(s - mu) / mu)))
        x = st["w"] + nu * oracle.grad_G(st["phi"], K3)
        a = np.abs(x) if w_norm == 0 else np.linalg.norm(x, axis=0)
        m = min(m, float(np.min(np.abs(a - alpha * nu) / (alpha * nu))))
        o = oracle.vomt_solve(r0, r1, K3, alpha, tau=tau, max_iters=1, check_every=1, init=st, w_norm=w_norm)
        st = {q: o[q] for q in ("ux", "uy", "w", "phi")}
    return m


@pytest.mark.parametrize("n,T", [(8, 30), (16, 10)])
@pytest.mark.parametrize("w_norm", [0, 1])
def test_unrolled_gradient_matches_oracle_away_from_kinks(n, T, w_norm):
    """Where no shrink argument comes near its threshold (checked in the oracle: at least 1%
    away, while FP32 perturbs arguments by about 1e-6 relative), the FP32 reverse mode equals
    the FP64 oracle's to the parity bar, 1e-3 relative L2."""
    r0, r1 = S.blob_pair(n, 3, seed=41)
    r0d, r1d = r0.astype(np.float32).astype(np.float64), r1.astype(np.float32).astype(np.float64)
    assert _kink_margin(r0d, r1d, T, 3.0, w_norm) > 1e-2
    J, d0, d1, da = A.unrolled_grad(_t(r0), _t(r1), K3, 1.0, T=T, ckpt=10, tau=3.0, w_norm=w_norm)
    Jo, g1, g0, gao = oracle.unrolled_grad(r0d, r1d, K3, 1.0, T, tau=3.0, w_norm=w_norm)
    assert J == pytest.approx(Jo, rel=1e-5)
    assert _rel(d1.cpu().numpy().astype(np.float64), g1) < 1e-3
    assert _rel(d0.cpu().numpy().astype(np.float64), g0) < 1e-3
    assert da == pytest.approx(gao, rel=1e-3)


@pytest.mark.parametrize("w_norm", [0, 1])
def test_unrolled_gradient_matches_oracle(w_norm):
    """16 x 16, T = 60: here some shrink argument passes within 3e-5 (relative) of its
    threshold (_kink_margin), so FP32 rounding can put a point on the other side of a kink for
    an iteration; the bar is 1e-2 relative L2 for this kinked case."""
    n, T = 16, 60
    r0, r1 = S.blob_pair(n, 3, seed=41)
    J, d0, d1, da = A.unrolled_grad(_t(r0), _t(r1), K3, 1.0, T=T, ckpt=20, tau=3.0, w_norm=w_norm)
    r0d, r1d = r0.astype(np.float32).astype(np.float64), r1.astype(np.float32).astype(np.float64)
    Jo, g1, g0, gao = oracle.unrolled_grad(r0d, r1d, K3, 1.0, T, tau=3.0, w_norm=w_norm)
    assert J == pytest.approx(Jo, rel=1e-5)
    assert _rel(d1.cpu().numpy().astype(np.float64), g1) < 1e-2
    assert _rel(d0.cpu().numpy().astype(np.float64), g0) < 1e-2
    assert da == pytest.approx(gao, rel=1e-2)


def test_unrolled_directional_derivatives_match_finite_differences():
    """32 mass-preserving directions; central differences (h = 1e-4) of the oracle's own
    T-iteration map.  Report-style check: most directions within 1e-2 relative (the map is
    piecewise smooth, and a direction may cross a shrink kink)."""
    n, T = 12, 40
    r0, r1 = S.blob_pair(n, 3, seed=42)
    r0 = r0.astype(np.float32).astype(np.float64)
    r1 = r1.astype(np.float32).astype(np.float64)
    _, _, d1, _ = A.unrolled_grad(_t(r0), _t(r1), K3, 1.0, T=T, ckpt=20, tau=3.0)
    g = d1.cpu().numpy().astype(np.float64)
    h = 1e-4

    def Jmap(rr1):
        return oracle.vomt_solve(r0, rr1, K3, 1.0, tau=3.0, max_iters=T, check_every=T)["metrics"]["primal"]

    ok = 0
    for d in S.mass_preserving_directions(r1, 32, seed=43):
        fd = (Jmap(r1 + h * d) - Jmap(r1 - h * d)) / (2 * h)
        ok += abs(fd - np.sum(g * d)) <= 1e-2 * abs(fd) + 1e-9
    assert ok >= 28, ok


def test_unrolled_cost_autograd_at_256():
    """The 256 x 256 colour-image size with T = 200 and checkpoints every 20 iterations:
    the autograd wrapper's gradient equals the oracle's reverse-mode gradient of the same map."""
    r0, r1 = S.color_image_pair(256, 3, seed=1005)
    rho1 = _t(r1).requires_grad_(True)
    J = A.unrolled_cost(_t(r0), rho1, K3, 1.0, T=200, ckpt=20)
    J.backward()
    Jo, g1, _, _ = oracle.unrolled_grad(r0.astype(np.float32).astype(np.float64),
                                       r1.astype(np.float32).astype(np.float64), K3, 1.0, 200)
    assert float(J) == pytest.approx(Jo, rel=1e-4)
    assert _rel(rho1.grad.cpu().numpy().astype(np.float64), g1) < 1e-2
