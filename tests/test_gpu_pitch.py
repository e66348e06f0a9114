"""Row pitch (the `pitch` of the boundary's grid arrays): every grid array may have rows of
n floats at a larger row pitch, e.g. views into padded buffers.  A pitched solve must give
the dense solve's result bit for bit (the library stages pitched arrays densely), leave the
row padding of the outputs untouched, and refuse a pitch below n.  Covered: vomt_solve
(cold and warm start), vomt_solve_host, momt_solve and vomt_backward."""
import ctypes

import numpy as np
import pytest

from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")
_native = V._native

K3 = S.COMPLETE_K3


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _padded(a, pitch, fill, dev):
    """[planes, n, n] array -> (padded [planes, n, pitch] tensor, view [planes, n, n])."""
    a = torch.as_tensor(np.asarray(a, np.float32))
    big = torch.full(a.shape[:-1] + (pitch,), fill, dtype=torch.float32, device=dev)
    big[..., :a.shape[-1]] = a.to(dev)
    return big, big[..., :a.shape[-1]]


def _call_solve(n, k, edges, r0, r1, pitch, warm=None, iters=300, tau=None):
    dev = _dev()
    lib = _native.load()
    g = _native.GraphArg(k, edges)
    l = g.tail.size
    b0, _ = _padded(r0, pitch, 7.0, dev)
    b1, _ = _padded(r1, pitch, 7.0, dev)
    if warm is None:
        bu = torch.full((2 * k, n, pitch), float("nan"), device=dev)
        bw = torch.full((max(l, 1), n, pitch), float("nan"), device=dev)
        bp = torch.full((k, n, pitch), float("nan"), device=dev)
    else:
        bu, _ = _padded(warm[0].reshape(2 * k, n, n).cpu().numpy(), pitch, float("nan"), dev)
        bw, _ = _padded(warm[1].cpu().numpy() if l else np.zeros((1, n, n)), pitch, float("nan"), dev)
        bp, _ = _padded(warm[2].cpu().numpy(), pitch, float("nan"), dev)
    p = V._params(tau, None, None, 0, 0, iters, 100, 0.0, 0.0, warm is not None, "auto", pitch=pitch)
    res = _native.Result()
    ctx = _native.context(0)
    rc = lib.vomt_solve(ctx, n, b0.data_ptr(), b1.data_ptr(), g.ref, 1.0, ctypes.byref(p), bu.data_ptr(),
                        bw.data_ptr() if l else None, bp.data_ptr(), ctypes.byref(res),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, bu, bw[:l], bp, res.as_dict()


@pytest.mark.parametrize("n,pitch", [(37, 40), (64, 96), (30, 31)])
def test_pitched_vector_solve_equals_dense(n, pitch):
    dev = _dev()
    r0, r1 = S.blob_pair(n, 3, seed=n)
    d0 = torch.from_numpy(r0.astype(np.float32)).to(dev)
    d1 = torch.from_numpy(r1.astype(np.float32)).to(dev)
    ref = V.solve(d0, d1, K3, 1.0, max_iters=300, check_every=100)
    rc, bu, bw, bp, res = _call_solve(n, 3, K3, r0, r1, pitch)
    assert rc == 0
    assert torch.equal(bp[..., :n], ref.phi)
    assert torch.equal(bu[..., :n].reshape(2, 3, n, n), ref.u)
    assert torch.equal(bw[..., :n], ref.w)
    assert res["primal"] == ref.result["primal"] and res["iters"] == 300
    for b in (bu, bw, bp):                       # the padding is never written
        assert torch.isnan(b[..., n:]).all()
    # warm start from pitched iterates continues the same trajectory
    ref2 = V.solve(d0, d1, K3, 1.0, max_iters=200, check_every=100, init=(ref.u, ref.w, ref.phi))
    rc, bu, bw, bp, res = _call_solve(n, 3, K3, r0, r1, pitch, warm=(ref.u, ref.w, ref.phi), iters=200)
    assert rc == 0
    assert torch.equal(bp[..., :n], ref2.phi)
    assert torch.equal(bu[..., :n].reshape(2, 3, n, n), ref2.u)


def test_pitched_host_solve_equals_dense():
    n, k, pitch = 33, 3, 36
    r0, r1 = S.blob_pair(n, k, seed=4)
    ref = V.solve_host(r0.astype(np.float32), r1.astype(np.float32), K3, 1.0, max_iters=200, check_every=100)
    lib = _native.load()
    g = _native.GraphArg(k, K3)
    h0 = np.full((k, n, pitch), 5.0, np.float32); h0[..., :n] = r0
    h1 = np.full((k, n, pitch), 5.0, np.float32); h1[..., :n] = r1
    hu = np.full((2 * k, n, pitch), np.nan, np.float32)
    hw = np.full((3, n, pitch), np.nan, np.float32)
    hp = np.full((k, n, pitch), np.nan, np.float32)
    p = V._params(None, None, None, 0, 0, 200, 100, 0.0, 0.0, False, "auto", pitch=pitch)
    res = _native.Result()
    rc = lib.vomt_solve_host(_native.context(0), n, h0.ctypes.data, h1.ctypes.data, g.ref, 1.0, ctypes.byref(p),
                             hu.ctypes.data, hw.ctypes.data, hp.ctypes.data, ctypes.byref(res), None)
    assert rc == 0
    assert np.array_equal(hp[..., :n], np.asarray(ref.phi))
    assert np.array_equal(hu[..., :n].reshape(2, k, n, n), np.asarray(ref.u))
    assert np.isnan(hp[..., n:]).all() and np.isnan(hu[..., n:]).all()


def test_pitched_matrix_solve_equals_dense():
    dev = _dev()
    n, k, N, pitch = 20, 3, 3, 24
    L0, L1 = S.tensor_field_pair(n, k, seed=8)
    L = S.random_L(k, N, seed=8)
    m0 = torch.from_numpy(L0.astype(np.float32)).to(dev)
    m1 = torch.from_numpy(L1.astype(np.float32)).to(dev)
    ref = V.momt_solve(m0, m1, L, 1.0, max_iters=200, check_every=100)
    lib = _native.load()
    b0, _ = _padded(L0, pitch, 3.0, dev)
    b1, _ = _padded(L1, pitch, 3.0, dev)
    kk = k * k
    bU = torch.full((2 * kk, n, pitch), float("nan"), device=dev)
    bW = torch.full((N * kk, n, pitch), float("nan"), device=dev)
    bP = torch.full((kk, n, pitch), float("nan"), device=dev)
    p = V._params(None, None, None, 1, 0, 200, 100, 0.0, 0.0, False, "auto", pitch=pitch)
    res = _native.Result()
    Lh = np.ascontiguousarray(L, np.float64)
    rc = lib.momt_solve(_native.context(0), n, k, b0.data_ptr(), b1.data_ptr(), N, Lh.ctypes.data, 1.0,
                        ctypes.byref(p), bU.data_ptr(), bW.data_ptr(), bP.data_ptr(), ctypes.byref(res),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.equal(bP[..., :n], ref.Phi)
    assert torch.equal(bU[..., :n].reshape(2, kk, n, n), ref.U)
    assert torch.equal(bW[..., :n].reshape(N, kk, n, n), ref.W)
    assert torch.isnan(bP[..., n:]).all() and torch.isnan(bW[..., n:]).all()


def test_pitched_envelope_backward_equals_dense():
    dev = _dev()
    B, k, l, n, pitch = 2, 3, 3, 19, 24
    rng = np.random.default_rng(3)
    phi = rng.normal(size=(B, k, n, n)).astype(np.float32)
    w = rng.normal(size=(B, l, n, n)).astype(np.float32)
    lib = _native.load()
    ctx = _native.context(0)

    def run(pitch_):
        P = torch.full((B, k, n, pitch_), float("nan"), device=dev); P[..., :n] = torch.from_numpy(phi).to(dev)
        Wt = torch.full((B, l, n, pitch_), float("nan"), device=dev); Wt[..., :n] = torch.from_numpy(w).to(dev)
        g0 = torch.full((B, k, n, pitch_), float("nan"), device=dev)
        g1 = torch.full((B, k, n, pitch_), float("nan"), device=dev)
        ga = torch.zeros(B, device=dev)
        rc = lib.vomt_backward(ctx, B, n, pitch_, k, l, 0, P.data_ptr(), Wt.data_ptr(), None, g0.data_ptr(),
                               g1.data_ptr(), ga.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        assert rc == 0
        return g0, g1, ga

    d0, d1, da = run(n)
    p0, p1, pa = run(pitch)
    assert torch.equal(p0[..., :n], d0) and torch.equal(p1[..., :n], d1) and torch.equal(pa, da)
    assert torch.isnan(p1[..., n:]).all()
    assert torch.allclose(d1.double().sum(dim=(1, 2, 3)), torch.zeros(B, dtype=torch.float64, device=dev),
                          atol=1e-3)


def test_pitch_below_n_is_refused():
    n = 16
    r0, r1 = S.blob_pair(n, 3, seed=2)
    rc, *_ = _call_solve(n, 3, K3, r0, r1, n, iters=10)
    assert rc == 0
    lib = _native.load()
    dev = _dev()
    g = _native.GraphArg(3, K3)
    t = torch.zeros((3, n, n), device=dev)
    u = torch.zeros((6, n, n), device=dev)
    p = V._params(None, None, None, 0, 0, 10, 10, 0.0, 0.0, False, "auto", pitch=n - 1)
    res = _native.Result()
    rc = lib.vomt_solve(_native.context(0), n, t.data_ptr(), t.data_ptr(), g.ref, 1.0, ctypes.byref(p),
                        u.data_ptr(), t.data_ptr(), t.data_ptr(), ctypes.byref(res), None)
    assert rc == -1
