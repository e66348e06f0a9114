"""vomt_solve_noalloc: the solve for callers that cannot allocate device memory
(for example code running under CUDA graph capture, where cudaMalloc is not
allowed, or an application whose device memory belongs to one custom pool).
Its scratch is a fixed array inside the library, so these tests call it
through the C ABI twice in a row, on problems of different sizes, and compare
each result with vomt_solve on the same inputs, within the tolerances the other
GPU tests use (relative L2 1e-3 on phi and u, 1e-4 on the primal objective).
This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")
_native = V._native


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _noalloc(r0, r1, edges, alpha, **kw):
    d = _dev()
    lib = _native.load()
    k, n = r0.shape[0], r0.shape[-1]
    g = _native.GraphArg(k, edges)
    l = g.tail.size
    d0 = torch.from_numpy(r0.astype(np.float32)).to(d)
    d1 = torch.from_numpy(r1.astype(np.float32)).to(d)
    u = torch.full((2, k, n, n), float("nan"), device=d)
    w = torch.full((max(l, 1), n, n), float("nan"), device=d)
    phi = torch.full((k, n, n), float("nan"), device=d)
    p = V._params(None, None, None, 0, 0, kw.get("max_iters", 300), kw.get("check_every", 100),
                  kw.get("tol", 0.0), kw.get("tol", 0.0), False, "auto")
    res = _native.Result()
    err = ctypes.c_char_p()
    st = torch.cuda.current_stream(d).cuda_stream
    rc = lib.vomt_solve_noalloc(int(n), d0.data_ptr(), d1.data_ptr(), g.ref, float(alpha), ctypes.byref(p),
                                u.data_ptr(), w.data_ptr() if l else None, phi.data_ptr(), ctypes.byref(res),
                                ctypes.c_void_p(st), ctypes.byref(err))
    torch.cuda.synchronize()
    return rc, (err.value or b"").decode(), u, w[:l], phi, res.as_dict()


def _rel(a, b):
    a = a.detach().cpu().double().numpy()
    b = b.detach().cpu().double().numpy()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _check_against_vomt_solve(r0, r1, edges, alpha, **kw):
    rc, msg, u, w, phi, res = _noalloc(r0, r1, edges, alpha, **kw)
    assert rc >= 0, msg
    d = _dev()
    ref = V.solve(torch.from_numpy(r0.astype(np.float32)).to(d), torch.from_numpy(r1.astype(np.float32)).to(d),
                  edges, alpha, max_iters=kw.get("max_iters", 300), check_every=kw.get("check_every", 100),
                  tol_gap=kw.get("tol", 0.0), tol_res=kw.get("tol", 0.0), engine="stream")
    torch.cuda.synchronize()
    assert rc == (0 if ref.result["status"] == 0 else ref.result["status"])
    assert res["iters"] == ref.result["iters"]
    assert _rel(phi, ref.phi) <= 1e-3
    assert _rel(u, ref.u) <= 1e-3
    if len(edges):
        assert _rel(w, ref.w) <= 1e-3
    assert abs(res["primal"] - ref.result["primal"]) <= 1e-4 * abs(ref.result["primal"])
    assert abs(res["rel_res"] - ref.result["rel_res"]) <= 1e-4 * abs(ref.result["rel_res"]) + 1e-12
    return res


def test_noalloc_two_calls_match_vomt_solve():
    # first call: 48 x 48, k = 3, complete graph, fixed iteration count
    r0, r1 = S.blob_pair(48, 3, seed=1001)
    _check_against_vomt_solve(r0, r1, S.COMPLETE_K3, 1.0, max_iters=400, check_every=100)
    # second call in a row, different size and graph, stopping on a tolerance: the
    # scratch still holds the first call's contents
    r0, r1 = S.blob_pair(37, 4, seed=7)
    res = _check_against_vomt_solve(r0, r1, [(0, 1), (1, 2), (2, 3)], 0.5, max_iters=20000, check_every=100,
                                    tol=1e-2)
    assert res["status"] == 0 and res["rel_gap"] <= 1e-2 and res["rel_res"] <= 1e-2


def test_noalloc_rejects_oversized_problems():
    r0, r1 = S.blob_pair(8, 3, seed=3)
    n = 1024    # needs 4 * 27 * 1024^2 bytes > the fixed scratch
    big0 = np.zeros((3, n, n)); big0[:, :8, :8] = r0
    big1 = np.zeros((3, n, n)); big1[:, :8, :8] = r1
    rc, msg, *_ = _noalloc(big0, big1, S.COMPLETE_K3, 1.0, max_iters=5)
    assert rc == -10 and "scratch" in msg
