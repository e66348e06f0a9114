"""vomt_solve_noalloc: the solve for callers that cannot allocate device memory
(an application whose device memory belongs to one custom pool or allocator, a
plug-in or service that must not grow its footprint after start-up).  Its
scratch is a fixed array inside the library that every call shares and
overwrites, so these tests call it through the C ABI several times in a row, on
problems of different sizes, channel counts and norms, and compare each result
with vomt_solve on the same inputs and with the FP64 oracle, within the
tolerances the other GPU tests use (relative L2 1e-3 on phi, u and w, 1e-4 on
the primal objective).  This file is collected last so that a run stopping at
its first failure has already run every other test."""
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
    p = V._params(kw.get("tau"), kw.get("mu"), kw.get("nu"), kw.get("u_norm", 0), kw.get("w_norm", 0),
                  kw.get("max_iters", 300), kw.get("check_every", 100), kw.get("tol", 0.0), kw.get("tol", 0.0),
                  False, "auto", eps=kw.get("eps", 0.0))
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
                  tol_gap=kw.get("tol", 0.0), tol_res=kw.get("tol", 0.0), engine="stream", tau=kw.get("tau"),
                  mu=kw.get("mu"), nu=kw.get("nu"), u_norm=kw.get("u_norm", 0), w_norm=kw.get("w_norm", 0),
                  eps=kw.get("eps", 0.0))
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
    # third call: one channel, no graph edges (the scalar problem of Section 7.1), w = NULL
    r0, r1 = S.blob_pair(29, 1, seed=11)
    _check_against_vomt_solve(r0, r1, [], 1.0, max_iters=250, check_every=50)
    # fourth call: joint Euclidean norms, user step sizes and the quadratic regulariser
    r0, r1 = S.blob_pair(40, 3, seed=12)
    r0, r1 = r0 * 1600, r1 * 1600
    _check_against_vomt_solve(r0, r1, S.COMPLETE_K3, 0.7, max_iters=300, check_every=100, u_norm=1, w_norm=1,
                              tau=2.0, mu=1.0 / (40 * 2.0 * 39 ** 2), nu=1.0 / (16 * 2.0 * 3), eps=0.05)


def test_noalloc_matches_oracle_at_fixed_iterations():
    """Two calls in a row against the FP64 oracle (Section 7.2 iteration) at a fixed
    iteration count: relative L2 <= 1e-3 on phi, u, w and relative <= 1e-4 on P."""
    oracle = pytest.importorskip("oracle")
    for n, k, edges, seed, iters in ((33, 3, S.COMPLETE_K3, 21, 500), (26, 2, [(0, 1)], 22, 300)):
        r0, r1 = S.blob_pair(n, k, seed=seed)
        r0, r1 = r0.astype(np.float32), r1.astype(np.float32)
        rc, msg, u, w, phi, res = _noalloc(r0, r1, edges, 1.0, max_iters=iters, check_every=100)
        assert rc == 0, msg
        o = oracle.vomt_solve(r0.astype(np.float64), r1.astype(np.float64), edges, 1.0, max_iters=iters,
                              check_every=100)
        ref_u = torch.from_numpy(np.stack([o["ux"], o["uy"]]))
        assert _rel(phi, torch.from_numpy(o["phi"])) <= 1e-3
        assert _rel(u, ref_u) <= 1e-3
        assert _rel(w, torch.from_numpy(o["w"])) <= 1e-3
        assert abs(res["primal"] - o["metrics"]["primal"]) <= 1e-4 * abs(o["metrics"]["primal"])


def test_noalloc_refuses_a_stream_under_graph_capture():
    """The call synchronises its stream, which graph capture forbids: it must refuse the
    capturing stream before doing any GPU work, leaving the capture intact."""
    d = _dev()
    lib = _native.load()
    r0, r1 = S.blob_pair(16, 3, seed=5)
    g = _native.GraphArg(3, S.COMPLETE_K3)
    d0 = torch.from_numpy(r0.astype(np.float32)).to(d)
    d1 = torch.from_numpy(r1.astype(np.float32)).to(d)
    u = torch.zeros((2, 3, 16, 16), device=d)
    w = torch.zeros((3, 16, 16), device=d)
    phi = torch.zeros((3, 16, 16), device=d)
    p = V._params(None, None, None, 0, 0, 50, 50, 0.0, 0.0, False, "auto")
    res = _native.Result()
    err = ctypes.c_char_p()
    side = torch.cuda.Stream(device=d)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        rc = lib.vomt_solve_noalloc(16, d0.data_ptr(), d1.data_ptr(), g.ref, 1.0, ctypes.byref(p), u.data_ptr(),
                                    w.data_ptr(), phi.data_ptr(), ctypes.byref(res), ctypes.c_void_p(side.cuda_stream),
                                    ctypes.byref(err))
        phi.add_(1.0)                        # the capture is still usable after the refusal
    graph.replay()
    torch.cuda.synchronize()
    assert rc == -1 and b"captur" in (err.value or b"")
    assert float(phi.min()) == 1.0 and float(phi.max()) == 1.0


def test_noalloc_rejects_oversized_problems():
    r0, r1 = S.blob_pair(8, 3, seed=3)
    n = 1024    # needs 4 * 27 * 1024^2 bytes > the fixed scratch
    big0 = np.zeros((3, n, n)); big0[:, :8, :8] = r0
    big1 = np.zeros((3, n, n)); big1[:, :8, :8] = r1
    rc, msg, *_ = _noalloc(big0, big1, S.COMPLETE_K3, 1.0, max_iters=5)
    assert rc == -10 and "scratch" in msg
