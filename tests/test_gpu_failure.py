"""Failure detection without a GPU fault.

The resident engine's blocks wait on one another (halo words, check rows), and
every wait is bounded.  Here block 0 skips one halo exchange on purpose (a
message dropped on the device, nothing faults) under a short wait budget: its
neighbours' waits run out, every block returns, and the solve reports
BARRIER_TIMEOUT.  The same context then solves normally and matches the FP64
oracle.  Input errors are made on the host and come back as status codes."""
import time

import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")
N = pytest.importorskip("paper_1712_10279_gb300._native")

K3 = S.COMPLETE_K3


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(_dev())


def test_dropped_halo_message_times_out_and_context_recovers():
    r0, r1 = S.blob_pair(64, 3, seed=77)
    d0, d1 = _t(r0), _t(r1)
    try:
        V.set_wait_policy(budget_ms=100.0, drop_exchange=3)
        t0 = time.perf_counter()
        with pytest.raises(N.VomtError) as ei:
            V.solve(d0, d1, K3, 1.0, max_iters=400, check_every=100, engine="resident")
        elapsed = time.perf_counter() - t0
        assert ei.value.status == -8          # VOMT_ERR_BARRIER_TIMEOUT
        assert elapsed < 5.0                  # bounded by the budget, not by a hang
    finally:
        V.set_wait_policy(0.0, 0)
    sol = V.solve(d0, d1, K3, 1.0, max_iters=400, check_every=100, engine="resident")
    ref = oracle.vomt_solve(r0.astype(np.float32).astype(np.float64), r1.astype(np.float32).astype(np.float64),
                            K3, 1.0, max_iters=400, check_every=100)
    assert sol.result["status"] == 0 and sol.result["blocks"] > 1
    assert sol.result["primal"] == pytest.approx(ref["metrics"]["primal"], rel=1e-4)


def test_wait_policy_arguments_are_checked():
    ctx = N.context(0)
    lib = N.load()
    assert lib.vomt_set_wait_policy(ctx, -1.0, 0) == -1
    assert lib.vomt_set_wait_policy(ctx, float("nan"), 0) == -1
    assert lib.vomt_set_wait_policy(ctx, 10.0, -2) == -1
    assert lib.vomt_set_wait_policy(None, 10.0, 0) == -1
    assert lib.vomt_set_wait_policy(ctx, 0.0, 0) == 0


def test_bad_inputs_return_status_codes():
    r0, r1 = S.blob_pair(16, 3, seed=78)
    bad = r1.copy()
    bad[0, 2, 2] = -1e-3
    with pytest.raises(N.VomtError) as ei:
        V.solve(_t(r0), _t(bad), K3, 1.0, max_iters=10)
    assert ei.value.status in (-2, -3)
    nan = r1.copy()
    nan[1, 3, 3] = np.nan
    with pytest.raises(N.VomtError) as ei:
        V.solve(_t(r0), _t(nan), K3, 1.0, max_iters=10)
    assert ei.value.status in (-2, -3, -7)
    sol = V.solve(_t(r0), _t(r1), K3, 1.0, max_iters=10)     # the context is still usable
    assert sol.result["status"] == 0
