"""Sanity check of the step-size rule against the paper's own convergence figures.

Table 1 (Section 8.1) runs V-OMT on a pair of colour images with three disks that keep
their place and change colour, with the tau it lists, and reports iterations to gap /
primal <= 1e-3: 5e3 at 64 x 64 (tau = 1) and 2e4 at 256 x 256 (tau = 3).  The paper's
images are not available; ``synthetic.three_disk_pair`` has the same structure.  With the
step rule mu = 1/(32 tau (n-1)^2), nu = 1/(4 tau lambda_max) of Section 7.2 and Table 1's
tau, the GPU path and the FP64 oracle must reach that gap within twice Table 1's count,
and their costs must agree to the parity bar."""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("n,tau,table1_iters", [(64, 1.0, 5000), (256, 3.0, 20000)])
def test_gap_1e3_within_table1_order(n, tau, table1_iters):
    dev = _dev()
    r0, r1 = S.three_disk_pair(n)
    r0 = r0.astype(np.float32).astype(np.float64)
    r1 = r1.astype(np.float32).astype(np.float64)
    kw = dict(tau=tau, max_iters=2 * table1_iters, check_every=100, tol_gap=1e-3, tol_res=1e9)
    sol = V.solve(torch.from_numpy(r0.astype(np.float32)).to(dev), torch.from_numpy(r1.astype(np.float32)).to(dev),
                  S.COMPLETE_K3, 1.0, **kw)
    r = sol.result
    assert r["status"] == 0 and r["rel_gap"] <= 1e-3, r
    assert r["iters"] <= 2 * table1_iters
    if n <= 64:
        ref = oracle.vomt_solve(r0, r1, S.COMPLETE_K3, 1.0, **kw)
        assert ref["metrics"]["converged"] == 1.0 and ref["iters"] <= 2 * table1_iters
        assert abs(ref["iters"] - r["iters"]) <= 200
        assert abs(r["primal"] - ref["metrics"]["primal"]) <= 1e-3 * abs(ref["metrics"]["primal"])
