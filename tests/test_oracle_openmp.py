"""The multi-core build of the oracle (the benchmark's OpenMP CPU baseline) splits only
loops over grid points whose iterations are independent, so it must reproduce the
one-thread build bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S


@pytest.fixture
def four_threads():
    try:
        oracle.set_threads(4)
    except Exception as ex:          # no OpenMP runtime for this compiler
        pytest.skip("OpenMP build unavailable: %s" % ex)
    yield
    oracle.set_threads(1)


def _run_vector():
    r0, r1 = S.blob_pair(24, 3, seed=91)
    return oracle.vomt_solve(r0, r1, S.COMPLETE_K3, 0.8, tau=4.0, max_iters=120, check_every=40, history=True)


def _run_matrix():
    L0, L1 = S.tensor_field_pair(12, 3, seed=92)
    L = S.random_L(3, 3, seed=92)
    return oracle.momt_solve(L0 * 144, L1 * 144, L, 1.0, tau=10.0, max_iters=60, check_every=30, history=True)


def test_openmp_build_is_bit_identical(four_threads):
    par_v, par_m = _run_vector(), _run_matrix()
    oracle.set_threads(1)
    ser_v, ser_m = _run_vector(), _run_matrix()
    for a, b, keys in ((par_v, ser_v, ("ux", "uy", "w", "phi", "history")),
                       (par_m, ser_m, ("Ux", "Uy", "W", "Phi", "history"))):
        for key in keys:
            assert np.array_equal(a[key], b[key]), key
