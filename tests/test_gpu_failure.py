"""Failure detection on the GPU without a GPU fault: the bounded wait that every pipeline
barrier of the tensor-core kernel uses is made to run out (an mbarrier phase that nothing
completes, 50 ms limit); the status comes back as QSGW_ERR_TIMEOUT, and the device stays usable
for a normal computation right after."""
import time

import numpy as np
import pytest

import oracle
from synthetic import TINY

from test_gpu_fp64 import rel_fro, run_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def test_bounded_wait_times_out_and_device_stays_usable(N):
    t = time.perf_counter()
    assert N.qsgw_selftest_wait_timeout(0.05) == N.QSGW_ERR_TIMEOUT
    assert time.perf_counter() - t < 5.0
    assert N.qsgw_selftest_wait_timeout(5.0) == N.QSGW_ERR_ARG  # the limit is bounded
    chi, Z, d = run_workload(N, TINY, N.QSGW_MIXED_F16X3)
    assert rel_fro(chi, oracle.chi0_full(Z, d, TINY.omega, TINY.spin)) <= 1e-6
