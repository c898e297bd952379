"""Failure detection on the GPU without a fault: every wait in the pass
kernels is bounded; a kernel that waits for a barrier nothing completes
must give up, raise the error flag the host reads, and leave the context
usable."""
import numpy as np
import pytest

from helpers import assert_parity, gpu_run, oracle_run
from paper_1211_2205_gb300 import capi
from test_gpu_parity import _random_problem

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    assert capi.selftest_bounded_wait() == capi.E_TIMEOUT
    # the same process keeps computing correctly afterwards
    p = _random_problem(5, (70, 45), ("periodic", "extrapolation"), "fp32", 901, 4)
    s, got = gpu_run(p, kernel="tiled", schedule="merged")
    o, ref = oracle_run(p, s)
    assert_parity(got, ref, 1e-5, "fp32")
    s.sync()
