"""Failure detection without a GPU fault: every device wait of the library is
bounded; when one runs out it records a timeout in the plan's device error word
and returns, and the host reads SEXPE_ETIMEOUT.  The self-test waits on a
barrier that nothing arrives on (limit ~1 ms) and the context stays usable:
a plan steps normally afterwards."""
import numpy as np
import pytest

from paper_2604_11558_gb300 import workloads as wl
from tests.gpu_helpers import assert_parity, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    from paper_2604_11558_gb300 import binding
    assert binding.selftest_wait_timeout() == 4          # SEXPE_ETIMEOUT
    assert binding.selftest_wait_timeout() == 4          # repeatable: nothing left hung
    w = wl.gray_scott_ball(n=(12, 10, 9), steps=3, seed=31)
    assert_parity(gpu_run(w, "split_tf32"), oracle_run(w), w["W0"], 1e-6, 1e-5)
