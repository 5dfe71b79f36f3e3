"""Device-side failure detection without a GPU fault.

Every TMA copy in the step kernels is awaited with a bounded mbarrier wait that,
when it runs out, records a timeout in the context's status word and returns.
The self-test entry point makes exactly that wait run out (it expects bytes that
nothing sends); the context then reports DUGKS_ETIMEOUT, while the device stays
usable: a new context on it steps and matches its result from before.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def run_drop(steps=20):
    prob = WL.drop64(order=3)
    with N.Solver.from_problem(prob, precision="fp32") as s:
        s.step(steps)
        assert s.status() == 0
        return s.phi()


def test_bounded_wait_times_out_and_device_stays_usable():
    before = run_drop()
    prob = WL.drop64(order=3)
    s = N.Solver.from_problem(prob, precision="fp32")
    try:
        s.step(3)
        assert s.status() == 0
        assert N.dugks_selftest_wait_timeout(s.ctx, 2000) == 0
        assert N.lib().dugks_status(s.ctx) == N.DUGKS_ETIMEOUT
        assert "wait" in N.dugks_last_error(s.ctx)
        # sticky: later calls on this context report the timeout too
        assert N.lib().dugks_step(s.ctx, 1) == N.DUGKS_ETIMEOUT
    finally:
        s.close()
    assert np.array_equal(run_drop(), before)


def test_selftest_rejects_bad_counts():
    prob = WL.drop64(order=3)
    with N.Solver.from_problem(prob, precision="fp32") as s:
        for bad in (0, (1 << 20) + 1):
            assert N.dugks_selftest_wait_timeout(s.ctx, bad) == N.DUGKS_EINVAL
        assert s.status() == 0
