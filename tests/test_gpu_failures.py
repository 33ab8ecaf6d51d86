"""Failure detection on the GPU without a fault: every device wait is bounded (about
a second) and reports a status the host reads.  A one-CTA self-test kernel makes an
mbarrier wait and a grid-barrier wait run out (nothing ever completes them); the
library reports E_TIMEOUT, clears the status, and the context steps on normally."""
import numpy as np
import pytest

from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_waits_report_timeout_and_the_context_recovers():
    from paper_2009_10400_b300 import tled
    prob = W.cube_h8(n=4)
    s = tled.Solver.from_problem(prob)
    for which in (0, 1):
        assert s.selftest_wait(which) == tled.E_TIMEOUT
    s.step(50)
    s.sync()  # no stale status
    ref = tled.Solver.from_problem(prob)
    ref.step(50)
    ref.sync()
    for a, b in ((s.displacement(), ref.displacement()), (s.temperature(), ref.temperature())):
        assert np.array_equal(a, b)
    assert s.selftest_wait(2) == tled.E_ARG
