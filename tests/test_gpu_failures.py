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
    assert s.selftest_wait(3) == tled.E_ARG
    assert s.selftest_wait(2) == tled.E_STATE  # the resident mode has no tile kernel launch


def test_tile_kernel_timeout_path_leaves_cleanly():
    """The streamed step's tile kernel with one tile's node staging left out: the
    CTA that holds the tile sees its bounded mbarrier wait run out, reads none of
    the missing lists, skips its element pass and leaves after waiting (bounded)
    for its own copies; the library reports E_TIMEOUT and clears it, and after
    the state is set again the context steps bitwise like a fresh one."""
    from paper_2009_10400_b300 import tled
    prob = W.cube_h8(n=10)
    flags = tled.default_flags(prob) | tled.STREAMED
    s = tled.Solver.from_problem(prob, flags=flags)
    assert not s.resident and not s.grid_resident
    assert s.plan_info()["n_tiles"] > 1
    assert s.selftest_wait(2) == tled.E_TIMEOUT
    z3, z = np.zeros((prob.nn, 3)), np.zeros(prob.nn)
    s.set_state(z3, z3, np.full(prob.nn, prob.T0), z, None)
    s.step(40)
    s.sync()
    ref = tled.Solver.from_problem(prob, flags=flags)
    ref.step(40)
    ref.sync()
    for a, b in ((s.displacement(), ref.displacement()), (s.temperature(), ref.temperature()),
                 (s.damage(), ref.damage())):
        assert np.array_equal(a, b)
