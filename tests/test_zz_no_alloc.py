"""The allocation-free diagnostics entry point (tled_get_stats_noalloc).

It exists for callers that cannot allocate device memory when they need the
numbers (real-time loops, or all device memory held by another allocator):
its scratch is a static device array, so it must agree with the
workspace-based tled_get_stats.  This file is named to
be collected last; it also passes when run alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _close(got, expect):
    # sums and maxima: relative; temperature extremes come back from T - T0 (absolute)
    idx = [0, 1, 4, 5]
    np.testing.assert_allclose(got[idx], expect[idx], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(got[2:4], expect[2:4], rtol=0, atol=1e-12)


def test_noalloc_stats_match_workspace_stats_twice():
    import torch

    from paper_2009_10400_b300 import tled

    prob = W.block_h8(n=12, h=4e-3)
    s = tled.Solver.from_problem(prob)
    s.step(300)
    ref = s.stats()
    T0 = prob.T0
    expect = np.array([ref["kinetic_energy"], ref["heat_content"], ref["T_max"] - T0, ref["T_min"] - T0,
                       ref["u_max"] ** 2, ref["damage_volume"]])
    for _ in range(2):  # two calls in a row share (and overwrite) the static scratch
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        s.stats_noalloc(out)
        s.sync()
        got = out.cpu().numpy()
        _close(got, expect)
    # a block count above the static scratch size is refused with a clear error
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(tled.TledError) as ei:
        s.stats_noalloc(out, n_blocks=297)
    assert ei.value.code == tled.E_ARG and "296" in str(ei.value)
    # fewer blocks give the same sums up to rounding order
    s.stats_noalloc(out, n_blocks=7)
    s.sync()
    _close(out.cpu().numpy(), expect)
    # an output in host memory (pageable or pinned), passed straight through the C ABI,
    # is refused by the host-side pointer check before anything is enqueued
    for host in (torch.zeros(6, dtype=torch.float64), torch.zeros(6, dtype=torch.float64).pin_memory()):
        rc = tled.lib().tled_get_stats_noalloc(s.h, 0, C.c_void_p(host.data_ptr()))
        assert rc == tled.E_ARG, rc
    s.sync()  # nothing was launched: the stream and the status are clean
