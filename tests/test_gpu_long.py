"""Parity at the workloads' own horizons: long FP32 trajectories against the
FP64 oracle, compared every 1000th step with the paper's error indicator
(Section 6.1: e = ||a - b||_2 / ||b||_2 on u and on theta = T - T0), the
maximum normalised error, and the damage fraction.

* The 128^3 block's generator at 32^3 (h = 4 mm; per-element material noise,
  four Gaussian sources) for 5000 steps, with the float-float accumulation of
  u and T on (the product setting) and off (plain FP32 sums), so the errors
  show what the compensation buys.
* The ~143k-tet ellipsoid (vMF fibres, moving source) for 10,000 steps.

The oracle runs on all host cores (its OpenMP step, bitwise the serial one).
"""
import numpy as np
import pytest

import oracle
from helpers import TOL_DAMAGE, TOL_E, compare
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _trajectories(prob, n_steps, every, flag_sets, T0=37.0):
    """One oracle trajectory against one library run per flag set; rows of
    errors per run, every `every` steps."""
    from paper_2009_10400_b300 import tled

    m = oracle.OracleModel(prob)  # the oracle's own stable step (R16), given to the library too
    gs = [tled.Solver.from_problem(prob, flags=f, dt=m.dt) for f in flag_sets]
    _, dt_mech, dt_th = gs[0].get_dt()  # the library's own bounds agree with the oracle's
    assert prob.dt_safety * min(dt_mech, dt_th) == pytest.approx(m.dt, rel=1e-12)
    s = m.init_state()
    rows = [[] for _ in gs]
    for k in range(every, n_steps + 1, every):
        for g in gs:
            g.step(every)
        m.step_parallel(s, every)
        for g, r in zip(gs, rows):
            g.sync()
            c = compare(g.displacement(), g.temperature(), g.damage(), s.u, s.T, s.Omega, T0=T0)
            c["step"] = k
            r.append(c)
    for g in gs:
        g.close()
    return rows, s


def _report(name, rows):
    for c in rows:
        print(f"{name} step {c['step']:6d}: e_u {c['e_u']:.3e} e_theta {c['e_theta']:.3e} "
              f"nre_u {c['nre_u']:.3e} nre_T {c['nre_T']:.3e} damage {c['d_abs']:.2e}")


def test_block_32_cubed_5000_steps_compensated_and_plain():
    from paper_2009_10400_b300 import tled

    p = W.block_h8(n=32, h=4e-3)
    base = tled.default_flags(p)
    assert base & tled.COMPENSATED
    (on, off), s = _trajectories(p, 5000, 1000, [base, base & ~tled.COMPENSATED])
    _report("32^3 compensated", on)
    _report("32^3 plain fp32", off)
    assert s.T.max() - p.T0 > 0.5  # the sources did heat the block
    for c in on:
        assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E and c["d_abs"] <= TOL_DAMAGE, c
    # the compensated sums are never worse than plain FP32 at the horizon
    assert on[-1]["e_theta"] <= off[-1]["e_theta"] and on[-1]["e_u"] <= off[-1]["e_u"], (on[-1], off[-1])


def test_ellipsoid_10k_steps_every_1000th():
    from paper_2009_10400_b300 import tled

    p = W.ellipsoid_t4()
    (rows,), s = _trajectories(p, 10000, 1000, [tled.default_flags(p)])
    _report("ellipsoid", rows)
    assert s.T.max() - p.T0 > 0.1  # 10k stable steps of this mesh (~12 us each) are ~0.12 s of heating
    for c in rows:
        assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E and c["d_abs"] <= TOL_DAMAGE, c
