"""Studies the readings call for: the effect of mass scaling (and of the
large fixed time step it allows) on the temperature field."""
import numpy as np
import pytest

from helpers import rel_l2
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_mass_scaling_effect_on_temperature_over_2s():
    """A planning-style scenario (16^3 H8 cube, 8 MW/m^3 source, gamma = 5)
    heated for 2 s three ways: full inertia at the stable step; the mass scale
    that makes dt = 0.01 s stable, at the same small step (isolates the
    mechanical inertia's effect on theta, which only enters through the source
    position x = X + u and the deformed-configuration conduction); and that
    mass scale at dt = 0.01 s (adds the explicit Euler time-step effect)."""
    import oracle
    from paper_2009_10400_b300 import tled
    q = W.sample_scenarios(1, seed=41)[0]
    q[0], q[4] = 8e6, 2.0
    base = W.scenario_problem(q, n=16, dt=0.01)
    base.dt, base.mass_scale = 0.0, 1.0  # the stable step of the unscaled problem
    pl = tled.HostPlanner()
    pl.setup_from(W.scenario_problem(q, n=16, dt=0.01))  # automatic mass scale for dt = 0.01 s
    s_m = pl.mass_scale()
    pl.close()
    assert s_m > 100.0
    np.testing.assert_allclose(s_m, oracle.mass_scale_for(base, 0.01), rtol=1e-12)

    def run(mass_scale, dt):
        p = W.scenario_problem(q, n=16, dt=0.01)
        p.mass_scale = mass_scale
        s = tled.Solver.from_problem(p, dt=dt)
        dt_used = s.get_dt()[0]
        n = int(round(2.0 / dt_used))
        s.step(n)
        s.sync()
        return s.temperature() - p.T0, s.displacement(), n * dt_used

    s0 = tled.Solver.from_problem(base, dt=0.0)
    dt_small = s0.get_dt()[0]  # stable step of the unscaled problem
    s0.close()
    th_full, u_full, t1 = run(1.0, dt_small)
    th_ms, u_ms, t2 = run(s_m, dt_small)
    th_big, _, t3 = run(s_m, 0.01)
    assert abs(t1 - 2.0) < dt_small and abs(t2 - 2.0) < dt_small and abs(t3 - 2.0) < 1e-9
    e_inertia = rel_l2(th_ms, th_full)
    e_step = rel_l2(th_big, th_full)
    print(f"mass scale {s_m:.3g}: theta change from inertia {e_inertia:.2e}, with dt 0.01 s {e_step:.2e}; "
          f"peak rise {th_full.max():.3f} K; |u| max {np.abs(u_full).max():.2e} m (scaled {np.abs(u_ms).max():.2e} m)")
    assert th_full.max() > 0.5
    assert e_inertia < 1e-3
    assert e_step < 2e-2
