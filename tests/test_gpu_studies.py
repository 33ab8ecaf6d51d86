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


def test_subcycling_vs_mass_scaling_vs_full_inertia_over_2s():
    """Study f4: the planning-style scenario heated for 2 s (8 MW/m^3, 16^3 H8,
    gamma = 5) with the thermal step 0.01 s of the planning runs, three ways
    against the reference (full inertia, every step a coupled step at the
    stable step): mechanical subcycling (T every 0.01 s, the mechanics in
    n_sub substeps at the stable step, full inertia), R17 mass scaling at
    0.01 s, and the mass scale at the small step.  Reports the temperature-rise
    and displacement changes and the device time of each."""
    import torch

    from paper_2009_10400_b300 import tled
    q = W.sample_scenarios(1, seed=41)[0]
    q[0], q[4] = 8e6, 2.0

    def problem(**kw):
        p = W.scenario_problem(q, n=16, dt=0.01)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def run(p):
        s = tled.Solver.from_problem(p)
        n = int(round(2.0 / s.get_dt()[0]))
        s.step(32)  # graphs captured
        s.sync()
        z3, z = np.zeros((p.nn, 3)), np.zeros(p.nn)
        s.set_state(z3, z3, np.full(p.nn, p.T0), z, None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(n)
        e1.record()
        s.sync()
        torch.cuda.synchronize()
        out = (s.temperature() - p.T0, s.displacement(), e0.elapsed_time(e1), n)
        s.close()
        return out

    pl = tled.HostPlanner()
    pl.setup_from(problem(mass_scale=1.0, dt=0.0))
    dt_mech = pl.stable_dt()[0]
    pl.close()
    n_sub = int(np.ceil(0.01 / (0.8 * dt_mech)))
    th_ref, u_ref, ms_ref, n_ref = run(problem(mass_scale=1.0, dt=0.0))
    th_sub, u_sub, ms_sub, n_s = run(problem(mass_scale=1.0, dt=0.01, n_sub=n_sub))
    th_ms, u_ms, ms_ms, _ = run(problem())  # automatic mass scale at 0.01 s
    e_sub, e_ms = rel_l2(th_sub, th_ref), rel_l2(th_ms, th_ref)
    eu_sub, eu_ms = rel_l2(u_sub, u_ref), rel_l2(u_ms, u_ref)
    print(f"2 s of heating, peak rise {th_ref.max():.3f} K, |u| max {np.abs(u_ref).max():.2e} m: full inertia "
          f"({n_ref} steps) {ms_ref:.1f} ms; subcycling n_sub={n_sub} ({n_s} substeps) theta {e_sub:.2e} u {eu_sub:.2e}"
          f" {ms_sub:.1f} ms; mass scaling theta {e_ms:.2e} u {eu_ms:.2e} {ms_ms:.1f} ms")
    assert th_ref.max() > 0.5
    assert e_sub < 1e-2 and e_ms < 2e-2
    # subcycling keeps the full inertia: its displacements follow the reference far more closely
    assert eu_sub < eu_ms
