"""Learned surrogate: the mass-scaled planning scenarios against the oracle,
and what a trained ensemble gains over running the solver (a small instance of
the surrogate workload: 8^3 cube, 512 probes, short heating)."""
import numpy as np
import pytest

import oracle
from helpers import TOL_E, compare
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_mass_scaled_planning_scenario_matches_oracle():
    """Fixed dt = 0.01 s with mass scaling, damping 5 1/s, inputs from the
    scenario sampler; 300 steps against the oracle with the same mass scale."""
    from paper_2009_10400_b300 import tled
    q = W.sample_scenarios(4, seed=11)[2]
    p = W.scenario_problem(q, n=8, dt=0.01)
    assert p.mass_scale < 0  # automatic: the library and the oracle each derive it from their own CFL bound
    m = oracle.OracleModel(p)
    assert m.mass_scale > 1.0
    s = m.init_state()
    m.step(s, 300)
    g = tled.Solver.from_problem(p)
    np.testing.assert_allclose(g.mass_scale(), m.mass_scale, rtol=1e-12)
    g.step(300)
    g.sync()
    c = compare(g.displacement(), g.temperature(), g.damage(), s.u, s.T, s.Omega)
    assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E, c


def test_surrogate_learns_and_falls_back():
    import time

    from paper_2009_10400_b300 import surrogate
    n, dt = 8, 0.05
    Q = W.sample_scenarios(1152, seed=12, duration=(5.0, 30.0))
    T, D, tm = surrogate.solve_scenarios(Q, n=n, dt=dt)
    assert np.all(np.isfinite(T)) and T.max() > 40.0
    Y = np.concatenate([T, D], 1)
    tr, te = slice(0, 1024), slice(1024, 1152)
    sur = surrogate.Surrogate(n_out=2 * n ** 3, width=256, depth=4, members=3, max_batch=4096)
    hist = sur.fit(Q[tr], Y[tr], epochs=60, batch=128, lr=2e-3, seed=1)
    assert hist[0][-1] < 0.25 * hist[0][0]
    mean, std = sur.predict(Q[te])
    big = np.repeat(Q[te], 32, axis=0)  # 4096 scenarios, one inference batch per member
    sur.predict(big)
    t0 = time.perf_counter()
    sur.predict(big)
    t_sur = time.perf_counter() - t0
    P = n ** 3
    mae = np.abs(mean[:, :P] - T[te]).mean()
    mae_base = np.abs(Y[tr, :P].mean(0) - T[te]).mean()  # predicting the training mean
    assert mae < 0.6 * mae_base, (mae, mae_base)
    # the ensemble spread flags its own large errors
    err = np.abs(mean[:, :P] - T[te]).max(1)
    spread = std[:, :P].max(1)
    assert np.corrcoef(err, spread)[0, 1] > 0.2
    # fallback: the uncertain cases come back from the solver exactly
    tol = float(np.quantile(spread, 0.75))
    out, fb, info = sur.solve(Q[te], P, tol=tol, n=n, dt=dt)
    assert 0 < fb.sum() < len(fb)
    np.testing.assert_allclose(out[fb], Y[te][fb], rtol=0, atol=1e-9)
    # at the stated tolerance of 1 K (the fallback rule as written: spread > 1 K goes to
    # the solver): the fraction answered by the surrogate and the worst answered error
    out1, fb1, info1 = sur.solve(Q[te], P, tol=1.0, n=n, dt=dt)
    err1 = np.abs(out1[:, :P] - T[te]).max(1)
    np.testing.assert_allclose(out1[fb1], Y[te][fb1], rtol=0, atol=1e-9)
    print(f"at 1 K: surrogate answers {np.mean(~fb1):.2f} of the cases, worst answered error "
          f"{err1[~fb1].max() if (~fb1).any() else 0.0:.3f} K, {len(fb1) / info1['seconds']:.1f} solves/s")
    # calibration against solver answers: with coverage 1, every calibration case
    # whose spread is at or below the threshold meets the tolerance
    tol_c = float(np.median(err))
    cal = slice(0, 64)
    tau, frac = sur.calibrate(Q[te][cal], Y[te][cal], P, tol=tol_c, coverage=1.0)
    assert frac < 1.0 and tau <= tol_c
    acc = spread[cal] <= tau
    assert acc.sum() == round(frac * 64) and np.all(err[cal][acc] <= tol_c)
    # speed: surrogate predictions vs solver scenarios per second
    solver_rate = len(Q) / tm["seconds"]
    sur_rate = len(big) / t_sur
    print(f"solver {solver_rate:.1f} scen/s, surrogate {sur_rate:.1f} scen/s, mae {mae:.3f} K (base {mae_base:.3f})")
    assert sur_rate > 3 * solver_rate


def test_surrogate_answers_at_one_kelvin():
    """The learned part at the stated accuracy: trained on the solver's data
    augmented by the cube's 16 reflections, with the spread threshold
    calibrated against the solver on 512 held-out scenarios (every calibration
    case at or below it within 0.8 K: the bench's policy, a margin below the
    stated 1 K), the surrogate answers a non-zero fraction of 256 further
    scenarios, every answer within 1 K of the solver, and the rest comes back
    from the solver exactly."""
    from paper_2009_10400_b300 import surrogate
    n, dt = 8, 0.05
    P = n ** 3
    n_tr, n_cal, n_ev = 2048, 512, 256
    Q = W.sample_scenarios(n_tr + n_cal + n_ev, seed=12, duration=(5.0, 30.0))
    T, D, tm = surrogate.solve_scenarios(Q, n=n, dt=dt)
    Y = np.concatenate([T, D], 1)
    tr, cal, ev = slice(0, n_tr), slice(n_tr, n_tr + n_cal), slice(n_tr + n_cal, n_tr + n_cal + n_ev)
    sur = surrogate.Surrogate(n_out=2 * P, width=256, depth=4, members=4, max_batch=4096, symmetric=True, grid=n,
                              max_rows=16 * n_tr)
    sur.fit(Q[tr], Y[tr], epochs=20, batch=128, lr=2e-3, seed=1, lr_end=1e-5)
    mean, std = sur.predict(Q[ev])
    err_ev = np.abs(mean[:, :P] - T[ev]).max(1)
    sp_ev = std[:, :P].max(1)
    for m in (1.0, 0.8, 0.6):  # the trade-off, for the record
        tau_m, f_m = sur.calibrate(Q[cal], Y[cal], P, tol=m, coverage=1.0)
        acc = sp_ev <= tau_m
        print(f"calibrated at {m:.1f} K: threshold {tau_m:.3f} K, answers {acc.mean():.3f} of the evaluation "
              f"cases, worst answered {err_ev[acc].max() if acc.any() else 0.0:.3f} K")
    tau, frac = sur.calibrate(Q[cal], Y[cal], P, tol=0.8, coverage=1.0)
    out, fb, info = sur.solve(Q[ev], P, tol=1.0, n=n, dt=dt)
    err = np.abs(out[:, :P] - T[ev]).max(1)
    rate = n_ev / info["seconds"]
    solver_rate = len(Q) / tm["seconds"]
    print(f"at 1 K: threshold {tau:.3f} K (calibration accepts {frac:.2f}); the surrogate answers "
          f"{np.mean(~fb):.2f} of the evaluation cases, worst answered error "
          f"{err[~fb].max() if (~fb).any() else 0.0:.3f} K; {rate:.1f} solves/s with fallback, "
          f"batched solver {solver_rate:.1f} solves/s; median worst-probe error {np.median(err_ev):.3f} K")
    np.testing.assert_allclose(out[fb], Y[ev][fb], rtol=0, atol=1e-9)  # fallbacks: the solver's answers
    assert (~fb).any(), (tau, frac)
    assert np.all(err[~fb] <= 1.0), err[~fb].max()
