"""Batched scenarios, probe interpolation and the autotuner, against the FP64
oracle run scenario by scenario."""
import numpy as np
import pytest

import oracle
from helpers import rel_l2, TOL_DAMAGE, TOL_E, compare
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _tled():
    from paper_2009_10400_b300 import tled
    return tled


def _scenarios_h8():
    rng = np.random.default_rng(21)
    out = []
    for i, n in enumerate((4, 6, 5)):
        p = W.cube_h8(n=n, jitter=0.1 * i, seed=30 + i)
        p.mu[:] *= rng.uniform(0.8, 1.2)
        p.kc[:] *= rng.uniform(0.8, 1.2)
        p.sources = np.array([W.source(rng.uniform(0.0125, 0.0375, 3), rng.uniform(1e6, 1e7),
                                       vel=rng.uniform(-0.01, 0.01, 3))])
        p.gamma = [0.0, 5.0, 2.0][i]
        out.append(p)
    return out


def _oracle_final(p, n_steps, dt):
    m = oracle.OracleModel(p, dt=dt)
    s = m.init_state()
    m.step(s, n_steps)
    return s


def test_batch_h8_each_scenario_matches_oracle():
    """Three H8 scenarios of different size, material, damping, moving source,
    step size and step count run in the same launches; each stops at its own
    step count and matches its oracle run."""
    tled = _tled()
    scen = _scenarios_h8()
    n_steps = [300, 120, 210]
    # the oracle's own stable step (R16) where no step is given
    dts = [oracle.OracleModel(p).dt if dt is None else dt for p, dt in zip(scen, [None, 2.0e-4, None])]
    b = tled.Batch()
    for p, n, dt in zip(scen, n_steps, dts):
        b.add(p, n, dt=dt)
    b.init()
    ran = b.run()
    b.sync()
    assert ran == max(n_steps)
    u, T, d = b.displacement(), b.temperature(), b.damage()
    for i, (p, n) in enumerate(zip(scen, n_steps)):
        info = b.scenario(i)
        assert info["steps"] == n and info["nodes"] == p.nn
        sl = slice(info["node_off"], info["node_off"] + info["nodes"])
        assert b.scenario_dt(i) == dts[i]
        ref = _oracle_final(p, n, dts[i])
        c = compare(u[sl], T[sl], d[sl], ref.u, ref.T, ref.Omega)
        assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E and c["d_abs"] <= TOL_DAMAGE, (i, c)



def test_batch_mixed_h8_t4_matches_oracle():
    """Hexahedral and tetrahedral scenarios in one batch (one launch per step,
    the element type chosen per tile), interleaved in the add order, with
    different step counts and a planning-style mass-scaled fixed step; each
    matches its own oracle run."""
    tled = _tled()
    scen = [W.cube_h8(n=5, seed=50), W.cube_t4(n=4, seed=51), W.cube_h8(n=4, jitter=0.1, seed=52),
            W.cube_t4(n=5, seed=53)]
    n_steps = [160, 240, 90, 200]
    for p in scen[2:]:  # the planning workloads' fixed dt with mass scaling and damping
        p.dt, p.gamma, p.mass_scale = 0.01, 5.0, -1.0  # R17, derived by the library and the oracle each
    dts = [p.dt if p.dt > 0 else oracle.OracleModel(p).dt for p in scen]  # the oracle's stable step (R16)
    b = tled.Batch()
    for p, n, dt in zip(scen, n_steps, dts):
        b.add(p, n, dt=dt)
    b.init()
    assert b.plan_info()["npe"] == 0
    assert b.run() == max(n_steps)
    b.sync()
    u, T, d = b.displacement(), b.temperature(), b.damage()
    for i, (p, n) in enumerate(zip(scen, n_steps)):
        info = b.scenario(i)
        sl = slice(info["node_off"], info["node_off"] + info["nodes"])
        ref = _oracle_final(p, n, dts[i])
        c = compare(u[sl], T[sl], d[sl], ref.u, ref.T, ref.Omega)
        assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E and c["d_abs"] <= TOL_DAMAGE, (i, c)

def test_batch_t4_matches_single_runs():
    tled = _tled()
    probs = [W.cube_t4(n=4, seed=40), W.cube_t4(n=5, seed=41)]
    dts = [oracle.OracleModel(p).dt for p in probs]
    b = tled.Batch()
    for p, dt in zip(probs, dts):
        b.add(p, 150, dt=dt)
    b.init()
    b.run()
    b.sync()
    T = b.temperature()
    for i, p in enumerate(probs):
        info = b.scenario(i)
        sl = slice(info["node_off"], info["node_off"] + info["nodes"])
        ref = _oracle_final(p, 150, dts[i])
        assert np.linalg.norm(T[sl] - ref.T) / np.linalg.norm(ref.T - 37) <= TOL_E


def test_probes_at_centroids_and_points():
    """Probes at H8 centroids give the mean of the 8 corners; probes at nodes give
    the nodal value; T4 probes give barycentric interpolation."""
    tled = _tled()
    p = W.cube_h8(n=6)
    X, conn = p.X, p.conn
    cen = X[conn].mean(1)[::5]
    nodes = X[[0, 17, 100]]
    s = tled.Solver.from_problem(p, probes=np.vstack([cen, nodes]))
    s.step(200)
    pr = s.probes()
    T, dmg = s.temperature(), s.damage()
    np.testing.assert_allclose(pr[0, :len(cen)], T[conn[::5]].mean(1), rtol=0, atol=1e-9)
    np.testing.assert_allclose(pr[1, :len(cen)], dmg[conn[::5]].mean(1), rtol=0, atol=1e-12)
    np.testing.assert_allclose(pr[0, len(cen):], T[[0, 17, 100]], rtol=0, atol=1e-9)
    # T4: a point inside a tetrahedron, barycentric weights
    q = W.cube_t4(n=3)
    e = 7
    bary = np.array([0.1, 0.2, 0.3, 0.4])
    pt = bary @ q.X[q.conn[e]]
    s4 = tled.Solver.from_problem(q, probes=pt[None])
    s4.step(100)
    T4 = s4.temperature()
    np.testing.assert_allclose(s4.probes()[0, 0], bary @ T4[q.conn[e]], rtol=0, atol=1e-9)
    with pytest.raises(tled.TledError):
        tled.Solver.from_problem(q, probes=np.array([[1.0, 1.0, 1.0]]))


@pytest.mark.parametrize("kind", ["h8_jittered", "t4"])
def test_probes_match_oracle_off_centroid(kind):
    """tled_get_probes against the oracle's own point location and shape-function
    interpolation (ora_probe): arbitrary points off the element centroids --
    on a jittered hex mesh these need the host's Newton solve of the trilinear
    map -- first on a set state (the probe path alone: FP32 weights and
    damage, so 2e-6 of the field's range), then after 300 coupled steps
    against the oracle's trajectory (the paper's e metric on the probe values,
    damage to 1e-3)."""
    tled = _tled()
    p = W.cube_h8(n=6, jitter=0.25, seed=21) if kind == "h8_jittered" else W.cube_t4(n=5, seed=22)
    rng = np.random.default_rng(23)
    lo, hi = p.X.min(0), p.X.max(0)
    pts = lo + (hi - lo) * rng.uniform(0.1, 0.9, (500, 3))
    m = oracle.OracleModel(p)
    s = tled.Solver.from_problem(p, probes=pts, dt=m.dt)
    st = W.random_state(p, 24, theta_scale=20.0)
    st["Omega"] = rng.uniform(0.0, 3.0, p.nn)
    s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"])
    os_ = m.state_from(**st)
    T_o, d_o = m.probe(os_, pts)
    pr = s.probes()
    np.testing.assert_allclose(pr[0], T_o, rtol=0, atol=2e-6 * np.ptp(st["T"]))
    np.testing.assert_allclose(pr[1], d_o, rtol=0, atol=2e-6)
    # a trajectory: both sides step 300 times from rest
    s2 = tled.Solver.from_problem(p, probes=pts, dt=m.dt)
    o = m.init_state()
    m.step(o, 300)
    s2.step(300)
    s2.sync()
    T_o, d_o = m.probe(o, pts)
    pr = s2.probes()
    assert rel_l2(pr[0] - p.T0, T_o - p.T0) <= TOL_E
    assert np.abs(pr[1] - d_o).max() <= TOL_DAMAGE
    assert np.ptp(T_o) > 0.02  # the sources heated the probed region


def test_autotune_then_parity():
    tled = _tled()
    p = W.block_h8(n=12, h=4e-3)
    m = oracle.OracleModel(p)
    s = tled.Solver.from_problem(p, dt=m.dt)
    ch = s.autotune(trial_steps=10)
    assert ch["tile_elems"] in (256, 192, 128) and ch["ctas"] >= 1 and not ch["cached"]
    s2 = tled.Solver.from_problem(p)
    assert s2.autotune(trial_steps=10)["cached"]
    # the cached choice includes the step mode (streamed, resident or grid-resident)
    assert (s2.resident, s2.grid_resident) == (s.resident, s.grid_resident)
    o = m.init_state()
    m.step(o, 200)
    s.step(200)
    s.sync()
    c = compare(s.displacement(), s.temperature(), s.damage(), o.u, o.T, o.Omega)
    assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E


def _flags(p, tled, extra=0):
    return tled.COMPENSATED | (tled.EXPANSION if p.expansion else 0) | (tled.TEMP_DEP if p.temp_dep else 0) | extra


@pytest.mark.parametrize("kind", ["brick", "h8", "t4"])
def test_resident_mode_equals_streamed(kind):
    """A problem that fits one CTA's shared memory runs in the resident mode (K steps per
    launch, one CTA) by default; the streamed tile + shared-node kernels give the same
    numbers (same arithmetic in the same order)."""
    tled = _tled()
    prob = {"brick": lambda: W.cube_h8(n=8), "h8": lambda: W.cube_h8(n=6, jitter=0.15, seed=91),
            "t4": lambda: W.cube_t4(n=4, seed=92)}[kind]()
    outs = []
    for extra in (0, tled.STREAMED):
        s = tled.Solver.from_problem(prob, flags=_flags(prob, tled, extra))
        assert s.resident == (extra == 0)
        s.step(250)  # 7 full graph chunks and a partial one
        s.sync()
        outs.append((s.displacement(), s.temperature(), s.damage(), s.get_state()["v"]))
    assert np.abs(outs[0][0]).max() > 0 and outs[0][1].max() > prob.T0 + 0.01
    for a, b in zip(*outs):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-6 * np.abs(b).max() + 1e-30)


def test_resident_batch_scenarios_stop_at_their_own_step_count():
    """Three small H8 scenarios of different step counts in the resident mode (one CTA
    each, finished scenarios' CTAs return at once) against the streamed batch."""
    tled = _tled()
    scen = _scenarios_h8()
    n_steps = [300, 120, 210]
    res = []
    for extra in (0, tled.STREAMED):
        b = tled.Batch()
        for p, n in zip(scen, n_steps):
            b.add(p, n, flags=_flags(p, tled, extra))
        b.init()
        assert b.resident == (extra == 0)
        assert b.run() == max(n_steps)
        b.sync()
        res.append((b.displacement(), b.temperature(), b.damage()))
    for a, c in zip(*res):
        np.testing.assert_allclose(a, c, rtol=0, atol=1e-6 * np.abs(c).max() + 1e-30)


@pytest.mark.parametrize("kind", ["brick", "h8", "t4_cem"])
def test_grid_resident_mode_equals_streamed(kind):
    """A single problem too large for one CTA but whose tiles all fit co-resident CTAs runs
    in the grid-resident mode (one cooperative launch per graph chunk, grid barriers between
    the phases) by default; the streamed kernels give the same numbers."""
    tled = _tled()
    if kind == "brick":
        prob = W.block_h8(n=16, h=3e-3)
    elif kind == "h8":
        prob = W.cube_h8(n=12, jitter=0.15, seed=93)
    else:
        prob = W.liver_f2()
    outs = []
    for extra in (0, tled.STREAMED):
        f = _flags(prob, tled, extra) | (tled.CEM43 if getattr(prob, "cem43", False) else 0)
        s = tled.Solver.from_problem(prob, flags=f, dt=0.0 if kind == "t4_cem" else None)
        assert s.grid_resident == (extra == 0) and not s.resident
        s.step(100)  # 3 full graph chunks and a partial one
        s.sync()
        o = [s.displacement(), s.temperature(), s.damage(), s.get_state()["v"]]
        if kind == "t4_cem":
            o.append(s.cem43())
        outs.append(o)
    assert np.abs(outs[0][0]).max() > 0
    for a, b in zip(*outs):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-6 * np.abs(b).max() + 1e-30)


def test_grid_resident_checkpoint_and_source_change_match_streamed():
    """Grid-resident mode across a checkpoint/restore and a heat-source change between
    steps (stream-ordered upload), against the streamed kernels doing the same."""
    tled = _tled()
    prob = W.block_h8(n=16, h=3e-3)
    moved = np.array(prob.sources)
    moved[:, 0] += 2e-3
    outs = []
    for extra in (0, tled.STREAMED):
        f = _flags(prob, tled, extra)
        a = tled.Solver.from_problem(prob, flags=f)
        assert a.grid_resident == (extra == 0)
        a.step(45)
        blob = a.save_state()
        b = tled.Solver.from_problem(prob, flags=f)
        b.load_state(blob)
        b.set_heat_sources(moved)
        b.step(37)
        b.sync()
        outs.append((b.displacement(), b.temperature(), b.damage()))
    for x, y in zip(*outs):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-6 * np.abs(y).max() + 1e-30)
