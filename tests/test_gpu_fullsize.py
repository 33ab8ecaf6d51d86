"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times: one step from a seeded mid-run state, with the oracle
computing sampled nodes one by one (its step_nodes), and properties that hold
at any size (the per-step heat balance)."""
import numpy as np
import pytest

import oracle
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _tled():
    from paper_2009_10400_b300 import tled
    return tled


def _compare_nodes(u, T, d, nodes, ou, oT, oO, T0):
    np.testing.assert_allclose(u[nodes], ou, rtol=0, atol=2e-6 * max(np.abs(ou).max(), 1e-30))
    np.testing.assert_allclose(T[nodes], oT, rtol=0, atol=2e-6 * max(np.abs(oT - T0).max(), 1e-30))
    np.testing.assert_allclose(d[nodes], oracle.damage_fraction(oO), rtol=0, atol=1e-6)


def test_block_h8_128_single_step_sampled_nodes_and_heat_balance():
    """The 128^3 block (2,097,152 H8, 2,146,689 nodes) exactly as the benchmark
    builds it: one step from a random mid-run state; 4096 sampled nodes against
    the oracle, and over all nodes the exact per-step heat balance (element
    conduction loads sum to zero, so the change of heat content is the source
    heat minus perfusion)."""
    tled = _tled()
    prob = W.block_h8(n=128)
    st = W.random_state(prob, 31, u_scale=2e-5, theta_scale=8.0)
    m = oracle.OracleModel(prob)
    s = tled.Solver.from_problem(prob)
    dt = s.get_dt()[0]
    assert dt == pytest.approx(m.dt, rel=1e-12)
    s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"], t=0.02, step=7)
    h0 = s.stats()["heat_content"]
    s.step(1)
    s.sync()
    u, T, d = s.displacement(), s.temperature(), s.damage()
    h1 = s.stats()["heat_content"]
    rng = np.random.default_rng(5)
    nodes = np.sort(rng.choice(prob.nn, 4096, replace=False))
    os_ = m.state_from(**st, t=0.02, step=7)
    ou, oT, oO = m.step_nodes(os_, nodes)
    _compare_nodes(u, T, d, nodes, ou, oT, oO, prob.T0)
    # heat balance over every node: sum_i C_i (theta+ - theta) = dt sum_i (V_i Q_i - Kb_i theta_i)
    x = prob.X + st["u"]
    Q = np.zeros(prob.nn)
    for r in np.asarray(prob.sources):
        c = r[0:3] + r[3:6] * 0.02
        Q += r[7] * np.exp(-((x - c) ** 2).sum(1) / (2 * r[6] ** 2))
    Kb = prob.wbcb * m.Vn
    th = st["T"] - prob.T0
    expect = dt * np.sum(m.Vn * Q - Kb * th)
    scale = dt * np.sum(np.abs(m.Vn * Q) + np.abs(Kb * th))
    got = h1 - h0
    # FP32 rounding of the per-node update and of the element loads is ~1e-7 of
    # the scale; a wrong sign or a dropped term would be O(1)
    assert abs(got - expect) <= 1e-4 * scale, (got, expect, scale)


def test_ellipsoid_t4_full_size_single_step_every_node():
    """The ~120k-tet Delaunay ellipsoid at full size: one step from a random
    state, every node against the oracle."""
    tled = _tled()
    prob = W.ellipsoid_t4()
    assert 90_000 < prob.ne < 150_000
    st = W.random_state(prob, 32, u_scale=1e-4)
    m = oracle.OracleModel(prob)
    s = tled.Solver.from_problem(prob)
    s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"], t=0.1, step=3)
    s.step(1)
    s.sync()
    os_ = m.state_from(**st, t=0.1, step=3)
    m.step(os_, 1)
    _compare_nodes(s.displacement(), s.temperature(), s.damage(), np.arange(prob.nn), os_.u, os_.T, os_.Omega,
                   prob.T0)


def test_planning_batch_256_single_step_sampled():
    """The 256-scenario mixed hex/tet planning batch, mass-scaled, autotuned as
    the benchmark runs it: one step from random per-scenario states; 12
    scenarios' sampled nodes against each scenario's own oracle model."""
    tled = _tled()
    scen = W.planning_scenarios(256)  # R17 mass scale: the library's and the oracle's own choice
    b = tled.Batch()
    for p in scen:
        b.add(p, p.n_steps)
    b.init()
    b.autotune(trial_steps=10)
    # the persisting-L2 window of this batch is larger than the 40 % of L2 the library sets
    # aside at most: the hit ratio covers only the capped share
    from cuda.bindings import runtime as rt
    err, l2 = rt.cudaDeviceGetAttribute(rt.cudaDeviceAttr.cudaDevAttrL2CacheSize, 0)
    assert err == rt.cudaError_t.cudaSuccess
    w = b.l2_window()
    assert w["window_bytes"] > 0.4 * l2
    assert 0.0 < w["hit_ratio"] <= 0.4 * l2 / w["window_bytes"] + 1e-6
    states = [W.random_state(p, 100 + i, u_scale=1e-4, n_prony=len(p.prony_g)) for i, p in enumerate(scen)]
    cat = {k: np.concatenate([st[k] for st in states]) for k in ("u", "v", "T", "Omega", "visc")}
    b.set_state(cat["u"], cat["v"], cat["T"], cat["Omega"], cat["visc"], t=0.05, step=5)
    b.step(1)
    b.sync()
    u, T, d = b.displacement(), b.temperature(), b.damage()
    rng = np.random.default_rng(6)
    picks = sorted(set(rng.choice(len(scen), 10, replace=False)) | {0, len(scen) - 1})
    kinds = set()
    for i in picks:
        p, st = scen[i], states[i]
        info = b.scenario(i)
        off = info["node_off"]
        m = oracle.OracleModel(p)  # the scenario's fixed dt (0.01 s) and the oracle's own R17 mass scale
        assert b.scenario_dt(i) == m.dt
        os_ = m.state_from(**st, t=0.05, step=5)
        nodes = np.sort(rng.choice(p.nn, min(256, p.nn), replace=False))
        ou, oT, oO = m.step_nodes(os_, nodes)
        _compare_nodes(u[off:off + p.nn], T[off:off + p.nn], d[off:off + p.nn], nodes, ou, oT, oO, p.T0)
        kinds.add(p.npe)
    assert kinds == {4, 8}
