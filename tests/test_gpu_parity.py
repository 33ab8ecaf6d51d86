"""Parity of the CUDA library against the FP64 oracle, element by element, on
the same seeded inputs (relative L2 of u and theta <= 1e-4, damage fraction
within 1e-3 absolute)."""
import numpy as np
import pytest

import oracle
from helpers import TOL_DAMAGE, TOL_E, compare, rel_l2, run_oracle
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _increments_match(s, m, st, os_, rtol=2e-5):
    """One step's velocity and temperature increments against the oracle's:
    these carry the element forces and thermal loads directly (u and T
    themselves are dominated by the state the step started from)."""
    g = s.get_state()
    free = m.prob.mask == 0
    dv_g = (g["v"] - st["v"])[free]
    dv_o = ((os_.u - os_.u_prev) / m.dt - st["v"])[free]
    assert np.abs(dv_g - dv_o).max() <= rtol * np.abs(dv_o).max(), np.abs(dv_g - dv_o).max() / np.abs(dv_o).max()
    dT_g, dT_o = g["T"] - st["T"], os_.T - st["T"]
    assert np.abs(dT_g - dT_o).max() <= rtol * np.abs(dT_o).max(), np.abs(dT_g - dT_o).max() / np.abs(dT_o).max()


def _tled():
    from paper_2009_10400_b300 import tled
    return tled


def _gpu_run(prob, n_steps, dt, every=None, tile_elems=0):
    tled = _tled()
    s = tled.Solver.from_problem(prob, dt=dt, tile_elems=tile_elems)
    snaps = []
    every = every or n_steps
    done = 0
    while done < n_steps:
        k = min(every, n_steps - done)
        s.step(k)
        s.sync()
        done += k
        snaps.append((done, s.displacement(), s.temperature(), s.damage()))
    return s, snaps


def _check_trajectory(prob, n_steps, every, tile_elems=0, tol_e=TOL_E):
    m, _, ref = run_oracle(prob, n_steps, every)
    _, got = _gpu_run(prob, n_steps, m.dt, every, tile_elems)
    worst = {}
    for (k, u_r, T_r, O_r), (k2, u, T, d) in zip(ref, got):
        assert k == k2
        c = compare(u, T, d, u_r, T_r, O_r, prob.T0)
        for key, v in c.items():
            worst[key] = max(worst.get(key, 0.0), v)
        assert c["e_u"] <= tol_e, (k, c)
        assert c["e_theta"] <= tol_e, (k, c)
        assert c["d_abs"] <= TOL_DAMAGE, (k, c)
    return worst


def test_cube_h8_2000_steps_matches_oracle():
    """5 cm cube of 8^3 H8, 2000 steps at the stable step, oracle every 500."""
    prob = W.cube_h8(n=8)
    w = _check_trajectory(prob, 2000, 500)
    print("cube_h8", w)


def test_cube_t4_ragged_tiles_matches_oracle():
    """Kuhn-split jittered tet cube (1296 tets: two tiles, the second ragged),
    per-element material noise and vMF fibres, moving source."""
    prob = W.cube_t4(n=6)
    w = _check_trajectory(prob, 600, 200)
    print("cube_t4", w)


def test_block_h8_noise_many_tiles_matches_oracle():
    """16^3 H8 block (8 tiles, interior and shared nodes) with +-10% material noise."""
    prob = W.block_h8(n=16, h=3e-3)
    w = _check_trajectory(prob, 400, 200)
    print("block_h8_16", w)


@pytest.mark.parametrize("shape", ["graded", "rotated"])
def test_graded_and_rotated_h8_blocks_match_oracle(shape):
    """Axis-aligned boxes of graded size (every element its own diagonal J0^-1)
    take the brick kernel; the same block rotated by 30 degrees about z (still
    parallelepipeds, J0 no longer diagonal) keeps the general H8 kernel.  Both
    against the oracle."""
    import dataclasses
    tled = _tled()
    prob = W.block_h8(n=12, h=3e-3)
    X = prob.X.copy()
    L = X.max(axis=0)
    if shape == "graded":  # x -> L (x / L)^1.4 per axis: monotone, every spacing different
        X = L * (X / L) ** 1.4
    else:
        c, s_ = np.cos(np.pi / 6), np.sin(np.pi / 6)
        X = np.stack([c * X[:, 0] - s_ * X[:, 1], s_ * X[:, 0] + c * X[:, 1], X[:, 2]], axis=1)
    prob = dataclasses.replace(prob, X=X)
    s = tled.Solver.from_problem(prob)
    assert s.brick == (shape == "graded")
    w = _check_trajectory(prob, 400, 200)
    print(shape, w)


def test_small_tiles_exercise_shared_nodes():
    """Tiny tiles (37 elements) make most nodes shared between tiles: the
    second-pass gather must give the same answer."""
    prob = W.cube_h8(n=6, jitter=0.2)
    w = _check_trajectory(prob, 300, 100, tile_elems=37)
    print("small tiles", w)


def test_ellipsoid_t4_matches_oracle():
    """Coarse seeded Delaunay ellipsoid 'liver' with vMF fibres and a moving source."""
    prob = W.ellipsoid_t4(spacing=9e-3)
    w = _check_trajectory(prob, 300, 100)
    print("ellipsoid", prob.ne, w)



@pytest.mark.parametrize("kind", ["h8", "t4"])
def test_large_extension_40pct_matches_oracle(kind):
    """Finite strain: the top face pulled up by 40 % of the edge (ramped over
    0.05 s, bottom fixed) on a compressible variant of the tissue (kappa =
    2 mu), so that |J - 1| exceeds 0.1 and the log1p/expm1 branch of
    J^(-2/3) - 1 runs beside the series; trajectory against the oracle."""
    prob = W.cube_h8(n=4, jitter=0.1, seed=61) if kind == "h8" else W.cube_t4(n=3, seed=62)
    prob.kappa[:] = 2.0 * prob.mu
    L = np.ptp(prob.X[:, 2])
    top = np.isclose(prob.X[:, 2], prob.X[:, 2].max())
    prob.mask = prob.mask.copy()
    prob.mask[top] = W.MASK_U
    prob.ubar = np.zeros((prob.nn, 3))
    prob.ubar[top, 2] = 0.4 * L
    prob.ramp_time = 0.05
    w = _check_trajectory(prob, 600, 150)
    print("extension", kind, w)
    _, s, _ = run_oracle(prob, 600, 600)
    assert np.ptp(s.u[:, 2] + prob.X[:, 2]) / L > 1.35  # the stretch was applied


def _aniso(prob, tilt=True):
    """Transversely isotropic thermal physics: three times the expansion and 2.5
    times the conductivity along the fibre, expansion made large enough to
    matter (alpha 2e-3), fibres tilted off the mesh axes."""
    prob.aniso_alpha, prob.aniso_k = 3.0, 2.5
    prob.alpha[:] = 2e-3
    if tilt and not prob.per_element:
        prob.a0[:] = np.array([1.0, 1.0, 0.5]) / 1.5
    return prob


@pytest.mark.parametrize("kind", ["h8", "t4"])
def test_anisotropic_thermal_physics_matches_oracle(kind):
    """Eq. 11's transversely isotropic thermal expansion about the fibre and
    conduction along the current fibre: heating trajectory against the oracle
    (H8 cube with tilted fibres, T4 cube with vMF fibres)."""
    prob = _aniso(W.cube_h8(n=6, jitter=0.1, seed=81) if kind == "h8" else W.cube_t4(n=5, seed=82))
    w = _check_trajectory(prob, 1500, 500)
    print("aniso", kind, w)


@pytest.mark.parametrize("kind", ["h8", "t4"])
def test_anisotropic_single_step_from_random_state(kind):
    tled = _tled()
    prob = _aniso(W.block_h8(n=8, h=4e-3) if kind == "h8" else W.cube_t4(n=5))
    st = W.random_state(prob, 23, theta_scale=20.0)
    m = oracle.OracleModel(prob)
    s = tled.Solver.from_problem(prob, dt=m.dt)
    s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"], t=0.01, step=5)
    s.step(1)
    s.sync()
    os_ = m.state_from(**st, t=0.01, step=5)
    m.step(os_, 1)
    np.testing.assert_allclose(s.displacement(), os_.u, rtol=0, atol=2e-6 * np.abs(os_.u).max())
    np.testing.assert_allclose(s.temperature(), os_.T, rtol=0, atol=2e-6 * np.abs(os_.T - 37).max())
    _increments_match(s, m, st, os_)
    # the anisotropic stable step and stored energy agree with the oracle's
    np.testing.assert_allclose(s.get_dt()[1:], (m.dt_mech, m.dt_th), rtol=1e-12)
    s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"])
    r = s.stats()
    ref = sum(m.energy(e, st["u"], st["T"]) for e in range(prob.ne))
    assert abs(r["strain_energy"] + r["hourglass_energy"] - ref) <= 1e-5 * abs(ref)

def test_auto_dt_matches_oracle():
    tled = _tled()
    for prob in (W.cube_h8(n=8), W.cube_t4(n=4), W.ellipsoid_t4(spacing=1.2e-2)):
        m = oracle.OracleModel(prob)
        s = tled.Solver.from_problem(prob)
        dt, dtm, dtt = s.get_dt()
        np.testing.assert_allclose(dt, m.dt, rtol=1e-12)
        np.testing.assert_allclose(dtm, m.dt_mech, rtol=1e-12)
        np.testing.assert_allclose(dtt, m.dt_th, rtol=1e-12)


@pytest.mark.parametrize("kind", ["h8", "t4"])
def test_single_step_from_random_state(kind):
    """One step from a seeded mid-run state (large u, theta, Prony state):
    every node's new u, T and Omega against the oracle."""
    tled = _tled()
    prob = W.block_h8(n=10, h=4e-3) if kind == "h8" else W.cube_t4(n=5)
    st = W.random_state(prob, 17)
    m = oracle.OracleModel(prob)
    s = tled.Solver.from_problem(prob, dt=m.dt, tile_elems=100)
    s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"], t=0.01, step=5)
    s.step(1)
    s.sync()
    os_ = m.state_from(**st, t=0.01, step=5)
    m.step(os_, 1)
    u, T, d = s.displacement(), s.temperature(), s.damage()
    np.testing.assert_allclose(u, os_.u, rtol=0, atol=2e-6 * np.abs(os_.u).max())
    np.testing.assert_allclose(T, os_.T, rtol=0, atol=2e-6 * np.abs(os_.T - 37).max())
    np.testing.assert_allclose(d, oracle.damage_fraction(os_.Omega), rtol=0, atol=1e-6)
    g = s.get_state()
    np.testing.assert_allclose(g["visc"], os_.visc, rtol=0, atol=1e-5 * np.abs(os_.visc).max())
    _increments_match(s, m, st, os_)


def test_deterministic_bitwise():
    tled = _tled()
    prob = W.block_h8(n=12, h=4e-3)
    outs = []
    for _ in range(2):
        s = tled.Solver.from_problem(prob, tile_elems=64)
        s.step(200)
        s.sync()
        outs.append((s.displacement(), s.temperature(), s.damage()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("streamed", [True, False])
def test_any_split_of_the_steps_is_bitwise_the_same(streamed):
    """A call of n steps replays the cached graphs of n's binary digits (and of
    32-step chunks): 69 steps in one call, one step at a time, and as 5 + 64 give
    bitwise the same state, in the streamed and in the resident mode."""
    tled = _tled()
    prob = W.block_h8(n=12, h=4e-3)
    flags = tled.default_flags(prob) | (tled.STREAMED if streamed else 0)
    outs = []
    for split in ([69], [1] * 69, [5, 64]):
        s = tled.Solver.from_problem(prob, flags=flags, tile_elems=64)
        assert (s.resident or s.grid_resident) == (not streamed)
        for n in split:
            s.step(n)
        s.sync()
        outs.append((s.displacement(), s.temperature(), s.damage()))
    assert np.abs(outs[0][0]).max() > 0
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


def test_brick_kernel_matches_general_h8():
    """An axis-aligned H8 block (vanishing reference hourglass projections,
    diagonal J0^-1) takes the brick kernel, which drops those terms and the
    round-off off-diagonal entries of J0^-1 (~1e-14 of the diagonal); the
    general H8 kernel computes them.  The two agree within 1e-6 after 400 steps;
    jittered H8 meshes, which keep the general kernel, are checked against the
    oracle above."""
    tled = _tled()
    prob = W.block_h8(n=20, h=3e-3)
    base = tled.COMPENSATED | tled.EXPANSION | (tled.TEMP_DEP if prob.temp_dep else 0)
    outs = []
    for flags in (base, base | tled.GENERAL_H8):
        s = tled.Solver.from_problem(prob, flags=flags)
        assert s.brick == (flags == base)
        s.step(400)
        s.sync()
        outs.append((s.displacement(), s.temperature() - prob.T0, s.damage()))
    assert np.abs(outs[0][0]).max() > 0 and outs[0][1].max() > 0.01
    assert rel_l2(outs[0][0], outs[1][0]) <= 1e-6
    assert rel_l2(outs[0][1], outs[1][1]) <= 1e-6
    assert np.abs(outs[0][2] - outs[1][2]).max() <= 1e-9


def test_checkpoint_resume_bitwise():
    tled = _tled()
    prob = W.cube_t4(n=5)
    a = tled.Solver.from_problem(prob)
    a.step(300)
    a.sync()
    ref = (a.displacement(), a.temperature(), a.damage())
    b = tled.Solver.from_problem(prob)
    b.step(150)
    blob = b.save_state()
    c = tled.Solver.from_problem(prob)
    c.load_state(blob)
    c.step(150)
    c.sync()
    got = (c.displacement(), c.temperature(), c.damage())
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    bad = bytearray(blob)
    bad[-1] ^= 0xFF
    with pytest.raises(tled.TledError) as ei:
        c.load_state(bytes(bad))
    assert ei.value.code == tled.E_FORMAT


def test_stats_match_state():
    tled = _tled()
    prob = W.cube_h8(n=8)
    s = tled.Solver.from_problem(prob)
    s.step(500)
    st = s.stats()
    T = s.temperature()
    u = s.displacement()
    assert st["status"] == 0
    np.testing.assert_allclose(st["T_max"], T.max(), rtol=1e-12)
    np.testing.assert_allclose(st["T_min"], T.min(), rtol=1e-12)
    np.testing.assert_allclose(st["u_max"], np.linalg.norm(u, axis=1).max(), rtol=1e-6)
    m = oracle.OracleModel(prob)
    np.testing.assert_allclose(st["heat_content"], (m.Cth * (T - 37.0)).sum(), rtol=1e-6)



def test_energy_reduction_matches_oracle():
    """The FP64 stored and hourglass energies of tled_get_stats against the
    oracle's element energies on random mid-run states with strains of order
    0.1-0.3 (jittered H8 with hourglass energy, a brick H8 cube -- its records
    hold the diagonal of J0^-1 --, T4 with per-element fibres)."""
    tled = _tled()
    cases = ((W.cube_h8(n=6, jitter=0.1, seed=8), False), (W.cube_h8(n=6, seed=8), True),
             (W.cube_t4(n=5, seed=9), False))
    for prob, brick in cases:
        st = W.random_state(prob, seed=3, u_scale=2e-3)
        s = tled.Solver.from_problem(prob)
        assert s.brick == brick
        s.set_state(st["u"], st["v"], st["T"], st["Omega"], st["visc"])
        r = s.stats()
        m = oracle.OracleModel(prob)
        ref = sum(m.energy(e, st["u"], st["T"]) for e in range(prob.ne))
        got = r["strain_energy"] + r["hourglass_energy"]
        assert abs(got - ref) <= 1e-5 * abs(ref), (prob.name, got, ref)
        if prob.npe == 4:
            assert r["hourglass_energy"] == 0.0
        else:
            assert 0.0 < r["hourglass_energy"] < r["strain_energy"]
        v = st["v"]
        ke = 0.5 * np.sum(m.M[:, None] * v * v)
        np.testing.assert_allclose(r["kinetic_energy"], ke, rtol=1e-6)


def test_energy_balance_on_gpu():
    """P9 on the device: the mechanical energy (mean kinetic energy of the two
    half steps around u_n plus the stored and hourglass energies, all from the
    FP64 reduction) only oscillates, within 1 % over 1500 steps, and follows
    the oracle's energy history."""
    from helpers import p9_energy_history, p9_initial, p9_problem
    tled = _tled()
    p = p9_problem()
    u0 = p9_initial(p)
    s = tled.Solver.from_problem(p)
    z = np.zeros_like(u0)
    s.set_state(u0, z, np.full(p.nn, p.T0), np.zeros(p.nn))
    E = []
    for _ in range(30):
        a = s.stats()
        s.step(1)
        b = s.stats()
        E.append(0.5 * (a["kinetic_energy"] + b["kinetic_energy"]) + a["strain_energy"] + a["hourglass_energy"])
        s.step(49)
    E = np.array(E)
    assert np.ptp(E) / E[0] < 1e-2
    m = oracle.OracleModel(p)
    assert s.get_dt()[0] == pytest.approx(m.dt, rel=1e-12)  # both derive the stable step (R16) on their own
    ref = p9_energy_history(m, p, u0, 30, 50)
    np.testing.assert_allclose(E, ref, rtol=1e-4)

def test_inversion_is_reported():
    """A huge prescribed compression of a single element inverts it; the device
    flags the element and tled_sync reports E_INVERTED (no device trap)."""
    tled = _tled()
    X, conn = W.hex_grid((1, 1, 1), (0.01, 0.01, 0.01))
    mat = W._material(1)
    ubar = np.zeros((8, 3))
    ubar[X[:, 2] > 0.005, 2] = -0.02  # top face pushed 2 cm below the bottom
    mask = np.full(8, W.MASK_U, np.uint8)
    prob = W.Problem(name="inv", npe=8, X=X, conn=conn, **mat, mask=mask, ubar=ubar, ramp_time=0.0)
    s = tled.Solver.from_problem(prob, dt=1e-5)
    s.step(3)
    with pytest.raises(tled.TledError) as ei:
        s.sync()
    assert ei.value.code == tled.E_INVERTED


@pytest.mark.parametrize("n_sub", [3, 8])
def test_subcycled_trajectory_matches_oracle(n_sub):
    """Mechanical subcycling (study f4): n_sub mechanical substeps per thermal
    step of 4 x the stable step, coupled heating with thermal expansion and
    Prony viscosity, against the oracle's own subcycled step
    (ora_step_subcycled); compared after every 20 thermal steps."""
    tled = _tled()
    p = W.cube_h8(n=6, jitter=0.15, seed=61)
    p.sources = np.array([W.source((0.02, 0.025, 0.03), 9e6, sigma=6e-3, vel=(0.01, 0.0, -0.005))])
    m1 = oracle.OracleModel(p)  # the stable (mechanical) step
    p.n_sub, p.dt = n_sub, 0.9 * n_sub * m1.dt
    m = oracle.OracleModel(p)
    g = tled.Solver.from_problem(p)
    assert g.get_dt()[0] == pytest.approx(p.dt / n_sub, rel=1e-15)
    s = m.init_state()
    for _ in range(5):
        m.step_thermal(s, 20)
        g.step(20 * n_sub)
        g.sync()
        c = compare(g.displacement(), g.temperature(), g.damage(), s.u, s.T, s.Omega, p.T0)
        assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E and c["d_abs"] <= TOL_DAMAGE, c
    print(f"subcycled n_sub={n_sub}", c)
    assert s.T.max() - p.T0 > 0.05 and np.abs(s.u).max() > 1e-9


def test_l2_window_is_set_and_the_limit_restored():
    """The streamed step's persisting-L2 window covers the shared nodes' (u, theta)
    and the partial sums; the context's persisting set-aside is raised for it
    and put back when the library context is destroyed."""
    from cuda.bindings import runtime as rt
    tled = _tled()
    lim = rt.cudaLimit.cudaLimitPersistingL2CacheSize
    err, before = rt.cudaDeviceGetLimit(lim)
    assert err == rt.cudaError_t.cudaSuccess
    prob = W.block_h8(n=12, h=4e-3)
    s = tled.Solver.from_problem(prob, flags=tled.default_flags(prob) | tled.STREAMED, tile_elems=64)
    info, w = s.plan_info(), s.l2_window()
    assert info["n_shared"] > 0
    assert w["window_bytes"] >= 16 * (info["n_shared"] + info["n_partials"])
    assert w["set_aside_bytes"] > 0 and 0.0 < w["hit_ratio"] <= 1.0
    s.step(10)
    s.sync()
    s.close()
    err, after = rt.cudaDeviceGetLimit(lim)
    assert err == rt.cudaError_t.cudaSuccess and after == before
