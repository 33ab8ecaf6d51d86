"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an exact
discrete closed form, an invariant, a brute-force finite difference, or a
scalar closed form derived independently of the oracle's tensor code.
"""
import numpy as np
import pytest

import oracle
from helpers import p9_energy_history, p9_initial, p9_problem
from paper_2009_10400_b300 import workloads as W


def _bar(n=16, L=0.08, w=0.005, **kw):
    X, conn = W.hex_grid((n, 1, 1), (L, w, w))
    ne = conn.shape[0]
    mat = W._material(ne, alpha=0.0)
    p = W.Problem(name="bar", npe=8, X=X, conn=conn, **mat, prony_g=(), prony_tau=(), **kw)
    return p


# ---------------------------------------------------------------------------
# P1: conduction operator, sign (R1), lumping (R10), explicit Euler (Eq. 20)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("stretch,aniso_k", [(1.0, 1.0), (1.3, 1.0), (1.0, 2.5), (1.3, 2.5)])
def test_p1_cosine_mode_exact_discrete_decay(stretch, aniso_k):
    """On an adiabatic n x 1 x 1 H8 bar the one-point operator acting on an
    x-only field is the 3-point stencil, so a cosine mode decays by an exact
    factor per step.  With the bar held at a uniform stretch s (all
    displacements prescribed) conduction in the deformed configuration (Eq. 6)
    scales the conductivity by J C^-1_xx = 1/s.  With fibres along the bar and
    anisotropic conductivity the bar conducts with k_fibre = aniso_k k (the
    current fibre stays along x, so the same 1/s applies)."""
    n, L, A = 16, 0.08, 2.0
    p = _bar(n, L)
    p.aniso_k = aniso_k
    h = L / n
    if stretch != 1.0:
        p.mask[:] = W.MASK_U
        p.ubar = np.zeros((p.nn, 3))
        p.ubar[:, 0] = (stretch - 1.0) * p.X[:, 0]
    p.dt = 0.5
    m = oracle.OracleModel(p)
    s = m.init_state()
    x = p.X[:, 0]
    s.T[:] = p.T0 + A * np.cos(np.pi * x / L)
    if stretch != 1.0:
        s.u[:] = p.ubar
        s.u_prev[:] = p.ubar
    nsteps = 200
    m.step(s, nsteps)
    rho, c, k = 1000.0, p.c_heat, 0.5 * aniso_k
    r = 1.0 - p.dt * 4.0 * k / (stretch * rho * c * h * h) * np.sin(np.pi * h / (2 * L)) ** 2 \
        - p.dt * p.wbcb / (rho * c)
    expect = p.T0 + A * np.cos(np.pi * x / L) * r ** nsteps
    np.testing.assert_allclose(s.T - p.T0, expect - p.T0, rtol=1e-9, atol=1e-12)


def test_p1_linear_profile_is_steady_with_held_ends():
    """Steady 1D conduction: a linear profile between held end temperatures
    (no perfusion) is a fixed point of Eq. (20)."""
    p = _bar(12, 0.06, wbcb=0.0)
    x = p.X[:, 0]
    ends = np.isclose(x, 0.0) | np.isclose(x, 0.06)
    p.mask[ends] |= W.MASK_T
    p.dt = 1.0
    m = oracle.OracleModel(p)
    s = m.init_state()
    s.T[:] = 37.0 + 20.0 * x / 0.06
    T0 = s.T.copy()
    m.step(s, 100)
    np.testing.assert_allclose(s.T, T0, rtol=0, atol=1e-11)


def test_p1_temperature_dependent_conductivity():
    """k(T) linear in T (Table 5 interpolation): a small cosine mode around a
    base temperature decays with k(T_base) = k (1 + beta_k (T_base - T_ref))."""
    n, L = 16, 0.08
    beta_k = (0.75 / 0.53 - 1.0) / 53.0
    p = _bar(n, L, wbcb=0.0, temp_dep=True, beta_k=beta_k, beta_c=0.0)
    p.dt = 1.0
    m = oracle.OracleModel(p)
    s = m.init_state()
    x = p.X[:, 0]
    Tb, A = 60.0, 1e-3
    s.T[:] = Tb + A * np.cos(np.pi * x / L)
    m.step(s, 1000)
    h = L / n
    keff = 0.5 * (1.0 + beta_k * (Tb - 37.0))
    r = 1.0 - p.dt * 4.0 * keff / (1000.0 * p.c_heat * h * h) * np.sin(np.pi * h / (2 * L)) ** 2
    # the O(beta_k A^2) nonlinearity of k(T_e) is far below the tolerance; using k
    # instead of k(T_base) would miss by ~3e-5
    np.testing.assert_allclose(s.T - Tb, A * np.cos(np.pi * x / L) * r ** 1000, rtol=0, atol=2e-9)


# ---------------------------------------------------------------------------
# uniform fields: perfusion / source / c(T) closed forms of Eq. (20)
# ---------------------------------------------------------------------------
def test_uniform_source_and_perfusion_recurrence():
    """Uniform T, uniform source Q (very wide Gaussian), perfusion w_b c_b:
    theta_n = theta_inf + (theta_0 - theta_inf) r^n with theta_inf = Q / (w_b c_b)
    and r = 1 - dt w_b c_b / (rho c): the exact discrete solution of Eq. (20)."""
    p = W.cube_h8(n=3)
    p.expansion = False
    Q = 2.0e5
    p.sources = np.array([W.source((0.025,) * 3, Q, sigma=1e6)])
    p.dt = 0.05
    m = oracle.OracleModel(p)
    s = m.init_state()
    m.step(s, 400)
    rho, c = 1000.0, p.c_heat
    th_inf = Q / p.wbcb
    r = 1.0 - p.dt * p.wbcb / (rho * c)
    expect = th_inf + (0.0 - th_inf) * r ** 400
    np.testing.assert_allclose(s.T - 37.0, expect, rtol=1e-6)


def test_temperature_dependent_heat_capacity():
    """Adiabatic uniform heating with c(T) = c (1 + beta_c (T - T_ref)):
    rho c ((T - T_ref) + beta_c/2 (T - T_ref)^2) = Q t (continuous solution);
    explicit Euler agrees to O(dt)."""
    beta_c = (4300.0 / 3600.0 - 1.0) / 53.0
    p = W.cube_h8(n=2)
    p.expansion = False
    p.temp_dep, p.beta_c, p.wbcb = True, beta_c, 0.0
    Q = 1.0e6
    p.sources = np.array([W.source((0.025,) * 3, Q, sigma=1e6)])
    p.dt = 0.01
    m = oracle.OracleModel(p)
    s = m.init_state()
    m.step(s, 2000)
    t = 20.0
    rc = 1000.0 * p.c_heat
    # solve rc (x + beta_c x^2 / 2) = Q t
    a, b, cc = rc * beta_c / 2, rc, -Q * t
    x = (-b + np.sqrt(b * b - 4 * a * cc)) / (2 * a)
    np.testing.assert_allclose(s.T - 37.0, x, rtol=2e-4)
    # without temperature dependence the rise would be Q t / (rho c), which differs
    assert abs(Q * t / rc - x) / x > 0.005


# ---------------------------------------------------------------------------
# P2: thermal expansion split + pull-back (Eqs. 7-11)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,aniso", [("h8", False), ("t4", False), ("h8", True), ("t4", True)])
def test_p2_free_thermal_expansion_is_stress_free(kind, aniso):
    """An unconstrained body at uniform theta with u = (F_th - I)(X - Xc) has
    zero nodal force: the elastic part of the deformation is the identity.
    Isotropic F_th = lambda I, or transversely isotropic about a tilted fibre
    m (Eq. 11) with three times the expansion along it."""
    p = W.cube_h8(n=3, jitter=0.2) if kind == "h8" else W.cube_t4(n=3)
    p.mask[:] = 0
    p.dt = 1e-5
    alpha = 1e-4
    p.alpha[:] = alpha  # uniform expansion coefficient: a homogeneous free-expansion field
    mvec = np.array([1.0, 0.0, 0.0])
    if aniso:
        mvec = np.array([1.0, 1.0, 0.5]) / 1.5
        p.a0[:] = mvec
        p.aniso_alpha, p.aniso_k = 3.0, 2.0
    m = oracle.OracleModel(p)
    s = m.init_state()
    theta = 12.0
    s.T[:] = p.T0 + theta
    lam = 1.0 + alpha * theta
    lam_m = 1.0 + p.aniso_alpha * alpha * theta
    Fth = lam * np.eye(3) + (lam_m - lam) * np.outer(mvec, mvec)
    Xc = p.X.mean(0)
    s.u[:] = (p.X - Xc) @ (Fth - np.eye(3)).T
    s.u_prev[:] = s.u
    m.step(s, 1)
    f, fT = m.forces()
    scale = p.mu.max() * 0.05 ** 2 * (lam - 1.0)
    assert np.abs(f).max() < 1e-9 * scale
    assert np.abs(fT).max() < 1e-12
    # the same displacement without the thermal split is strongly stressed
    p.expansion = False
    m2 = oracle.OracleModel(p)
    s2 = m2.init_state()
    s2.T[:] = p.T0 + theta
    s2.u[:] = s.u_prev
    s2.u_prev[:] = s.u_prev
    m2.step(s2, 1)
    f2, _ = m2.forces()
    assert np.abs(f2).max() > 1e-3 * scale


# ---------------------------------------------------------------------------
# P3: homogeneous uniaxial stretch, scalar closed form of the stress
# ---------------------------------------------------------------------------
def _dW(l1, l2, mu, kappa, k1, k2, lam=1.0):
    """Partial derivatives dW/dl1 and dW/dl2 of the thermally split energy
    W = lam^3 Psi(diag(l1, l2, l2) / lam) written as a scalar function of the
    stretches (Table 5 + R7), differentiated by hand."""
    a, b = l1 / lam, l2 / lam
    J = a * b * b
    Jm23 = J ** (-2.0 / 3.0)
    Jm53 = J ** (-5.0 / 3.0)
    I1 = a * a + 2 * b * b
    x = Jm23 * a * a - 1.0
    dpsi_f = k1 * x * np.exp(k2 * x * x)
    # d/da and d/db of Psi(a, b, b)
    dI1b_da = 2 * a * Jm23 - 2.0 / 3.0 * Jm53 * b * b * I1
    dI1b_db = 4 * b * Jm23 - 2.0 / 3.0 * Jm53 * 2 * a * b * I1
    dI4b_da = 2 * a * Jm23 - 2.0 / 3.0 * Jm53 * b * b * a * a
    dI4b_db = -2.0 / 3.0 * Jm53 * 2 * a * b * a * a
    dPa = 0.5 * mu * dI1b_da + kappa * (J - 1) * b * b + dpsi_f * dI4b_da
    dPb = 0.5 * mu * dI1b_db + kappa * (J - 1) * 2 * a * b + dpsi_f * dI4b_db
    # chain rule through a = l1/lam, b = l2/lam and the lam^3 factor
    return lam ** 2 * dPa, lam ** 2 * dPb


@pytest.mark.parametrize("theta", [0.0, 30.0])
def test_p3_uniaxial_stretch_face_forces(theta):
    """Homogeneous F = diag(l1, l2, l2) (all nodes prescribed): interior nodal
    forces vanish and face force sums equal P11 * A and P22 * A, with P from the
    hand-differentiated scalar energy (fibres along x, HGO fibre term)."""
    n, Ls = 3, 0.03
    X, conn = W.hex_grid((n, n, n), (Ls, Ls, Ls))
    mat = W._material(conn.shape[0], alpha=1e-3)
    p = W.Problem(name="uni", npe=8, X=X, conn=conn, **mat, prony_g=(), prony_tau=(),
                  mask=np.full(X.shape[0], W.MASK_U, np.uint8))
    l1, l2 = 1.25, 0.93
    p.ubar = np.stack([(l1 - 1) * X[:, 0], (l2 - 1) * X[:, 1], (l2 - 1) * X[:, 2]], 1)
    p.dt = 1e-6
    m = oracle.OracleModel(p)
    s = m.init_state()
    s.u[:] = p.ubar
    s.u_prev[:] = p.ubar
    s.T[:] = p.T0 + theta
    m.step(s, 1)
    f, _ = m.forces()
    lam = 1.0 + 1e-3 * theta
    P11, P22x2 = _dW(l1, l2, 3e3, 3e5, 1e3, 10.0, lam)
    A = Ls * Ls
    right = np.isclose(X[:, 0], Ls)
    top = np.isclose(X[:, 1], Ls)
    np.testing.assert_allclose(f[right, 0].sum(), P11 * A, rtol=1e-10)
    np.testing.assert_allclose(f[top, 1].sum(), 0.5 * P22x2 * A, rtol=1e-10)
    inner = np.all((X > 1e-9) & (X < Ls - 1e-9), axis=1)
    assert np.abs(f[inner]).max() < 1e-10 * abs(P11) * A


# ---------------------------------------------------------------------------
# P4: forces are the gradient of the stored energy (brute-force FD)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,aniso", [("h8", False), ("t4", False), ("h8", True), ("t4", True)])
def test_p4_force_is_energy_gradient(kind, aniso):
    """Forces are the gradient of the stored energy V0 det(F_th) Psi(F F_th^-1)
    (+ hourglass), thermal loads the gradient of the conduction quadratic form;
    also with transversely isotropic expansion and conductivity (R26)."""
    rng = np.random.default_rng(11)
    if kind == "h8":
        X, conn = W.hex_grid((2, 1, 1), (0.02, 0.01, 0.01), jitter=0.15, rng=rng)
        npe = 8
    else:
        X, conn = W.kuhn_tets((1, 1, 1), (0.01, 0.01, 0.01))
        X = X + rng.uniform(-0.1, 0.1, X.shape) * 0.01
        conn = W._orient_tets(X, conn)
        npe = 4
    ne = conn.shape[0]
    fib = W.vmf_directions(ne, 2.0, (1, 1, 0), rng)
    mat = W._material(ne, rng, noise=0.2, fibre=fib, alpha=2e-3)
    p = W.Problem(name="fd", npe=npe, X=X, conn=conn, **mat, prony_g=(), prony_tau=(), kappa_hg=0.3)
    if aniso:
        p.aniso_alpha, p.aniso_k = 3.0, 2.5
    p.dt = 1e-4
    m = oracle.OracleModel(p)
    u = rng.uniform(-1, 1, (p.nn, 3)) * 0.001
    T = 37.0 + rng.uniform(0, 20, p.nn)
    eps = 1e-8
    for e in range(ne):
        fe, fTe, _, detF = m.element(e, u, T)
        assert detF > 0.5
        cn = conn[e]
        num = np.zeros((npe, 3))
        for a in range(npe):
            for i in range(3):
                up, um = u.copy(), u.copy()
                up[cn[a], i] += eps
                um[cn[a], i] -= eps
                num[a, i] = (m.energy(e, up, T) - m.energy(e, um, T)) / (2 * eps)
        np.testing.assert_allclose(fe, num, rtol=2e-5, atol=1e-7 * np.abs(num).max())
        # thermal load = gradient of the conduction quadratic form at fixed k
        Tk = T[cn].mean()
        numT = np.zeros(npe)
        for a in range(npe):
            Tp, Tm = T.copy(), T.copy()
            Tp[cn[a]] += 1e-3
            Tm[cn[a]] -= 1e-3
            numT[a] = (m.thermal_energy(e, u, Tp, Tk) - m.thermal_energy(e, u, Tm, Tk)) / 2e-3
        np.testing.assert_allclose(fTe, numT, rtol=1e-7, atol=1e-9 * np.abs(numT).max())


# ---------------------------------------------------------------------------
# P5: frame invariance
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,aniso", [("h8", False), ("t4", False), ("h8", True), ("t4", True)])
def test_p5_rigid_rotation(kind, aniso):
    """A rigid rotation of a deformed configuration rotates the internal forces
    and leaves the thermal loads unchanged; with anisotropic conductivity this
    holds only because the conductivity follows the current fibre F a0."""
    p = W.cube_h8(n=2, jitter=0.2) if kind == "h8" else W.cube_t4(n=2)
    if aniso:
        p.aniso_alpha, p.aniso_k = 3.0, 4.0
    p.mask[:] = 0
    p.dt = 1e-6
    rng = np.random.default_rng(5)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    Q = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    m = oracle.OracleModel(p)
    T = 37.0 + rng.uniform(0, 10, p.nn)
    u0 = rng.uniform(-1, 1, (p.nn, 3)) * 1e-3  # a deformed configuration phi(X) = X + u0
    ur = (p.X + u0) @ Q.T - p.X + 0.01     # the same, rigidly rotated and translated
    for e in range(p.ne):
        f0, fT0, _, _ = m.element(e, u0, T)
        fr, fTr, _, _ = m.element(e, ur, T)
        # internal forces rotate with the body; thermal loads are unchanged (C = I)
        np.testing.assert_allclose(fr, f0 @ Q.T, atol=1e-9 * (1 + np.abs(f0).max()))
        np.testing.assert_allclose(fTr, fT0, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# P6: assembly invariants and the adiabatic heat balance
# ---------------------------------------------------------------------------
def test_p6_element_sums_and_heat_balance():
    p = W.cube_t4(n=3)
    p.dt = 1e-4
    m = oracle.OracleModel(p)
    st = W.random_state(p, 3, u_scale=1e-3)
    s = m.state_from(**st)
    for e in range(0, p.ne, 7):
        fe, fTe, _, _ = m.element(e, s.u, s.T, s.visc[e])
        assert np.abs(fe.sum(0)).max() < 1e-10 * np.abs(fe).max()
        assert abs(fTe.sum()) < 1e-10 * np.abs(fTe).max()
    T_old = s.T.copy()
    fixedT = (p.mask & W.MASK_T) != 0
    m.step(s, 1)
    heat = (m.Cth * (s.T - T_old)).sum()
    Qr = np.zeros(p.nn)
    for src in p.sources:
        c = src[:3] + src[3:6] * 0.0
        r2 = ((p.X + st["u"] - c) ** 2).sum(1)
        Qr += src[7] * np.exp(-r2 / (2 * src[6] ** 2))
    expect = p.dt * (m.Vn * (-p.wbcb * (T_old - p.Ta) + p.Qm + Qr))[~fixedT].sum()
    np.testing.assert_allclose(heat, expect, rtol=1e-9)


def test_lumped_mass_conserves_mass_and_volume():
    for p in (W.cube_h8(n=4), W.cube_t4(n=3)):
        m = oracle.OracleModel(p)
        vol = 0.05 ** 3
        np.testing.assert_allclose(m.V0.sum(), vol, rtol=1e-12)
        np.testing.assert_allclose(m.Vn.sum(), vol, rtol=1e-12)
        np.testing.assert_allclose(m.M.sum(), 1000.0 * vol, rtol=1e-12)
        np.testing.assert_allclose(m.Cth.sum(), 1000.0 * p.c_heat * vol, rtol=1e-12)


# ---------------------------------------------------------------------------
# P7: Prony recurrence, exact discrete relaxation
# ---------------------------------------------------------------------------
def test_p7_prony_relaxation_under_held_strain():
    """Held strain: S~_n = S (1 - phi (1 - b^(n+1))), b = tau / (dt + tau); long
    time limit (1 - phi) S (relaxation function of the generalised Maxwell model)."""
    n, Ls = 2, 0.02
    X, conn = W.hex_grid((n, n, n), (Ls, Ls, Ls))
    mat = W._material(conn.shape[0])
    ubar = np.stack([0.1 * X[:, 0], -0.03 * X[:, 1], 0.02 * X[:, 2]], 1)
    common = dict(name="prony", npe=8, X=X, conn=conn, **mat,
                  mask=np.full(X.shape[0], W.MASK_U, np.uint8), ubar=ubar, dt=0.01)
    pe = W.Problem(**common, prony_g=(), prony_tau=())
    pv = W.Problem(**common, prony_g=(0.5,), prony_tau=(0.3,))
    me, mv = oracle.OracleModel(pe), oracle.OracleModel(pv)
    se, sv = me.init_state(), mv.init_state()
    for s in (se, sv):
        s.u[:] = ubar
        s.u_prev[:] = ubar
    me.step(se, 1)
    fe, _ = me.forces()
    b = 0.3 / (0.01 + 0.3)
    for k in range(700):
        mv.step(sv, 1)
        fv, _ = mv.forces()
        np.testing.assert_allclose(fv, fe * (1 - 0.5 * (1 - b ** (k + 1))), rtol=1e-10,
                                   atol=1e-12 * np.abs(fe).max())
    np.testing.assert_allclose(fv, 0.5 * fe, rtol=1e-6, atol=1e-9 * np.abs(fe).max())


# ---------------------------------------------------------------------------
# P8: central difference with mass-proportional damping
# ---------------------------------------------------------------------------
def test_p8_rigid_translation_with_damping():
    """Force-free rigid translation: v_(n+1/2) = r v_(n-1/2) with
    r = (1 - gamma dt/2)/(1 + gamma dt/2), so u_n = u_0 + dt v0 r (1 - r^n)/(1 - r)."""
    p = W.cube_t4(n=2)
    p.mask[:] = 0
    p.gamma = 70.0
    p.dt = 1e-4  # below the stable step, so rounding noise cannot grow
    p.sources = np.zeros((0, 10))
    m = oracle.OracleModel(p)
    s = m.init_state()
    v0 = np.array([0.3, -0.2, 0.1])
    s.u[:] = 0.001
    s.u_prev[:] = 0.001 - p.dt * v0
    m.step(s, 200)
    r = (1 - p.gamma * p.dt / 2) / (1 + p.gamma * p.dt / 2)
    expect = 0.001 + p.dt * v0 * r * (1 - r ** 200) / (1 - r)
    np.testing.assert_allclose(s.u, np.broadcast_to(expect, s.u.shape), rtol=1e-10)



# ---------------------------------------------------------------------------
# P9: energy balance of the central-difference scheme
# ---------------------------------------------------------------------------
def test_p9_energy_balance_is_second_order():
    """With no damping, no Prony terms, no thermal load and a fixed face, the
    mechanical energy of the explicit scheme only oscillates, and the
    oscillation shrinks like dt^2 (central difference is second order and
    symplectic); it does not drift.  Stored energy and kinetic energy are
    independent code paths (element potential vs nodal masses), so a wrong
    force (sign, factor, missing term) or a wrong mass breaks this balance."""
    p = p9_problem()
    u0 = p9_initial(p)
    m1 = oracle.OracleModel(p)
    dt = m1.dt
    E1 = p9_energy_history(m1, p, u0, 30, 50)
    m2 = oracle.OracleModel(p, dt=dt / 2)
    E2 = p9_energy_history(m2, p, u0, 30, 100)
    f1 = np.ptp(E1) / E1[0]
    f2 = np.ptp(E2) / E2[0]
    assert f1 < 1e-2, f1
    assert 3.0 < f1 / f2 < 5.0, (f1, f2)
    # the energy did move between kinetic and stored (the test is not vacuous)
    v = m1.state_from(u0, np.zeros_like(u0), np.full(p.nn, p.T0), np.zeros(p.nn), None)
    m1.step(v, 200)
    k = 0.5 * np.sum(m1.M[:, None] * ((v.u - v.u_prev) / m1.dt) ** 2)
    assert k > 0.05 * E1[0], (k, E1[0])


# ---------------------------------------------------------------------------
# the paper's own source and dose read-out (uniform spheres, CEM43)
# ---------------------------------------------------------------------------
def test_uniform_sphere_source_heat_balance():
    """One step from rest with a uniform spherical source (the paper's liver
    case) and no perfusion or metabolic heat: the element conduction loads sum
    to zero, so the heat content rises by exactly dt * P * (sum of the lumped
    volumes of the nodes inside the sphere), counted here independently."""
    p = W.cube_h8(n=6, jitter=0.1, seed=71)
    p.wbcb, p.Qm, p.expansion = 0.0, 0.0, False
    c, r, P = np.array([0.021, 0.024, 0.027]), 0.011, 7e6
    p.sources = np.array([W.source(c, P, sigma=r, sphere=True)])
    d = np.linalg.norm(p.X - c, axis=1)
    assert np.min(np.abs(d - r)) > 1e-6  # membership is unambiguous
    inside = d <= r
    assert 0 < inside.sum() < p.nn
    m = oracle.OracleModel(p)
    s = m.init_state()
    m.step(s, 1)
    dQ = np.sum(m.Cth * (s.T - p.T0))
    np.testing.assert_allclose(dQ, m.dt * P * m.Vn[inside].sum(), rtol=1e-12)


def test_cem43_at_held_temperatures():
    """CEM43 at temperatures held fixed: t/60 * R^(43 - T) minutes exactly, with
    R = 0.5 at or above 43 C (45 C: 4 t/60) and 0.25 below (40 C: t/60 / 64)."""
    p = W.cube_h8(n=2)
    p.sources = np.zeros((0, 11))
    p.mask = p.mask | W.MASK_T  # every temperature held
    m = oracle.OracleModel(p, dt=0.01)
    s = m.init_state()
    T = np.full(p.nn, 40.0)
    T[:9] = 45.0
    T[9:18] = 43.0
    s.T[:] = T
    m.step(s, 300)
    t = 300 * 0.01
    np.testing.assert_allclose(s.T, T)
    np.testing.assert_allclose(s.cem[:9], 4.0 * t / 60.0, rtol=1e-13)
    np.testing.assert_allclose(s.cem[9:18], t / 60.0, rtol=1e-13)
    np.testing.assert_allclose(s.cem[18:], t / 60.0 / 64.0, rtol=1e-13)

# ---------------------------------------------------------------------------
# P10: Arrhenius integral
# ---------------------------------------------------------------------------
def test_p10_arrhenius_constant_temperature_and_paper_claim():
    """At constant T the explicit integral is exactly linear in the step count,
    and with the liver constants tissue at 60 C is necrotised within seconds
    while 37 C tissue is essentially undamaged (the paper's remark on CEM43 and
    the Arrhenius integral)."""
    p = W.cube_h8(n=1)
    p.expansion = False
    p.sources = np.zeros((0, 10))
    p.wbcb = 0.0
    p.dt = 0.01
    m = oracle.OracleModel(p)
    for Tc, lo, hi in ((60.0, 1.0, np.inf), (37.0, 0.0, 0.01)):
        s = m.init_state()
        s.T[:] = Tc
        m.step(s, 1)
        one = s.Omega.copy()
        m.step(s, 999)
        np.testing.assert_allclose(s.Omega, 1000 * one, rtol=1e-12)
        d = oracle.damage_fraction(s.Omega)  # after 10 s
        assert lo <= s.Omega.min() and s.Omega.max() <= hi, (Tc, s.Omega.max())
        if Tc == 60.0:
            assert d.min() > 0.63


# ---------------------------------------------------------------------------
# P11: hourglass shape vectors are orthogonal to linear fields
# ---------------------------------------------------------------------------
def test_p11_hourglass_orthogonality():
    p = W.cube_h8(n=3, jitter=0.25)
    m = oracle.OracleModel(p)
    G = m.hg_gamma  # (ne, 8, 4)
    Xe = p.X[p.conn]  # (ne, 8, 3)
    assert np.abs(G.sum(1)).max() < 1e-12
    assert np.abs(np.einsum("eak,eaj->ekj", G, Xe)).max() < 1e-14
    # and they are not trivially zero
    assert np.abs(G).max() > 0.5


# ---------------------------------------------------------------------------
# critical time step on a uniform cube (R16): L = h, c_d from the moduli
# ---------------------------------------------------------------------------
def test_stable_dt_uniform_cube():
    p = W.cube_h8(n=8)
    m = oracle.OracleModel(p)
    h = 0.05 / 8
    cd = np.sqrt((3e5 + 4 * 3e3 / 3 + 4 * 1e3) / 1000.0)
    np.testing.assert_allclose(m.dt_mech, h / cd, rtol=1e-12)
    np.testing.assert_allclose(m.dt, 0.8 * h / cd, rtol=1e-12)
    assert m.dt_th > 100 * m.dt_mech


# ---------------------------------------------------------------------------
# P6 continued: a moving Gaussian source at t > 0 (R14: c(t) = c0 + v t)
# ---------------------------------------------------------------------------
def test_p6_moving_source_heat_balance_at_later_time():
    """One step from a mid-run state at t1 > 0 with a moving source (and one
    already switched off): the heat content rises by dt sum_i V_i (Q_r(x_i, t1)
    - perfusion), with Q_r centred at c0 + v t1 and x_i = X_i + u_i; the element
    conduction loads sum to zero.  Centring the source at c0 - v t1 or at c0
    would miss by far more than the tolerance (checked)."""
    p = W.cube_h8(n=6, jitter=0.1, seed=11)
    c0, v, sig, P = np.array([0.012, 0.02, 0.03]), np.array([0.02, 0.01, -0.015]), 4e-3, 6e6
    p.sources = np.array([W.source(c0, P, sigma=sig, vel=v),
                          W.source((0.025, 0.025, 0.025), 9e6, sigma=sig, t_on=0.0, t_off=0.3)])
    p.dt = 1e-4
    m = oracle.OracleModel(p)
    st = W.random_state(p, 4, u_scale=1e-3)
    t1 = 0.6
    s = m.state_from(**st, t=t1, step=6000)
    T_old = s.T.copy()
    m.step(s, 1)
    heat = (m.Cth * (s.T - T_old)).sum()
    fixedT = (p.mask & W.MASK_T) != 0
    x = p.X + st["u"]

    def expected(centre):
        Qr = P * np.exp(-((x - centre) ** 2).sum(1) / (2 * sig * sig))
        return p.dt * (m.Vn * (-p.wbcb * (T_old - p.Ta) + p.Qm + Qr))[~fixedT].sum()

    np.testing.assert_allclose(heat, expected(c0 + v * t1), rtol=1e-9)
    for wrong in (c0 - v * t1, c0, c0 + v * (t1 + p.dt)):
        assert abs(expected(wrong) - heat) > 1e-6 * abs(heat), wrong
    assert s.t == pytest.approx(t1 + p.dt, abs=0, rel=1e-15)


# ---------------------------------------------------------------------------
# P3 continued: prescribed displacement ramp, applied at t_{n+1} (R19)
# ---------------------------------------------------------------------------
def test_p3_prescribed_displacement_ramp_mid_ramp():
    """u_bar ramps linearly over ramp_time; after step n the prescribed
    components hold (n dt / ramp_time) u_bar exactly (u_{n+1} at t_{n+1}), and
    u_bar itself once the ramp is over.  A ramp evaluated at t_n, or a wrong
    slope, fails at the first step."""
    p = W.cube_h8(n=3)
    p.sources = np.zeros((0, 10))
    top = np.isclose(p.X[:, 2], 0.05)
    p.mask[top] = W.MASK_U
    p.ubar = np.zeros((p.nn, 3))
    p.ubar[top, 2] = 4e-3
    p.ubar[top, 0] = -1e-3
    p.dt = 1e-4
    p.ramp_time = 10 * p.dt
    m = oracle.OracleModel(p)
    s = m.init_state()
    held = p.mask.astype(bool)
    for n in range(1, 15):
        m.step(s, 1)
        frac = min(1.0, n * p.dt / p.ramp_time)
        np.testing.assert_allclose(s.u[top], frac * p.ubar[top], rtol=1e-14, atol=0)
        np.testing.assert_array_equal(s.u[held & ~top], 0.0)
    # the free nodes have moved (the ramp drives the body)
    assert np.abs(s.u[~held]).max() > 1e-6


# ---------------------------------------------------------------------------
# R16 thermal Gershgorin bound on a uniform cube, in closed form
# ---------------------------------------------------------------------------
def _uniform_cube_row_sum(kappa_t, r_k):
    """Sum over b of |K_ab| of one cube element of side h, in units of h k / 16,
    for conduction along a0 = x scaled by r_k and the thermal hourglass of
    coefficient kappa_t.  Corner a = (sx, sy, sz) in {-1, 1}^3: grad h_a =
    s_a / (4 h), V = h^3, so V grad h_a . D grad h_b = (h k / 16)(p + q + r +
    (r_k - 1) p) with p = sx_a sx_b etc.; the hourglass vectors of a brick are
    the base vectors h_alpha (their projections vanish), BB = 3 / (2 h^2), so
    k_hgT = kappa_t V BB / 8 = 3 kappa_t h / 16 and K^hg_ab = k k_hgT (pq + qr +
    pr + pqr)."""
    a = (1, 1, 1)
    total = 0.0
    for b in [(x, y, z) for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)]:
        p, q, r = a[0] * b[0], a[1] * b[1], a[2] * b[2]
        total += abs(p + q + r + (r_k - 1) * p + 3 * kappa_t * (p * q + q * r + p * r + p * q * r))
    return total


@pytest.mark.parametrize("kappa_t,r_k,expect_R", [(0.1, 1.0, 10.8), (0.0, 1.0, 12.0), (0.1, 2.5, None)])
def test_stable_dt_thermal_gershgorin_closed_form(kappa_t, r_k, expect_R):
    """R16's thermal bound dt_th = min_i 2 C_i / (sum_j |K_ij| + w_b c_b V_i) on a
    uniform n^3 cube: every node, interior or boundary, gets
    2 rho c h^3 / (8 (h k / 16) R + w_b c_b h^3) with R the element's absolute
    row sum worked out by hand (10.8 for the default hourglass coefficient 0.1:
    4.2 + 3 x 0.4 + 3 x 1 + 2.4)."""
    n, side = 4, 0.05
    h = side / n
    p = W.cube_h8(n=n)
    p.kappa_hgT = kappa_t
    p.aniso_k = r_k
    p.a0 = np.tile([1.0, 0.0, 0.0], (p.ne, 1))
    m = oracle.OracleModel(p)
    R = _uniform_cube_row_sum(kappa_t, r_k)
    if expect_R is not None:
        assert R == pytest.approx(expect_R, rel=1e-14)
    rho, c, k = 1000.0, p.c_heat, 0.5
    dt_th = 2 * rho * c * h ** 3 / (8 * h * k / 16 * R + p.wbcb * h ** 3)
    np.testing.assert_allclose(m.dt_th, dt_th, rtol=1e-12)


# ---------------------------------------------------------------------------
# P10 continued: the Arrhenius integral's exact value with R18's constants
# ---------------------------------------------------------------------------
def test_p10_arrhenius_exact_value():
    """At a held temperature Omega(t) = t A exp(-E_a / (R (T + 273.15))) with
    A = 7.39e39 1/s, E_a = 2.577e5 J/mol, R = 8.314 J/(mol K) (R18); the rates at
    37, 60 and 90 C are about 2.92e-4, 0.290 and 631 1/s."""
    p = W.cube_h8(n=1)
    p.sources = np.zeros((0, 10))
    p.mask = p.mask | W.MASK_T  # hold every temperature
    m = oracle.OracleModel(p, dt=0.01)
    A, Ea, R = 7.39e39, 2.577e5, 8.314
    for Tc, rate in ((37.0, 2.92e-4), (60.0, 0.290), (90.0, 631.0)):
        s = m.init_state()
        s.T[:] = Tc
        m.step(s, 250)
        k = A * np.exp(-Ea / (R * (Tc + 273.15)))
        np.testing.assert_allclose(s.Omega, 250 * 0.01 * k, rtol=1e-12)
        assert k == pytest.approx(rate, rel=3e-3)


# ---------------------------------------------------------------------------
# probes: shape-function interpolation at arbitrary points
# ---------------------------------------------------------------------------
def _probe_points(p, k, seed):
    rng = np.random.default_rng(seed)
    lo, hi = p.X.min(0), p.X.max(0)
    return lo + (hi - lo) * rng.uniform(0.12, 0.88, (k, 3))


@pytest.mark.parametrize("kind", ["h8_jittered", "t4"])
def test_probe_reproduces_linear_fields(kind):
    """Linear fields are interpolated exactly by T4 barycentric and by
    isoparametric H8 shape functions, on distorted elements too, provided the
    point is located correctly (x(xi) = x): T = a + b . x and a damage fraction
    linear in x come back exactly at arbitrary (off-centroid) points."""
    p = W.cube_h8(n=5, jitter=0.25, seed=4) if kind == "h8_jittered" else W.cube_t4(n=4, jitter=0.15)
    m = oracle.OracleModel(p)
    s = m.init_state()
    b, g = np.array([300.0, -200.0, 150.0]), np.array([4.0, 2.0, -3.0])
    s.T[:] = 40.0 + p.X @ b
    d_nodes = 0.4 + p.X @ g
    s.Omega[:] = -np.log1p(-d_nodes)
    x = _probe_points(p, 300, 3)
    T, d = m.probe(s, x)
    np.testing.assert_allclose(T, 40.0 + x @ b, rtol=0, atol=1e-11)
    np.testing.assert_allclose(d, 0.4 + x @ g, rtol=0, atol=1e-12)


def test_probe_trilinear_on_bricks_and_nodes():
    """On axis-aligned bricks the trilinear shape functions reproduce x y z
    exactly (x, y, z are affine in the natural coordinates), which pins the
    H8 interpolation itself, not only partition of unity; a probe on a node
    returns that node's value (any field)."""
    X, conn = W.hex_grid((3, 4, 2), (0.03, 0.05, 0.02))
    mat = W._material(conn.shape[0])
    p = W.Problem(name="bricks", npe=8, X=X, conn=conn, **mat)
    m = oracle.OracleModel(p)
    s = m.init_state()
    s.T[:] = 1e5 * X[:, 0] * X[:, 1] * X[:, 2]
    x = _probe_points(p, 200, 8)
    T, _ = m.probe(s, x)
    np.testing.assert_allclose(T, 1e5 * x[:, 0] * x[:, 1] * x[:, 2], rtol=1e-12, atol=1e-15)
    rng = np.random.default_rng(1)
    s.T[:] = 37 + rng.uniform(0, 20, p.nn)
    s.Omega[:] = rng.uniform(0, 3, p.nn)
    T, d = m.probe(s, X[::5])
    np.testing.assert_allclose(T, s.T[::5], rtol=1e-13)
    np.testing.assert_allclose(d, oracle.damage_fraction(s.Omega[::5]), rtol=1e-13)
    with pytest.raises(ValueError, match="outside"):
        m.probe(s, [[0.5, 0.5, 0.5]])


# ---------------------------------------------------------------------------
# the oracle on all host cores is the same computation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["h8", "t4"])
def test_parallel_oracle_is_bitwise_serial(kind):
    """ora_step_parallel (elements in parallel, fixed-order node gather) gives
    bitwise the state of the plain element-order ora_step."""
    p = W.cube_h8(n=6, jitter=0.2, seed=9) if kind == "h8" else W.cube_t4(n=4)
    p.sources = np.array([W.source((0.02, 0.025, 0.03), 8e6, sigma=6e-3, vel=(0.01, 0, 0))])
    m = oracle.OracleModel(p)
    st = W.random_state(p, 2, u_scale=1e-3)
    a, b = m.state_from(**st), m.state_from(**st)
    m.step(a, 30)
    m.step_parallel(b, 30)
    for f in ("u", "u_prev", "T", "Omega", "visc", "cem"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    assert a.t == b.t and a.step == b.step


# ---------------------------------------------------------------------------
# R17 mass scaling from the oracle's own CFL bound
# ---------------------------------------------------------------------------
def test_mass_scale_for_fixed_step():
    """s_m = (dt / (0.8 dt_mech))^2 with dt_mech = h / c_d, c_d = sqrt((kappa +
    4 mu / 3 + 4 k1) / rho) on a uniform cube; with that scale the safe
    mechanical step is dt itself."""
    p = W.cube_h8(n=8)
    h, dt = 0.05 / 8, 0.01
    cd = np.sqrt((3e5 + 4 * 3e3 / 3 + 4 * 1e3) / 1000.0)
    s_m = oracle.mass_scale_for(p, dt)
    np.testing.assert_allclose(s_m, (dt * cd / (0.8 * h)) ** 2, rtol=1e-12)
    p.mass_scale = s_m
    m = oracle.OracleModel(p, dt=dt)
    m.stable_dt(0.8)
    np.testing.assert_allclose(0.8 * m.dt_mech, dt, rtol=1e-12)


# ---------------------------------------------------------------------------
# mechanical subcycling (study f4): reductions to the plain step
# ---------------------------------------------------------------------------
def test_subcycling_with_one_substep_is_the_plain_step():
    p = W.cube_h8(n=4, jitter=0.2, seed=12)
    p.sources = np.array([W.source((0.02, 0.025, 0.03), 8e6, sigma=6e-3, vel=(0.01, 0, 0))])
    m = oracle.OracleModel(p)
    st = W.random_state(p, 5, u_scale=1e-3)
    a, b = m.state_from(**st), m.state_from(**st)
    m.step(a, 25)
    m.step_thermal(b, 25)
    for f in ("u", "u_prev", "T", "Omega", "visc", "cem"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)


def test_subcycling_thermal_part_is_the_plain_thermal_step():
    """Displacements held at zero (every component prescribed, no expansion): the
    subcycled temperature, damage and dose after N thermal steps are exactly
    those of N plain steps of the thermal step (the substeps change nothing the
    heat equation sees, and T advances once per thermal step, explicitly)."""
    p = W.cube_h8(n=4, jitter=0.2, seed=13)
    p.mask[:] = W.MASK_U
    p.expansion = False
    p.sources = np.array([W.source((0.02, 0.025, 0.03), 8e6, sigma=6e-3, vel=(0.01, -0.02, 0))])
    p.dt, p.n_sub = 2e-3, 7
    sub = oracle.OracleModel(p)
    p1 = W.cube_h8(n=4, jitter=0.2, seed=13)
    p1.mask[:] = W.MASK_U
    p1.expansion = False
    p1.sources = p.sources
    p1.dt = 2e-3
    plain = oracle.OracleModel(p1)
    a, b = sub.init_state(), plain.init_state()
    a.T[:] = b.T[:] = 37.0 + np.linspace(0, 8, p.nn)
    sub.step_thermal(a, 30)
    plain.step(b, 30)
    for f in ("T", "Omega", "cem"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    np.testing.assert_array_equal(a.u, 0.0)
    assert a.step == 30 * 7 and a.t == pytest.approx(30 * 2e-3, rel=1e-12)
    assert a.T.max() > 37.5


def test_subcycling_mechanical_part_is_the_plain_substep():
    """No heat (no sources or perfusion, uniform T = T0): N thermal steps of n_sub
    substeps move the body exactly as N n_sub plain steps of the substep
    (Prony recurrence, damping and Eq. 27 over the substep; the prescribed
    displacement ramp at each substep's end)."""
    def problem(**kw):
        p = W.cube_h8(n=3, jitter=0.15, seed=14)
        p.sources = np.zeros((0, 11))
        p.wbcb, p.gamma = 0.0, 3.0
        top = p.X[:, 2] > 0.042  # the top layer of nodes (jittered around z = 5 cm)
        p.mask[top] = W.MASK_U
        p.ubar = np.zeros((p.nn, 3))
        p.ubar[top, 2] = 2e-3
        p.ramp_time = 0.02
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    n_sub, dts = 5, 2.5e-3
    sub = oracle.OracleModel(problem(dt=dts, n_sub=n_sub))
    plain = oracle.OracleModel(problem(dt=dts / n_sub))
    a, b = sub.init_state(), plain.init_state()
    sub.step_thermal(a, 12)
    plain.step(b, 12 * n_sub)
    for f in ("u", "u_prev", "visc"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    assert a.t == b.t
    assert np.abs(a.u).max() > 1e-3  # the ramp has moved the top face and the body follows
