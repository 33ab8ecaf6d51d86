"""Shared helpers of the test-suite: run the oracle and the CUDA library on the
same seeded problem and compare with the paper's error metrics."""
import numpy as np

from paper_2009_10400_b300 import workloads as W

import oracle


def rel_l2(a, b):
    """Total error indicator e = ||a - b||_2 / ||b||_2 (Section 6.1)."""
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def nre_max(a, b):
    """Max normalised relative error |a - b| / (max b - min b) (Section 6.1)."""
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    rng = b.max() - b.min()
    return np.abs(a - b).max() / rng if rng > 0 else np.abs(a - b).max()


def run_oracle(prob, n_steps, every=None, dt=None):
    m = oracle.OracleModel(prob, dt=dt)
    s = m.init_state()
    snaps = []
    every = every or n_steps
    done = 0
    while done < n_steps:
        k = min(every, n_steps - done)
        m.step(s, k)
        done += k
        snaps.append((done, s.u.copy(), s.T.copy(), s.Omega.copy()))
    return m, s, snaps


def compare(u, T, d, u_ref, T_ref, Om_ref, T0=37.0):
    return dict(e_u=rel_l2(u, u_ref), e_theta=rel_l2(T - T0, T_ref - T0),
                d_abs=float(np.abs(d - oracle.damage_fraction(Om_ref)).max()),
                nre_u=nre_max(u, u_ref), nre_T=nre_max(T, T_ref))


# tolerances stated by the task for FP32 results against the FP64 oracle
TOL_E = 1e-4        # relative L2 of displacement and of temperature rise
TOL_DAMAGE = 1e-3   # absolute damage fraction


# P9 energy balance (shared by the oracle pin and the GPU test)
def p9_problem():
    """P9 set-up: 4^3 jittered H8 cube, no Prony terms, no expansion, no
    sources, no damping, bottom face fixed."""
    p = W.cube_h8(n=4, jitter=0.1, seed=5)
    p.prony_g, p.prony_tau = (), ()  # phi = 0
    p.expansion = False
    p.sources = np.zeros((0, 10))
    p.gamma = 0.0
    return p


def p9_initial(p):
    """A smooth bending/shear field with the bottom face fixed, at rest."""
    X, L = p.X, 0.05
    u0 = np.zeros_like(X)
    u0[:, 0] = 2e-3 * np.sin(np.pi * X[:, 2] / (2 * L))
    u0[:, 1] = 1e-3 * np.sin(np.pi * X[:, 2] / (2 * L)) * X[:, 0] / L
    u0[p.mask.astype(bool)] = 0.0
    return u0


def p9_energy_history(m, p, u0, n_samples, every):
    """Mechanical energy E_n = (K_{n-1/2} + K_{n+1/2})/2 + sum_e W_e(u_n) at every
    `every`-th step: kinetic energy of the two half-step velocities around u_n
    (Eq. 27 in velocity form) plus the stored energy of the elements."""
    s = m.state_from(u0, np.zeros_like(u0), np.full(p.nn, p.T0), np.zeros(p.nn), None)

    def kin(s):
        v = (s.u - s.u_prev) / m.dt
        return 0.5 * np.sum(m.M[:, None] * v * v)

    E = []
    for _ in range(n_samples):
        k0 = kin(s)
        w = sum(m.energy(e, s.u, s.T) for e in range(p.ne))
        m.step(s, 1)
        E.append(0.5 * (k0 + kin(s)) + w)
        m.step(s, every - 1)
    return np.array(E)
