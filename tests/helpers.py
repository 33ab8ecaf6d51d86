"""Shared helpers of the test-suite: run the oracle and the CUDA library on the
same seeded problem and compare with the paper's error metrics."""
import numpy as np

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
