"""Learned surrogate for treatment planning: scenario parameters -> temperature
and damage at probe points after heating, trained on data from the batched
coupled solver, with an ensemble spread test that sends uncertain cases back
to the solver.

The ensemble is the library's surrogate engine (``tled_sur``, include/tled_mlp.h):
the target transform and standardisation, the seeded initialisation and row
permutations, graph-replayed training on the tensor-core kernels, inference,
the ensemble statistics with the fallback decision and the calibration of the
spread threshold all run in the library; the data and the fallback answers come
from ``tled.Batch``.  This module only sequences those calls and moves arrays.
"""
from __future__ import annotations

import time

import numpy as np

from . import tled
from . import workloads as W
from .mlp import SurrogateEngine, spread_threshold  # noqa: F401 (re-exported)


def solve_scenarios(Q, n=16, dt=0.01, chunk=512, device=0):
    """Run every scenario row of Q (see workloads.SURROGATE_INPUTS) to the end of
    its heating time with the batched solver; returns temperature and damage
    at the n^3 element-centroid probes, shape (len(Q), n^3) each, and timing."""
    Q = np.atleast_2d(Q)
    P = n ** 3
    T = np.empty((len(Q), P))
    D = np.empty((len(Q), P))
    steps = 0
    t0 = time.perf_counter()
    for s0 in range(0, len(Q), chunk):
        part = Q[s0:s0 + chunk]
        b = tled.Batch(device=device)
        for q in part:
            prob = W.scenario_problem(q, n=n, dt=dt)  # mass scaled by the library (R17)
            b.add(prob, prob.n_steps, probes=W.centroids(prob))
        b.init()
        steps += b.run()
        out = b.probes()
        b.sync()
        for i in range(len(part)):
            info = b.scenario(i)
            sl = slice(info["probe_off"], info["probe_off"] + info["probes"])
            T[s0 + i] = out[0, sl]
            D[s0 + i] = out[1, sl]
        b.close()
    return T, D, dict(seconds=time.perf_counter() - t0, launch_steps=steps)


def cube_symmetries(n=16, side=0.05, n_in=12):
    """The 16 reflections of the scenario cube that leave its heating problem
    unchanged -- x, y, z mirrored and x <-> y swapped (the faces are adiabatic
    and the source is a Gaussian; the one mechanical boundary, the held bottom,
    moves nodes by ~1e-5 of an element, so temperatures follow the reflection)
    -- as the surrogate engine's tables: the source position mapped (inputs 1-3),
    the other inputs unchanged, and the n^3 element-centroid probes (x fastest;
    temperatures then damage) permuted with the reflection.  Returns (src, a, b,
    perm) with [16][n_in] and [16][2 n^3] entries."""
    import itertools

    ijk = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    ijk = ijk[:, ::-1]  # rows in x-fastest probe order: (i, j, k) of probe i + n (j + n k)
    src, a, b, perm = [], [], [], []
    for fx, fy, fz, sw in itertools.product((0, 1), repeat=4):
        s_ = np.arange(n_in)
        a_ = np.ones(n_in)
        b_ = np.zeros(n_in)
        for col, f in ((1, fx), (2, fy), (3, fz)):
            if f:
                a_[col], b_[col] = -1.0, side
        if sw:  # x' and y' read the (mirrored) y and x
            s_[1], s_[2] = 2, 1
            a_[1], a_[2] = a_[2], a_[1]
            b_[1], b_[2] = b_[2], b_[1]
        # the map is g = (swap) after (mirrors); the mapped scenario's field is T'(x) = T(g^-1 x),
        # so probe p of the mapped row reads probe g^-1(p) = (mirrors) after (swap) of the data row
        q = ijk.copy()
        if sw: q[:, [0, 1]] = q[:, [1, 0]]
        if fx: q[:, 0] = n - 1 - q[:, 0]
        if fy: q[:, 1] = n - 1 - q[:, 1]
        if fz: q[:, 2] = n - 1 - q[:, 2]
        p = q[:, 0] + n * (q[:, 1] + n * q[:, 2])
        src.append(s_)
        a.append(a_)
        b.append(b_)
        perm.append(np.concatenate([p, n ** 3 + p]))
    return np.array(src), np.array(a), np.array(b), np.array(perm)


P_REF = 5e6  # W/m^3: the temperature outputs are learned per unit of power / P_REF
T_REF = 37.0  # C: initial and arterial temperature of the scenarios


class Surrogate:
    """Ensemble of MLPs [features, width x (depth - 1), n_out] (the library's
    surrogate engine).  The 12 inputs are mapped to [-1, 1] over the sampling
    ranges; the source position also enters as sin / cos features at n_freq
    octaves (the answer is a peak that moves with the source).  The first
    n_T outputs are temperatures; with `per_power` the networks learn the
    temperature rise per unit source power, (T - T_REF) / (P / P_REF) -- the
    bioheat part of the model is linear in the source power (c and k
    temperature independent; the source centre moves with displacements of
    ~1e-5 m) -- and the answers are scaled back by each scenario's power.
    Targets are standardised per output (norm 0) or with one scale per output
    group (norm 1: temperatures, damage), so that the loss weighs physical
    errors alike."""

    def __init__(self, n_out, width=512, depth=6, members=5, max_batch=4096, device=0, n_in=12, n_T=None,
                 per_power=True, norm=1, max_rows=20480, max_epochs=64, n_freq=0, symmetric=False, grid=16):
        self.n_T = n_out // 2 if n_T is None else n_T
        self.n_members = members
        self.max_batch = max_batch
        self.device = device
        # optional sin / cos features of the source position (inputs 1-3) at n_freq octaves
        self.engine = SurrogateEngine([n_in] + [width] * (depth - 1) + [n_out], members, self.n_T, max_batch,
                                      max_rows, max_epochs, device=device, n_freq=n_freq, enc_cols=(1, 2, 3),
                                      max_sym=16 if symmetric else 0)
        self.dims = [self.engine.n_feat] + [width] * (depth - 1) + [n_out]
        lo, hi = W.surrogate_ranges()
        self.engine.set_inputs(lo, hi)
        self.engine.set_outputs(0 if per_power else -1, P_REF, T_REF, norm)
        if symmetric:  # the training set augmented by the 16 reflections of the cube
            self.engine.set_symmetries(*cube_symmetries(grid, n_in=n_in))
        self.tau = None

    def _dev(self):
        return f"cuda:{self.device}"

    def fit(self, Q, Y, epochs=50, batch=256, lr=1e-3, seed=0, lr_end=None, bootstrap=False):
        """Train every member (Adam on the standardised targets, seeded
        initialisation and per-epoch permutations; lr decaying by a cosine to
        lr_end when given; bootstrap resampling per member); returns the mean
        training loss per epoch of each member."""
        import torch
        X = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=self._dev())
        Yd = torch.tensor(np.asarray(Y), dtype=torch.float32, device=self._dev())
        hist = self.engine.train(X, Yd, epochs, batch, lr, seed, lr_end=lr_end, bootstrap=bootstrap)
        return [list(map(float, h)) for h in hist]

    def predict_device(self, Xd, n_spread, tol, want_std=True):
        """Ensemble answer for raw scenario rows Xd (device float32 [m][12]):
        mean and std [m][n_out] in physical units, spread [m] (max std over the
        first n_spread outputs) and fallback flags [m], all on the device."""
        import torch
        m, dev = Xd.shape[0], Xd.device
        mean = torch.empty(m, self.dims[-1], dtype=torch.float32, device=dev)
        std = torch.empty(m, self.dims[-1], dtype=torch.float32, device=dev) if want_std else None
        spread = torch.empty(m, dtype=torch.float32, device=dev)
        fb = torch.empty(m, dtype=torch.uint8, device=dev)
        for b0 in range(0, m, self.max_batch):
            sl = slice(b0, min(m, b0 + self.max_batch))
            self.engine.predict(Xd[sl], n_spread, tol, mean[sl], std[sl] if want_std else None, spread[sl], fb[sl])
        return mean, std, spread, fb

    def predict(self, Q, n_spread=0, tol=0.0):
        """Ensemble mean and standard deviation of the outputs, physical units
        (host float64 arrays)."""
        import torch
        Xd = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=self._dev())
        mean, std, _, _ = self.predict_device(Xd, n_spread, tol)
        return mean.double().cpu().numpy(), std.double().cpu().numpy()

    def calibrate(self, Q, Y, n_probe_T, tol=1.0, coverage=1.0):
        """The library's spread threshold from solver answers Y for scenarios Q:
        the largest tau <= tol such that, of the cases with spread <= tau, at
        least `coverage` have a temperature error (max over probes) <= tol;
        solve() then sends cases with spread > tau to the solver.  Returns (tau,
        accepted fraction of the calibration set)."""
        import torch
        X = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=self._dev())
        Yd = torch.tensor(np.asarray(Y), dtype=torch.float32, device=self._dev())
        self.tau, frac = self.engine.calibrate(X, Yd, n_probe_T, tol, coverage)
        return self.tau, frac

    def solve(self, Q, n_probe_T, tol=1.0, n=16, dt=0.01):
        """Surrogate answers; cases the library flags (ensemble spread of
        temperature, max over probes, above tol kelvin -- or above the
        calibrated threshold when calibrate() was called) are re-run by the
        batched solver.  Returns (outputs, fallback mask, timings)."""
        import torch
        t0 = time.perf_counter()
        Xd = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=self._dev())
        thr = self.tau
        if thr is not None and thr < 0:  # calibration accepted nothing: every case to the solver
            thr = -1.0
        mean, _, spread, fbd = self.predict_device(Xd, n_probe_T, tol if thr is None else thr, want_std=False)
        out = mean.double().cpu().numpy()
        fb = fbd.cpu().numpy().astype(bool)
        t1 = time.perf_counter()
        info = dict(surrogate_seconds=t1 - t0, fallback=int(fb.sum()), spread=spread.cpu().numpy())
        if fb.any():
            T, D, tm = solve_scenarios(np.atleast_2d(Q)[fb], n=n, dt=dt)
            out[fb] = np.concatenate([T, D], 1)
            info["solver_seconds"] = tm["seconds"]
        info["seconds"] = time.perf_counter() - t0
        return out, fb, info
