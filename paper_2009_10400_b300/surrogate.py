"""Learned surrogate for treatment planning: scenario parameters -> temperature
and damage at probe points after heating, trained on data from the batched
coupled solver, with an ensemble spread test that sends uncertain cases back
to the solver.

The network runs on the library's tensor-core kernels (``mlp.MLP``); the data
and the fallback come from ``tled.Batch``.  Normalisation, batching and the
ensemble statistics are plain tensor bookkeeping around those calls.
"""
from __future__ import annotations

import time

import numpy as np

from . import tled
from . import workloads as W
from .mlp import MLP


def mass_scaled(prob):
    """Choose the mechanical mass scale so that the fixed dt is the safe
    mechanical step (the thermal step bounds dt from above)."""
    pl = tled.HostPlanner()
    pl.set_mesh(prob.npe, prob.X, prob.conn)
    pl.set_material(tled.material_from_problem(prob))
    pl.set_params(dt=prob.dt, dt_safety=prob.dt_safety, gamma=prob.gamma, mass_scale=1.0)
    dt_mech, dt_th = pl.stable_dt()
    pl.close()
    if prob.dt > prob.dt_safety * dt_th:
        raise ValueError(f"dt {prob.dt} exceeds the thermal stable step {prob.dt_safety * dt_th}")
    prob.mass_scale = max(1.0, (prob.dt / (prob.dt_safety * dt_mech)) ** 2)
    return prob


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
            prob = mass_scaled(W.scenario_problem(q, n=n, dt=dt))
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


def he_init(dims, rng):
    """He-normal weights, zero biases, in the library's parameter order."""
    parts = []
    for K, N in zip(dims[:-1], dims[1:]):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / K), N * K))
        parts.append(np.zeros(N))
    return np.concatenate(parts).astype(np.float32)


class Surrogate:
    """Ensemble of MLPs (inputs scaled to [-1, 1] over the sampling ranges,
    outputs standardised per probe value)."""

    def __init__(self, n_out, width=512, depth=6, members=5, max_batch=4096, device=0, n_in=12):
        self.dims = [n_in] + [width] * (depth - 1) + [n_out]
        self.members = [MLP(self.dims, max_batch=max_batch, device=device) for _ in range(members)]
        self.max_batch = max_batch
        self.device = device
        self.in_lo, self.in_hi = W.surrogate_ranges()
        self.y_mean = self.y_std = None

    def _x(self, Q):
        import torch
        Xn = 2.0 * (np.atleast_2d(Q) - self.in_lo) / (self.in_hi - self.in_lo) - 1.0
        return torch.tensor(Xn, dtype=torch.float32, device=f"cuda:{self.device}")

    def fit(self, Q, Y, epochs=50, batch=256, lr=1e-3, seed=0):
        """Adam on the mean squared error of the standardised outputs, every
        member from its own initialisation and sample order; returns the mean
        training loss per epoch of each member."""
        import torch
        Y = np.asarray(Y, np.float64)
        self.y_mean = Y.mean(0)
        self.y_std = np.maximum(Y.std(0), 1e-3 * max(Y.std(), 1e-12))
        dev = f"cuda:{self.device}"
        Xd = self._x(Q)
        Yd = torch.tensor((Y - self.y_mean) / self.y_std, dtype=torch.float32, device=dev)
        n = len(Q) - len(Q) % batch
        hist = []
        for mi, net in enumerate(self.members):
            rng = np.random.default_rng(seed + 1000 * mi)
            net.set_params(he_init(self.dims, rng))
            g = torch.Generator(device=dev)
            g.manual_seed(seed + mi)
            losses = []
            for _ in range(epochs):
                perm = torch.randperm(len(Q), device=dev, generator=g)[:n]
                xs, ys = Xd[perm], Yd[perm]  # one shuffle per epoch, then contiguous batches
                acc = torch.zeros(1, dtype=torch.float32, device=dev)
                for b0 in range(0, n, batch):
                    acc += net.train_step(xs[b0:b0 + batch], ys[b0:b0 + batch], lr)
                losses.append(acc)
            net.sync()
            hist.append([float(v) / (n // batch) for v in torch.stack(losses).cpu()])
        return hist

    def predict(self, Q):
        """Ensemble mean and standard deviation of the outputs, physical units."""
        import torch
        Xd = self._x(Q)
        m = len(Q)
        B = self.max_batch
        pad = (-m) % 128
        if pad:
            Xd = torch.cat([Xd, torch.zeros(pad, Xd.shape[1], device=Xd.device)])
        outs = []
        for net in self.members:
            ys = [net.forward(Xd[b0:b0 + B]) for b0 in range(0, len(Xd), B)]
            outs.append(torch.cat(ys)[:m])
        S = torch.stack(outs)
        scale = torch.tensor(self.y_std, dtype=torch.float32, device=S.device)
        shift = torch.tensor(self.y_mean, dtype=torch.float32, device=S.device)
        mean = (S.mean(0) * scale + shift).double().cpu().numpy()
        std = (S.std(0, unbiased=False) * scale).double().cpu().numpy()
        return mean, std

    def solve(self, Q, n_probe_T, tol=1.0, n=16, dt=0.01):
        """Surrogate answers; cases whose ensemble spread of temperature (max over
        probes) exceeds tol kelvin are re-run by the batched solver.  Returns
        (outputs, fallback mask, timings)."""
        t0 = time.perf_counter()
        mean, std = self.predict(Q)
        t1 = time.perf_counter()
        spread = std[:, :n_probe_T].max(1)
        fb = spread > tol
        out = mean.copy()
        info = dict(surrogate_seconds=t1 - t0, fallback=int(fb.sum()))
        if fb.any():
            T, D, tm = solve_scenarios(np.atleast_2d(Q)[fb], n=n, dt=dt)
            out[fb] = np.concatenate([T, D], 1)
            info["solver_seconds"] = tm["seconds"]
        info["seconds"] = time.perf_counter() - t0
        return out, fb, info
