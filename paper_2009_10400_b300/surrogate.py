"""Learned surrogate for treatment planning: scenario parameters -> temperature
and damage at probe points after heating, trained on data from the batched
coupled solver, with an ensemble spread test that sends uncertain cases back
to the solver.

The network runs on the library's tensor-core kernels (``mlp.MLP``): the input
map, the mini-batch row gather, training, inference and the ensemble
statistics with the fallback decision are library kernels; the data and the
fallback answers come from ``tled.Batch``.  The Python side only shuffles row
indices, standardises the training targets once and moves arrays.
"""
from __future__ import annotations

import time

import numpy as np

from . import tled
from . import workloads as W
from .mlp import MLP


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


def spread_threshold(spread, err, tol, coverage=1.0):
    """Largest spread threshold tau (<= tol) such that the cases with spread <=
    tau -- a prefix of the cases sorted by spread -- have err <= tol in at least
    a `coverage` fraction; -1 if no prefix qualifies (everything to the solver).
    Returns (tau, accepted fraction)."""
    spread, err = np.asarray(spread, float), np.asarray(err, float)
    order = np.argsort(spread, kind="stable")
    ok = np.cumsum(err[order] <= tol) / np.arange(1, len(order) + 1)  # coverage of each prefix
    good = np.nonzero(ok >= coverage)[0]
    if not len(good):
        return -1.0, 0.0
    k = int(good[-1]) + 1  # the longest qualifying prefix
    tau = float(spread[order[k - 1]])
    if tau > tol:  # never accept a spread above the tolerance itself
        k = int(np.searchsorted(spread[order], tol, side="right"))
        tau = tol
    return tau, k / len(order)


def he_init(dims, rng):
    """He-normal weights, zero biases, in the library's parameter order."""
    parts = []
    for K, N in zip(dims[:-1], dims[1:]):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / K), N * K))
        parts.append(np.zeros(N))
    return np.concatenate(parts).astype(np.float32)


P_REF = 5e6  # W/m^3: the temperature outputs are learned per unit of power / P_REF
T_REF = 37.0  # C: initial and arterial temperature of the scenarios


class Surrogate:
    """Ensemble of MLPs.  Inputs are mapped to [-1, 1] over the sampling ranges
    inside the first layer's input kernel.  The first n_T outputs are
    temperatures: with `per_power` the network learns the temperature rise per
    unit source power, (T - T_REF) / (P / P_REF) -- the bioheat part of the
    model is linear in the source power (c and k temperature independent, the
    source centre moves with displacements of ~1e-5 m), which removes a factor
    of ten of dynamic range from the regression -- and the ensemble kernel
    multiplies it back by each scenario's power read from its raw input row.
    All outputs are learned standardised per output and mapped back by the
    ensemble kernel."""

    def __init__(self, n_out, width=512, depth=6, members=5, max_batch=4096, device=0, n_in=12, n_T=None,
                 per_power=True):
        self.n_T = n_out // 2 if n_T is None else n_T
        self.per_power = per_power
        self.dims = [n_in] + [width] * (depth - 1) + [n_out]
        self.members = [MLP(self.dims, max_batch=max_batch, device=device) for _ in range(members)]
        self.max_batch = max_batch
        self.device = device
        lo, hi = W.surrogate_ranges()
        for net in self.members:
            net.set_input_scaling(0.5 * (lo + hi), 2.0 / (hi - lo))
        self.y_mean = self.y_std = None
        self._ys = None
        self._side = None  # one stream per member for side-by-side inference

    def _dev(self):
        return f"cuda:{self.device}"

    def fit(self, Q, Y, epochs=50, batch=256, lr=1e-3, seed=0):
        """Adam on the mean squared error of the standardised outputs, every
        member from its own initialisation and sample order (one seeded
        permutation of the rows per epoch, consumed in contiguous mini-batches
        of the device-resident data set); returns the mean training loss per
        epoch of each member."""
        import torch
        Y = np.array(Y, np.float64)
        if self.per_power:
            Y[:, :self.n_T] = (Y[:, :self.n_T] - T_REF) / (np.atleast_2d(Q)[:, :1] / P_REF)
        self.y_mean = Y.mean(0)
        self.y_std = np.maximum(Y.std(0), 1e-3 * max(Y.std(), 1e-12))
        dev = self._dev()
        self._scale = torch.tensor(self.y_std, dtype=torch.float32, device=dev)
        self._shift = torch.tensor(self.y_mean, dtype=torch.float32, device=dev)
        off = np.zeros(self.dims[-1])
        if self.per_power:
            off[:self.n_T] = T_REF
        self._offset = torch.tensor(off, dtype=torch.float32, device=dev)
        Xd = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=dev)
        Yd = torch.tensor((Y - self.y_mean) / self.y_std, dtype=torch.float32, device=dev)
        n = len(Q) - len(Q) % batch
        hist = []
        for mi, net in enumerate(self.members):
            rng = np.random.default_rng(seed + 1000 * mi)
            net.set_params(he_init(self.dims, rng))
            losses = []
            for _ in range(epochs):
                perm = torch.tensor(rng.permutation(len(Q))[:n].astype(np.int32), device=dev)
                acc = torch.zeros(1, dtype=torch.float32, device=dev)
                for b0 in range(0, n, batch):
                    acc += net.train_step_rows(Xd, Yd, perm[b0:b0 + batch], lr)
                losses.append(acc)
            net.sync()
            hist.append([float(v) / (n // batch) for v in torch.stack(losses).cpu()])
        return hist

    def predict_device(self, Xd, n_spread, tol, want_std=True):
        """Ensemble answer for raw scenario rows Xd (device float32 [m][12]):
        mean and std [m][n_out] in physical units, spread [m] (max std over the
        first n_spread outputs) and fallback flags [m], all on the device."""
        import torch
        from .mlp import ensemble
        m = Xd.shape[0]
        pad = (-m) % 128
        if pad:
            Xd = torch.cat([Xd, torch.zeros(pad, Xd.shape[1], dtype=Xd.dtype, device=Xd.device)])
        mp = m + pad
        if self._ys is None or self._ys[0].shape[0] < mp:
            self._ys = [torch.empty(mp, self.dims[-1], dtype=torch.float32, device=Xd.device)
                        for _ in self.members]
        ys = [y[:mp] for y in self._ys]
        # the members' forward passes side by side, one stream each, joined before the
        # ensemble statistics (the outputs live across calls, the inputs outlive the join)
        main = torch.cuda.current_stream(self.device)
        if self._side is None:
            self._side = [torch.cuda.Stream(device=self.device) for _ in self.members]
        ready = main.record_event()
        for net, y, side in zip(self.members, ys, self._side):
            side.wait_event(ready)
            net.set_stream(side)
            for b0 in range(0, mp, self.max_batch):
                net.forward(Xd[b0:b0 + self.max_batch], out=y[b0:b0 + self.max_batch])
            net.set_stream(main)
            main.wait_stream(side)
        if self.per_power:
            mean, std, spread, fb = ensemble(ys, self._scale, self._shift, n_spread, tol, device=self.device,
                                             want_std=want_std, row_src=Xd, row_mult=1.0 / P_REF,
                                             n_row_scaled=self.n_T, out_offset=self._offset)
        else:
            mean, std, spread, fb = ensemble(ys, self._scale, self._shift, n_spread, tol, device=self.device,
                                             want_std=want_std)
        return mean[:m], (std[:m] if std is not None else None), spread[:m], fb[:m]

    def predict(self, Q, n_spread=0, tol=0.0):
        """Ensemble mean and standard deviation of the outputs, physical units
        (host float64 arrays)."""
        import torch
        Xd = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=self._dev())
        mean, std, _, _ = self.predict_device(Xd, n_spread, tol)
        return mean.double().cpu().numpy(), std.double().cpu().numpy()

    def calibrate(self, Q, Y, n_probe_T, tol=1.0, coverage=1.0):
        """Spread threshold from solver answers: on calibration scenarios Q with
        solver outputs Y, the largest threshold tau on the ensemble spread such
        that, among the cases with spread <= tau, at least `coverage` of them
        have a temperature error (max over probes) <= tol.  solve() then sends
        cases with spread > tau to the solver.  Returns (tau, accepted fraction
        of the calibration set)."""
        mean, std = self.predict(Q)
        err = np.abs(mean[:, :n_probe_T] - np.asarray(Y)[:, :n_probe_T]).max(1)
        spread = std[:, :n_probe_T].max(1)
        self.tau, frac = spread_threshold(spread, err, tol, coverage)
        return self.tau, frac

    def solve(self, Q, n_probe_T, tol=1.0, n=16, dt=0.01):
        """Surrogate answers; cases whose ensemble spread of temperature (max over
        probes) exceeds the threshold -- tol kelvin, or the calibrated threshold
        when calibrate() was called -- are re-run by the batched solver.  Returns
        (outputs, fallback mask, timings)."""
        import torch
        t0 = time.perf_counter()
        Xd = torch.tensor(np.atleast_2d(Q), dtype=torch.float32, device=self._dev())
        thr = getattr(self, "tau", None)
        mean, _, spread, fbd = self.predict_device(Xd, n_probe_T, tol if thr is None else max(thr, 0.0),
                                                   want_std=False)
        out = mean.double().cpu().numpy()
        fb = fbd.cpu().numpy().astype(bool)
        if thr is not None and thr < 0:  # calibration accepted nothing
            fb[:] = True
        t1 = time.perf_counter()
        info = dict(surrogate_seconds=t1 - t0, fallback=int(fb.sum()), spread=spread.cpu().numpy())
        if fb.any():
            T, D, tm = solve_scenarios(np.atleast_2d(Q)[fb], n=n, dt=dt)
            out[fb] = np.concatenate([T, D], 1)
            info["solver_seconds"] = tm["seconds"]
        info["seconds"] = time.perf_counter() - t0
        return out, fb, info
