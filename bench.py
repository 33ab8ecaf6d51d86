#!/usr/bin/env python3
"""Benchmark of the coupled thermo-visco-hyperelastic TLED step on B300.

A bench "step" is one explicit coupled time step of the whole mesh: element
pass, deterministic node gather, and the displacement / temperature / damage
updates.  The default workload is the 128^3 hexahedral block (2,097,152 H8,
2,146,689 nodes, +-10 % per-element material noise, 4 Gaussian sources).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload block_h8|ellipsoid_t4]
    python bench.py --impl reference ...     # the FP64 CPU oracle, timed on host cores

Prints one JSON line.  Metric: coupled element-steps per second (whole job),
plus the HBM roofline fraction of the fused step kernels.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled element-steps/s"
UNIT = "element-steps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def make_problem(workload):
    from paper_2009_10400_b300 import workloads as W

    if workload == "block_h8":
        return W.block_h8(n=128)
    if workload == "ellipsoid_t4":
        return W.ellipsoid_t4()
    if workload == "cube_h8_8":
        return W.cube_h8(n=8)
    if workload.startswith("block_h8_"):  # block_h8_N (h = 1 mm) or block_h8_N_hXmm
        parts = workload.split("_")
        h = float(parts[3][1:-2]) * 1e-3 if len(parts) > 3 else 1e-3
        return W.block_h8(n=int(parts[2]), h=h)
    raise SystemExit(f"unknown workload {workload}")


def probe_lattice(prob, n):
    """n^3 probe points: on a block, a lattice spanning the inner 80 % of its box; on
    any other mesh (whose box holds points outside it), the centroids of n^3
    elements spread evenly over the element order."""
    if prob.name.startswith("block_h8"):
        lo, hi = prob.X.min(0), prob.X.max(0)
        g = [np.linspace(lo[j] + 0.1 * (hi[j] - lo[j]), hi[j] - 0.1 * (hi[j] - lo[j]), n) for j in range(3)]
        return np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    idx = np.linspace(0, prob.ne - 1, min(n ** 3, prob.ne)).astype(np.int64)
    return prob.X[prob.conn[idx]].mean(1)


def algorithmic_bytes(prob, n_prony):
    """Layout-independent floor of the bytes one coupled step must move: every
    element constant and state array touched once -- connectivity (int32),
    shape-function derivatives dh/dX (3 floats per corner), V0, the
    per-element material (mu, kappa, k1, k2, k, alpha) and fibre when they
    vary, the Prony state read and written (6 floats per term each way) -- and
    per node the gather of u and theta (16 B), X0 (12), u hi/lo read and write
    (48), v read and write (24), theta hi/lo read and write (16), Omega read
    and write (8) and m, V, mask (12): 136 B.  (H8 with per-element material
    and one Prony term: 204 B per element + 136 B per node.)"""
    npe = prob.npe
    elem = npe * (4 + 12) + 4 + 2 * 4 * 6 * n_prony
    if prob.per_element:
        if not all(np.allclose(getattr(prob, f), getattr(prob, f)[0]) for f in ("mu", "kappa", "k1", "k2", "kc",
                                                                                  "alpha")):
            elem += 6 * 4
        if not np.allclose(prob.a0, prob.a0[0]):
            elem += 3 * 4
    return elem * prob.ne + 136 * prob.nn


def layout_bytes(prob, n_prony, brick=False):
    """Bytes the same step moves in this library's layout (uint16 local
    connectivity -- an upper bound: tiles of equal structure share one record --,
    J0^-1 instead of dh/dX, its diagonal for axis-aligned bricks, float4 nodal
    records): element record 2 npe + 40 B (bricks 2 npe + 16 B; +24 material,
    +12 fibre) and the Prony state, 128 B per node."""
    npe = prob.npe
    elem = 2 * npe + (3 if brick else 9) * 4 + 4 + 2 * 4 * 6 * n_prony
    if prob.per_element:
        elem += 6 * 4
        if not np.allclose(prob.a0, prob.a0[0]):
            elem += 3 * 4
    return elem * prob.ne + 128 * prob.nn


def kernel_traffic(workload):
    """DRAM bytes (read + write) per step of the tile and shared-node kernels
    from the committed ncu capture, or None when there is none for this
    workload or the kernel source has changed since it was taken."""
    import hashlib

    try:
        entry = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[workload]
        src = open(os.path.join(ROOT, "paper_2009_10400_b300", "csrc", "tled_kernels.cu"), "rb").read()
        if hashlib.sha1(src).hexdigest() != entry["kernel_source_sha1"]:
            return None
        return float(entry["dram_bytes_per_step"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """SM clock and throttle-reason sampling during the timed region, in
    process through NVML (the driver's libnvidia-ml, read-only queries) every
    ~1 ms from a background thread, so that even a few-millisecond region gets
    samples and no nvidia-smi process competes with the timed work.  Use
    mark_start()/mark_end() around the region; summary() reports the samples
    inside it (or the nearest ones, stated, if the region was shorter than one
    sampling interval)."""

    # NVML clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index, interval=1e-3):
        self.index = index
        self.interval = interval
        self.samples = []  # (host time, sm MHz, reasons bitmask)
        self.max_mhz = None
        self.t_start = self.t_end = None
        self._stop = threading.Event()
        self._nvml = None

    def _open(self):
        import ctypes as C

        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                L = C.CDLL(name)
                break
            except OSError:
                L = None
        if L is None or L.nvmlInit_v2() != 0:
            return None
        h = C.c_void_p()
        if L.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(h)) != 0:
            return None
        mx = C.c_uint()
        if L.nvmlDeviceGetMaxClockInfo(h, C.c_int(1), C.byref(mx)) == 0:  # NVML_CLOCK_SM = 1
            self.max_mhz = float(mx.value)
        return L, h

    def _run(self):
        import ctypes as C

        L, h = self._nvml
        clk, rs = C.c_uint(), C.c_ulonglong()
        get_reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            t = time.perf_counter()
            if L.nvmlDeviceGetClockInfo(h, C.c_int(1), C.byref(clk)) == 0 and get_reasons(h, C.byref(rs)) == 0:
                self.samples.append((t, float(clk.value), int(rs.value)))
            self._stop.wait(self.interval)

    def __enter__(self):
        try:
            self._nvml = self._open()
        except Exception:
            self._nvml = None
        if self._nvml:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
            time.sleep(0.02)  # a few samples before the region
        return self

    def mark_start(self):
        self.t_start = time.perf_counter()

    def mark_end(self):
        self.t_end = time.perf_counter()

    def __exit__(self, *a):
        if self._nvml:
            time.sleep(0.005)
            self._stop.set()
            self._thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "samples": 0,
                    "source": "nvml"}
        t0 = self.t_start if self.t_start is not None else self.samples[0][0]
        t1 = self.t_end if self.t_end is not None else self.samples[-1][0]
        inside = [x for x in self.samples if t0 <= x[0] <= t1]
        where = "inside the timed region"
        if not inside:  # region shorter than a sampling interval: the samples around it
            inside = sorted(self.samples, key=lambda x: min(abs(x[0] - t0), abs(x[0] - t1)))[:2]
            where = "nearest to the timed region (shorter than one sampling interval)"
        mask = 0
        for x in inside:
            mask |= x[2]
        reasons = sorted(n for b, n in self.REASONS.items() if mask & b)
        return {"sm_mhz": float(np.median([x[1] for x in inside])), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(inside), "source": "nvml", "where": where}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_sample(prob, max_steps, seconds=12.0, warmup=1, warmup_seconds=10.0, parallel=False):
    """Time the FP64 oracle as it stands on a bounded sample of the workload:
    up to `warmup` untimed steps (at least one, stopping after about
    `warmup_seconds`), then as many full steps as fit in about `seconds` (at
    least 1, at most max_steps).  parallel: the oracle's OpenMP step on every
    host core (elements in parallel, fixed-order node gather; bitwise the
    single-threaded result)."""
    import oracle

    t0 = time.perf_counter()
    m = oracle.OracleModel(prob)
    setup = time.perf_counter() - t0
    s = m.init_state()
    step = m.step_parallel if parallel else m.step
    cores = oracle.threads() if parallel else 1
    t0 = time.perf_counter()
    n_warm, one = 0, float("inf")
    while n_warm < max(1, warmup):
        t1 = time.perf_counter()
        step(s, 1)
        one = min(one, time.perf_counter() - t1)  # the first step also starts the thread pool
        n_warm += 1
        if time.perf_counter() - t0 > warmup_seconds:
            break
    steps = int(max(1, min(max_steps, seconds // max(one, 1e-9))))
    t0 = time.perf_counter()
    step(s, steps)
    el = time.perf_counter() - t0
    how = f"OpenMP on {cores} host cores, fixed-order node gather" if parallel else "single-threaded"
    return {"value": prob.ne * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{prob.name}: {steps} full steps after {n_warm} warm-up step(s) ({el:.1f} s, "
                      f"set-up {setup:.1f} s), FP64 C oracle, {how}", "steps": steps, "warmup": n_warm,
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


def cpu_sample_subprocess(args, parallel, workload=None, max_steps=None, seconds=None):
    """cpu_oracle_sample of a workload (default: the bench's) in a fresh Python process."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload or args.workload,
           "--cpu-steps", str(max_steps or args.cpu_steps), "--cpu-seconds", str(seconds or args.cpu_seconds)]
    if parallel:
        cmd.append("--cpu-parallel")
    r = subprocess.run(cmd, capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_trajectory_child(workload, n_steps, every, dt, path):
    """Child process of the precision leg: the FP64 oracle's trajectory of the
    workload on all host cores, snapshots (u, T, Omega) every `every` steps to
    an .npz file."""
    import oracle

    prob = make_problem(workload)
    m = oracle.OracleModel(prob, dt=dt)
    s = m.init_state()
    snaps = {}
    for k in range(every, n_steps + 1, every):
        m.step_parallel(s, every)
        snaps[f"u{k}"], snaps[f"T{k}"], snaps[f"O{k}"] = s.u.copy(), s.T.copy(), s.Omega.copy()
    np.savez(path, **snaps)


def rel_l2(a, b):
    """The paper's error indicator e = ||a - b||_2 / ||b||_2 (Section 6.1)."""
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def nre_max(a, b):
    """Maximum normalised relative error |a - b| / (max b - min b) (Section 6.1)."""
    a, b = np.ravel(a), np.ravel(b)
    return float(np.abs(a - b).max() / np.ptp(b))


def precision_leg(args, device, stream, n=32, n_steps=5000, every=1000):
    """Per-result error against the FP64 oracle for the 128^3 block's generator
    at n^3 (h = 4 mm): n_steps steps, compared every `every` steps, with the
    float-float accumulation of u and T on (the product setting) and off."""
    import tempfile

    from paper_2009_10400_b300 import tled

    workload = f"block_h8_{n}_h4mm"
    prob = make_problem(workload)
    base = tled.default_flags(prob)
    runs = {"compensated": base, "plain_fp32": base & ~tled.COMPENSATED}
    gs = {k: tled.Solver.from_problem(prob, device=device, stream=stream, flags=f) for k, f in runs.items()}
    dt = gs["compensated"].get_dt()[0]
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "oracle.npz")
        t0 = time.perf_counter()
        subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-trajectory", path, "--workload", workload,
                        "--steps", str(n_steps), "--oracle-every", str(every), "--oracle-dt", repr(dt)], check=True)
        oracle_s = time.perf_counter() - t0
        ref = dict(np.load(path))
    out = {"workload": f"{workload}: the 128^3 block's generator at {n}^3, h = 4 mm, {prob.ne} H8, {n_steps} "
                       f"steps at dt {dt:.4e} s", "every": every, "oracle": "FP64 C oracle, OpenMP on all host cores",
           "oracle_s": oracle_s, "tolerance": {"e_u": 1e-4, "e_theta": 1e-4, "damage_abs": 1e-3}}
    for name, g in gs.items():
        rows = []
        for k in range(every, n_steps + 1, every):
            g.step(every)
            g.sync()
            u, T, d = g.displacement(), g.temperature(), g.damage()
            uo, To, Oo = ref[f"u{k}"], ref[f"T{k}"], ref[f"O{k}"]
            rows.append({"step": k, "e_u": rel_l2(u, uo), "e_theta": rel_l2(T - prob.T0, To - prob.T0),
                         "nre_u": nre_max(u, uo), "nre_T": nre_max(T, To),
                         "damage_abs": float(np.abs(d + np.expm1(-Oo)).max())})
        out[name] = rows
        g.close()
    out["peak_rise_K"] = float(ref[f"T{n_steps}"].max() - prob.T0)
    return out


def workload_config(prob):
    """The `config` object of a bench line: what the workload is (the same for
    both arms)."""
    return {"workload": prob.name, "elements": prob.ne, "nodes": prob.nn,
            "element": "H8" if prob.npe == 8 else "T4",
            "floor_bytes_per_step": algorithmic_bytes(prob, len(prob.prony_g)),
            "l2": "inputs larger than L2 (no flush needed)" if algorithmic_bytes(prob, len(prob.prony_g)) > 126e6
            else "L2-resident working set"}


def run_reference(args):
    """The reference arm: the FP64 oracle on all host cores (OpenMP, bitwise
    the single-threaded oracle), same workload, metric and unit.  Exactly
    --warmup untimed and --steps timed steps; each step is one oracle step of
    the whole workload, or -- when W + K full steps would not fit in about
    --ref-seconds -- of a smaller block of the same generator (stated)."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle

    prob = make_problem(args.workload if args.workload != "surrogate" else "block_h8")
    sample = prob
    t0 = time.perf_counter()
    m = oracle.OracleModel(sample)
    s = m.init_state()
    m.step_parallel(s, 1)
    one = time.perf_counter() - t0
    t0 = time.perf_counter()
    m.step_parallel(s, 1)
    one = time.perf_counter() - t0
    n_total = args.warmup + args.steps
    if prob.name.startswith("block_h8") and n_total * one > args.ref_seconds:
        # a smaller block of the same generator: element count scaled to fit the budget
        from paper_2009_10400_b300 import workloads as W

        n_side = round(prob.ne ** (1 / 3))
        k = max(8, int(n_side * (args.ref_seconds / (n_total * one)) ** (1 / 3)))
        sample = W.block_h8(n=k)
        m = oracle.OracleModel(sample)
        s = m.init_state()
    m.step_parallel(s, args.warmup)
    t0 = time.perf_counter()
    m.step_parallel(s, args.steps)
    el = time.perf_counter() - t0
    value = sample.ne * args.steps / el
    cores = oracle.threads()
    what = "every step one step of the whole workload" if sample is prob else \
        f"every step one step of the same generator's {sample.name} ({sample.ne} elements; {prob.ne} would not fit)"
    cpu = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{what}: {args.steps} timed steps after {args.warmup} warm-up steps ({el:.1f} s), FP64 C "
                     f"oracle, OpenMP on {cores} host cores with a fixed-order node gather (bitwise the "
                     f"single-threaded oracle)", "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    # run on the host cores of the launch's box (n_gpus = the launch's world size, for bookkeeping)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(prob),
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def small_configs(device, stream, steps=2000, args=None):
    """The L2-resident workloads (8^3 H8 cube; ~120k-tet ellipsoid): steps/s,
    element-steps/s and the floor bytes per second they stream from L2 (no HBM
    fraction is claimed for them), beside the FP64 oracle on all host cores
    (a bounded sample in a child process)."""
    import torch

    from paper_2009_10400_b300 import tled
    from paper_2009_10400_b300 import workloads as W

    out = []
    for prob in (W.cube_h8(n=8), W.ellipsoid_t4()):
        s = tled.Solver.from_problem(prob, device=device, stream=stream)
        s.step(64)
        s.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) * 1e-3
        s.sync()
        s.close()
        row = {"workload": prob.name, "elements": prob.ne, "nodes": prob.nn, "steps": steps,
               "steps_per_s": steps / sec, "element_steps_per_s": prob.ne * steps / sec,
               "floor_bytes_per_step": algorithmic_bytes(prob, len(prob.prony_g)),
               "l2_gbs": algorithmic_bytes(prob, len(prob.prony_g)) * steps / sec / 1e9}
        if args is not None and not args.no_cpu_baseline:
            name = "cube_h8_8" if prob.npe == 8 else "ellipsoid_t4"
            row["cpu_oracle"] = cpu_sample_subprocess(args, True, workload=name, max_steps=steps, seconds=6.0)
        out.append(row)
    return out


def cpu_planning_sample(n_scen, n_sub, max_steps=200):
    """The batched planning workload's CPU reference: the FP64 oracle on all host
    cores over a stratified subset of the scenarios, each run for at most
    max_steps steps and its time extrapolated to the scenario's step count."""
    import oracle
    from paper_2009_10400_b300 import workloads as W

    scen = W.planning_scenarios(n_scen)
    sub = list(range(0, len(scen), max(1, len(scen) // n_sub)))[:n_sub]
    total, el_steps = 0.0, 0
    for i in sub:
        p = scen[i]
        m = oracle.OracleModel(p)
        s = m.init_state()
        m.step_parallel(s, 2)  # first touch
        k = min(max_steps, p.n_steps)
        t0 = time.perf_counter()
        m.step_parallel(s, k)
        total += (time.perf_counter() - t0) * p.n_steps / k
        el_steps += p.ne * p.n_steps
    return {"solves_per_s": len(sub) / total, "element_steps_per_s": el_steps / total, "cores": oracle.threads(),
            "sample": f"{len(sub)} of the {n_scen} scenarios (stratified), each {max_steps} steps timed and its time "
                      f"extrapolated to its step count, FP64 C oracle, OpenMP on {oracle.threads()} host cores",
            "kind": "oracle", "extrapolated": True}


def planning_bench(args, device, stream):
    """Batched treatment planning: every scenario to the end of its heating
    time in one batch (one launch per step, autotuned tiling), against running
    a stratified subset of the same scenarios one solver at a time; both timed
    with CUDA events on the solver stream, set-up excluded.  The subset's plain
    results are compared with the batch's to show both are the same solve."""
    import torch

    from paper_2009_10400_b300 import tled
    from paper_2009_10400_b300 import workloads as W

    t_setup = time.perf_counter()
    scen = W.planning_scenarios(args.plan_scenarios)  # R17 mass scaling chosen by the library
    b = tled.Batch(device=device, stream=stream)
    for p in scen:
        b.add(p, p.n_steps)
    b.init()
    tune = b.autotune(trial_steps=10)
    setup_s = time.perf_counter() - t_setup
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    launch_steps = b.run()
    ev1.record(stream)
    torch.cuda.synchronize()
    batch_s = ev0.elapsed_time(ev1) * 1e-3
    st = b.stats()
    Tb = b.temperature()
    Db = b.damage()
    infos = [b.scenario(i) for i in range(len(scen))]
    b.close()

    sub = list(range(0, len(scen), max(1, len(scen) // args.plan_subset)))[:args.plan_subset]
    plain_s, du, dT, dD = 0.0, 0.0, 0.0, 0.0
    for i in sub:
        p = scen[i]
        s = tled.Solver.from_problem(p, device=device, stream=stream)
        s.step(1)  # graph capture outside the timed region; advances one step
        s.sync()
        ev0.record(stream)
        s.step(p.n_steps - 1)
        ev1.record(stream)
        torch.cuda.synchronize()
        plain_s += ev0.elapsed_time(ev1) * 1e-3 * p.n_steps / max(1, p.n_steps - 1)
        sl = slice(infos[i]["node_off"], infos[i]["node_off"] + infos[i]["nodes"])
        dT = max(dT, float(np.abs(s.temperature() - Tb[sl]).max()))
        dD = max(dD, float(np.abs(s.damage() - Db[sl]).max()))
        s.close()
    n = len(scen)
    el_steps = sum(p.ne * p.n_steps for p in scen)
    plain_rate = len(sub) / plain_s
    return {
        "workload": f"planning_{n}: hex or tet 5 cm cube, 2k-60k elements (log-uniform), 60-600 s at dt 0.01 s "
                    "with mass scaling, 1-10 MW/m^3 source in the inner half, mu and k x U(0.8, 1.2)",
        "scenarios": n, "elements": int(sum(p.ne for p in scen)), "element_steps": int(el_steps),
        "batched_solves_per_s": n / batch_s, "batched_s": batch_s, "launch_steps": int(launch_steps),
        "batched_element_steps_per_s": el_steps / batch_s,
        "plain_solves_per_s": plain_rate, "plain_subset": len(sub), "plain_subset_s": plain_s,
        "speedup": (n / batch_s) / plain_rate,
        "autotune": tune, "setup_s": setup_s,
        "subset_max_abs_diff": {"T_K": dT, "damage": dD},
        "status": st["status"],
    }


def run_surrogate(args):
    """Learned surrogate workload: training data from the batched solver, the
    ensemble trained on the tensor-core kernels, then inference on a batch of
    4096 scenarios (device-timed: the members' forward passes and the ensemble
    kernel) and end to end (scenario rows from pinned host memory, answers and
    fallback flags back to pinned host memory), and the fallback to the solver
    on the test scenarios above the spread tolerance."""
    import torch

    from paper_2009_10400_b300 import surrogate
    from paper_2009_10400_b300 import workloads as W

    torch.cuda.set_device(0)
    dev = "cuda:0"
    stream = torch.cuda.current_stream()
    n, P = args.sur_grid, args.sur_grid ** 3
    n_train, n_test = args.sur_scenarios, args.sur_test
    Q = W.sample_scenarios(n_train + n_test, seed=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T, D, tm = surrogate.solve_scenarios(Q, n=n, dt=0.01, chunk=args.sur_chunk)
    gen_s = time.perf_counter() - t0
    Y = np.concatenate([T, D], 1)
    tr, te = slice(0, n_train), slice(n_train, n_train + n_test)
    # the training set augmented by the cube's 16 reflections (an epoch is a pass over it)
    n_sym = 16
    sur = surrogate.Surrogate(n_out=2 * P, width=512, depth=6, members=args.sur_members, max_batch=4096,
                              symmetric=True, grid=n, max_rows=n_sym * n_train, max_epochs=max(64, args.sur_epochs))
    t0 = time.perf_counter()
    hist = sur.fit(Q[tr], Y[tr], epochs=args.sur_epochs, batch=256, lr=1e-3, seed=0,
                   lr_end=args.sur_lr_end if args.sur_lr_end > 0 else None)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    n_train_steps = args.sur_members * args.sur_epochs * (n_sym * n_train // 256)

    # ---- inference, device-timed: members' forwards + ensemble kernel, inputs resident
    Bq = 4096
    big = np.resize(Q[te], (Bq, Q.shape[1]))
    Xd = torch.tensor(big, dtype=torch.float32, device=dev)
    for _ in range(3):
        sur.predict_device(Xd, P, args.sur_tol)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        sur.predict_device(Xd, P, args.sur_tol)
    ev1.record(stream)
    torch.cuda.synchronize()
    inf_s = ev0.elapsed_time(ev1) * 1e-3 / reps
    flop = 2.0 * Bq * args.sur_members * sum(k * m for k, m in zip(sur.dims[:-1], sur.dims[1:]))
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        psrc = "measured"
    except Exception:
        peak, psrc = 1800.0, "fallback"
    # ---- end to end: pinned host rows in, mean (float32), spread and flags out
    Xh = torch.tensor(big, dtype=torch.float32).pin_memory()
    Mh = torch.empty((Bq, 2 * P), dtype=torch.float32).pin_memory()
    Sh = torch.empty(Bq, dtype=torch.float32).pin_memory()
    Fh = torch.empty(Bq, dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        xd = Xh.to(dev, non_blocking=True)
        mean, _, spread, fbd = sur.predict_device(xd, P, args.sur_tol, want_std=False)
        Mh.copy_(mean, non_blocking=True)
        Sh.copy_(spread, non_blocking=True)
        Fh.copy_(fbd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / reps

    # ---- held-out scenarios: the first half calibrates the spread threshold against
    #      the solver's answers, the second half is answered (surrogate or fallback)
    n_cal = n_test // 2
    cal = slice(n_train, n_train + n_cal)
    ev = slice(n_train + n_cal, n_train + n_test)
    mean_te, std_te = sur.predict(Q[te])
    err_sur = np.abs(mean_te[:, :P] - T[te]).max(1)
    spread_te = std_te[:, :P].max(1)
    raw_acc = spread_te <= args.sur_tol
    # the fallback rule as written (spread above the tolerance goes to the solver) ...
    out_r, fb_r, info_r = sur.solve(Q[ev], P, tol=args.sur_tol, n=n, dt=0.01)
    err_r = np.abs(out_r[:, :P] - T[ev]).max(1)
    # ... and with the threshold calibrated against the solver on the other held-out half
    # (calibrated against a tolerance below the stated one, so that the threshold carries a margin
    # to the scenarios it has not seen)
    tau, cal_acc = sur.calibrate(Q[cal], Y[cal], P, tol=args.sur_tol * args.sur_cal_margin,
                                 coverage=args.sur_coverage)
    out, fb, info = sur.solve(Q[ev], P, tol=args.sur_tol, n=n, dt=0.01)
    err_out = np.abs(out[:, :P] - T[ev]).max(1)
    acc = ~fb
    solver_rate = (n_train + n_test) / tm["seconds"]
    line = {
        "metric": "surrogate scenario-solves/s", "value": Bq / inf_s, "unit": "scenario-solves/s",
        "n_gpus": 1, "steps": reps, "warmup": 3, "ms_per_step": 1e3 * inf_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
        "config": {"workload": f"surrogate: {n}^3 H8 cube, {P} probes, {2 * P} outputs, MLP {sur.dims}, "
                               f"{args.sur_members} members, {args.sur_epochs} epochs, batch 256, inference {Bq}",
                   "train_scenarios": n_train, "test_scenarios": n_test, "tol_K": args.sur_tol,
                   "step": f"one ensemble inference of {Bq} scenarios (members' forwards + ensemble statistics)"},
        "roofline": {"bound": "tensor", "achieved": flop / inf_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flop / inf_s / 1e12 / peak, "traffic": None, "peak_source": psrc,
                     "kernel": "umma_gemm_kernel (tcgen05, bf16) over the ensemble's forward passes"},
        "e2e": {"value": Bq / e2e_s, "unit": "scenario-solves/s", "h2d_bytes_per_step": int(Xh.numel() * 4),
                "d2h_bytes_per_step": int(Mh.numel() * 4 + Sh.numel() * 4 + Fh.numel())},
        "solver_solves_per_s": solver_rate, "data_generation_s": gen_s,
        "fit_s": fit_s, "train_steps": n_train_steps,
        "train_tflops": 3 * 2.0 * 256 * n_train_steps * sum(k * m for k, m in zip(sur.dims[:-1], sur.dims[1:]))
                        / fit_s / 1e12,
        "final_train_loss": [h[-1] for h in hist],
        "test_mae_K": float(np.abs(mean_te[:, :P] - T[te]).mean()),
        "test_median_max_err_K": float(np.median(err_sur)),
        "test_max_err_K_surrogate_only": float(err_sur.max()),
        "spread_rule": {"accepted_fraction": float(raw_acc.mean()),
                        "accepted_with_err_above_tol": float(np.mean(err_sur[raw_acc] > args.sur_tol))
                        if raw_acc.any() else None,
                        "eval_fallback_fraction": float(fb_r.mean()),
                        "eval_accepted_max_err_K": float(err_r[~fb_r].max()) if (~fb_r).any() else None,
                        "eval_solve_with_fallback_s": info_r["seconds"],
                        "eval_effective_solves_per_s": (ev.stop - ev.start) / info_r["seconds"]},
        "calibrated": {"tau_K": tau, "coverage": args.sur_coverage, "calibration_accepted": cal_acc,
                       "calibration_tol_K": args.sur_tol * args.sur_cal_margin,
                       "eval_scenarios": int(ev.stop - ev.start), "fallback_fraction": float(fb.mean()),
                       "accepted_max_err_K": float(err_out[acc].max()) if acc.any() else None,
                       "accepted_with_err_above_tol": float(np.mean(err_out[acc] > args.sur_tol))
                       if acc.any() else None,
                       "answered_max_err_K": float(err_out.max()),
                       "solve_with_fallback_s": info["seconds"],
                       "effective_solves_per_s": (ev.stop - ev.start) / info["seconds"]},
        "speedup_vs_solver": (Bq / inf_s) / solver_rate,
        "training": f"{args.sur_epochs} epochs over the training scenarios augmented by the cube's {n_sym} "
                    f"reflections ({n_sym * n_train} rows), batch 256, Adam lr 1e-3"
                    + (f" decayed along a cosine to {args.sur_lr_end:g}" if args.sur_lr_end > 0 else "")
                    + ", each member from its own "
                    "seeded initialisation and permutations, members side by side (one CUDA graph per epoch)",
    }
    print(json.dumps(line))
    return 0

def run_surrogate_inference(args):
    """Kernel benchmark of the surrogate's inference path alone: the 5-member
    ensemble of [12, 512 x 5, 8192] MLPs with seeded He-initialised weights
    (throughput does not depend on the weight values), 4096 scenarios per
    inference, device-timed; the tcgen05 GEMMs' FLOP rate against the measured
    BF16 peak."""
    import torch

    from paper_2009_10400_b300 import surrogate
    from paper_2009_10400_b300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    P = args.sur_grid ** 3
    sur = surrogate.Surrogate(n_out=2 * P, width=512, depth=6, members=args.sur_members, max_batch=4096,
                              per_power=False)
    rng = np.random.default_rng(0)
    for k in range(args.sur_members):  # seeded He-normal weights (throughput does not depend on them)
        sur.engine.set_member_params(k, np.concatenate(
            [np.concatenate([rng.normal(0.0, np.sqrt(2.0 / K), N * K), np.zeros(N)])
             for K, N in zip(sur.dims[:-1], sur.dims[1:])]))
    dev = "cuda:0"
    Xd = torch.tensor(W.sample_scenarios(4096, seed=7), dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        sur.predict_device(Xd, P, args.sur_tol)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        sur.predict_device(Xd, P, args.sur_tol)
    ev1.record(stream)
    torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) * 1e-3 / args.steps
    flop = 2.0 * 4096 * args.sur_members * sum(k * m for k, m in zip(sur.dims[:-1], sur.dims[1:]))
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        psrc = "measured"
    except Exception:
        peak, psrc = 1800.0, "fallback"
    line = {"metric": "surrogate scenario-solves/s", "value": 4096 / sec, "unit": "scenario-solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * sec, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": f"surrogate inference: MLP {sur.dims}, {args.sur_members} members, batch 4096, "
                                   "seeded He-initialised weights"},
            "roofline": {"bound": "tensor", "achieved": flop / sec / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flop / sec / 1e12 / peak, "traffic": None, "peak_source": psrc,
                         "kernel": "umma_gemm_kernel (tcgen05) forward passes + ensemble_kernel"},
            "gpu_launches": args.steps * (args.sur_members * (1 + len(sur.dims) - 1) + 1)}
    print(json.dumps(line))
    return 0

def run_liver(args):
    """The paper's liver heating case (25 s of heating with three uniform
    spherical sources, temperature-dependent c and k, CEM43 tracked) from rest,
    device-timed: element-steps/s and simulated seconds per wall-clock second,
    with the 60 C isotherm volume, the damaged volume and the peak dose."""
    import torch

    from paper_2009_10400_b300 import tled
    from paper_2009_10400_b300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prob = W.liver_f2()
    s = tled.Solver.from_problem(prob, stream=stream)
    dt = s.get_dt()[0]
    n = int(round(prob.duration / dt))
    if args.liver_steps > 0:  # a shorter run (profiling)
        n = min(n, args.liver_steps)
    mode = "grid-resident" if s.grid_resident else "resident" if s.resident else "streamed"
    s.step(max(args.warmup, 3) * 32)  # graphs captured, caches warm
    s.sync()
    z3, z = np.zeros((prob.nn, 3)), np.zeros(prob.nn)
    s.set_state(z3, z3, np.full(prob.nn, prob.T0), z, None)  # back to rest, dose cleared
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        ev0.record(stream)
        s.step(n)
        ev1.record(stream)
        torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) * 1e-3
    s.sync()
    st = s.stats()
    cem = s.cem43()
    line = {"metric": "coupled element-steps/s", "value": prob.ne * n / sec, "unit": "element-steps/s",
            "n_gpus": 1, "steps": n, "warmup": max(args.warmup, 3) * 32, "ms_per_step": 1e3 * sec / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"liver_f2: synthetic ellipsoid, {prob.ne} T4, {prob.nn} nodes, 3 uniform "
                                   f"spheres D = 1 cm at 9.70536 MW/m^3, c(T), k(T), Q_m 33.8 kW/m^3, "
                                   f"{n * dt:g} s of heating at dt {dt:.3e} s", "cem43": True, "mode": mode},
            "simulated_s_per_wall_s": prob.duration / sec, "wall_s": sec,
            "T_max_C": st["T_max"], "ablation_volume_60C_cm3": 1e6 * s.isotherm_volume(60.0),
            "damaged_volume_cm3": 1e6 * st["damage_volume"], "cem43_max_min": float(cem.max()),
            "clocks": clk.summary(),
            # per graph chunk (32 steps, the rest as its binary digits): one step kernel (resident
            # modes) or a tile and a shared-node kernel per step (streamed), and the clock bump
            "gpu_launches": graph_chunks(n) * 2 if mode != "streamed" else n * 2 + graph_chunks(n)}
    print(json.dumps(line))
    return 0

def graph_chunks(n):
    """Graph launches of an n-step call: chunks of 32 steps, the rest as its binary digits."""
    return n // 32 + bin(n % 32).count("1")


def run_gpu(args):
    import torch

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_2009_10400_b300 import tled

    prob = make_problem(args.workload)
    stream = torch.cuda.current_stream()
    probes = probe_lattice(prob, args.probes)
    flags = tled.default_flags(prob) | (tled.GENERAL_H8 if args.general_h8 else 0)
    s = tled.Solver.from_problem(prob, device=local, stream=stream, probes=probes, flags=flags)
    brick = s.brick
    kernel_desc = ("resident (one CTA, K steps per launch)" if s.resident else
                   "grid-resident (one cooperative launch of K steps, one CTA per tile)" if s.grid_resident else
                   "streamed (tile + shared-node kernels)") + \
        ("; H8 brick instance: every element an axis-aligned brick, reference hourglass projections exactly zero"
         if s.brick else "; general H8 instance (TLED_GENERAL_H8)" if args.general_h8 else "")
    info = s.plan_info()
    l2_window = s.l2_window()
    dt = s.get_dt()[0]
    n_prony = len(prob.prony_g)

    # ---- warm-up (graphs captured here) and the device-timed region: K steps,
    #      inputs resident in HBM (larger than L2); clocks sampled throughout
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        s.step(args.warmup)
        s.sync()
        barrier(ws)
        torch.cuda.synchronize()
        clk.mark_start()
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    barrier(ws)
    s.sync()
    ms = ev0.elapsed_time(ev1)
    ms = reduce_max(ms, ws, f"cuda:{local}")
    value = ws * prob.ne * args.steps / (ms * 1e-3)
    if s.resident or s.grid_resident:  # one step kernel per graph chunk, and the clock bump
        gpu_launches = graph_chunks(args.steps) * 2
    else:  # a tile kernel and a shared-node kernel per step, and one clock bump per graph chunk
        gpu_launches = args.steps * (1 + (1 if info["n_shared"] > 0 else 0)) + graph_chunks(args.steps)

    # ---- roofline: the step's kernel pair per step over the timed region (CUDA events on the
    #      solver stream; the region holds K tile + shared-node launches and one clock bump per
    #      graph chunk); the split between the two kernels from launches timed one by one
    k_tile, k_sh = s.step_timed(args.roofline_steps)
    s.sync()
    per_step_kernel_ms = ms / args.steps
    alg = algorithmic_bytes(prob, n_prony)
    hbm, src = peaks()
    achieved = alg / (per_step_kernel_ms * 1e-3) / 1e9
    traffic = None if args.general_h8 else kernel_traffic(prob.name)  # the capture is of the brick instance

    # ---- end to end through the C ABI with host buffers, every step: the step's
    #      source settings from pinned host memory, one step, and the step's result
    #      (temperature and damage at the probe lattice) back to pinned host memory
    #      The read-back is pipelined: step i's probe values are copied into one of two
    #      pinned buffers behind step i + 1's launch, and the host waits for (and reads)
    #      step i's copy before it enqueues step i + 2's into the same buffer.
    n_e2e = args.e2e_steps
    src_host = torch.tensor(np.array(prob.sources), dtype=torch.float64).pin_memory()
    P_dev = torch.empty((2, len(probes)), dtype=torch.float64, device=f"cuda:{local}")
    P_host = [torch.empty((2, len(probes)), dtype=torch.float64).pin_memory() for _ in range(2)]
    ev = [torch.cuda.Event() for _ in range(2)]
    def e2e_loop(n):
        t_probe = 0.0
        for i in range(n + 1):
            if i < n:
                s.set_heat_sources(src_host.numpy())  # H2D: this step's source settings
                s.step(1)
                s.probes(out=P_dev)                   # probe temperatures and damage, on the device
                P_host[i % 2].copy_(P_dev, non_blocking=True)  # D2H into pinned memory
                ev[i % 2].record(stream)
            if i >= 1:
                ev[(i - 1) % 2].synchronize()         # step i - 1's result is on the host
                t_probe += float(P_host[(i - 1) % 2][0, 0])
        return t_probe

    with torch.cuda.stream(stream):  # untimed warm-up of the same loop (single-step graph, copies, events)
        e2e_loop(max(args.warmup, 50))
    barrier(ws)
    torch.cuda.synchronize()
    # the host loop keeps one step queued ahead of the device; a garbage-collection pause of
    # the interpreter inside the ~90 ms loop would idle the device (seen as 15 % outliers)
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e2e_loop(n_e2e)
        torch.cuda.synchronize()
        e2e_dt = time.perf_counter() - t0
    finally:
        gc.enable()
    e2e_s = reduce_max(e2e_dt, ws, f"cuda:{local}")
    e2e_value = ws * prob.ne * n_e2e / e2e_s
    s.sync()

    st = s.stats()
    s.close()
    del s
    torch.cuda.empty_cache()
    smalls = None if args.no_planning else small_configs(local, stream, args=args if rank == 0 and ws == 1 else None)
    precision = None
    if not args.no_precision and rank == 0 and prob.name.startswith("block_h8"):
        precision = precision_leg(args, local, stream)
    plan = None
    if not args.no_planning and prob.name.startswith("block_h8"):
        plan = planning_bench(args, local, stream)
        plan["scenario_solves_per_s"] = ws * plan["batched_solves_per_s"]
        if not args.no_cpu_baseline and rank == 0 and ws == 1:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-planning",
                                "--plan-scenarios", str(args.plan_scenarios)], capture_output=True, text=True, check=True)
            plan["cpu_oracle"] = json.loads(r.stdout.strip().splitlines()[-1])

    out = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            # the oracle on every host core (the headline baseline) and on one core, each in a
            # child process without torch (whose own OpenMP threads would compete for the cores)
            cpu = cpu_sample_subprocess(args, parallel=True)
            cpu["single_core"] = cpu_sample_subprocess(args, parallel=False)
        clocks = clk.summary()
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(prob),
            "plan": {"dt_s": dt, "tiles": info["n_tiles"], "shared_nodes": info["n_shared"],
                     "layout_bytes_per_step": layout_bytes(prob, n_prony, brick),
                     "accumulation": "float-float compensated u and T", "parallelism": f"replicas x{ws}",
                     "kernels": kernel_desc, "l2_persisting": l2_window},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": "tile_step_kernel + shared_step_kernel (one step)",
                         "algorithmic_bytes_per_step": alg,
                         "algorithmic_bytes_per_element_step": alg / prob.ne,
                         "layout_bytes_per_step": layout_bytes(prob, n_prony, brick),
                         "kernel_ms_per_step": per_step_kernel_ms,
                         "timing": "kernel_ms_per_step: the timed region's device time per step (graph "
                                   "replays of the tile and shared-node kernels, one clock bump per chunk); "
                                   "tile_kernel_ms, shared_kernel_ms: %d steps with each launch alone between "
                                   "CUDA events (outside graphs, so each includes its launch gap)"
                                   % args.roofline_steps,
                         "tile_kernel_ms": k_tile / args.roofline_steps,
                         "shared_kernel_ms": k_sh / args.roofline_steps,
                         "tile_share": k_tile / (k_tile + k_sh), "peak_source": src,
                         **({} if workload_config(prob)["l2"].startswith("inputs larger") else
                            {"note": "L2-resident working set: no HBM fraction is claimed for it"})},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(src_host.numel() * 8),
                    "d2h_bytes_per_step": int(P_host[0].numel() * 8), "steps": n_e2e,
                    "note": "every step: tled_set_heat_sources from pinned host, tled_step(1), tled_get_probes "
                            "(T and damage at a %d-point lattice) and its copy to pinned host; the host waits for "
                            "step i's copy while step i + 1 runs (two pinned buffers)" % len(probes)},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "precision": precision,
            "planning": plan,
            "small_configs": smalls,
            "final": {"T_max": st["T_max"], "u_max": st["u_max"], "status": st["status"]},
        }
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default="block_h8")
    ap.add_argument("--roofline-steps", type=int, default=50)
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--liver-steps", type=int, default=0, help="liver_f2: stop after this many steps (0: 25 s)")
    ap.add_argument("--probes", type=int, default=16)
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--ref-seconds", type=float, default=90.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-planning", action="store_true")
    ap.add_argument("--general-h8", action="store_true", help="keep the general H8 kernel on brick meshes")
    ap.add_argument("--plan-scenarios", type=int, default=256)
    ap.add_argument("--plan-subset", type=int, default=32)
    ap.add_argument("--sur-grid", type=int, default=16)
    ap.add_argument("--sur-scenarios", type=int, default=18000)
    ap.add_argument("--sur-test", type=int, default=2000)
    ap.add_argument("--sur-chunk", type=int, default=512)
    ap.add_argument("--sur-members", type=int, default=5)
    ap.add_argument("--sur-epochs", type=int, default=50)
    ap.add_argument("--sur-lr-end", type=float, default=1e-5, help="cosine learning-rate decay target (0: constant)")
    ap.add_argument("--sur-tol", type=float, default=1.0)
    ap.add_argument("--sur-coverage", type=float, default=1.0)
    ap.add_argument("--sur-cal-margin", type=float, default=0.8)
    ap.add_argument("--no-precision", action="store_true", help="skip the 32^3 long-run error leg")
    ap.add_argument("--oracle-trajectory", default=None, help=argparse.SUPPRESS)  # child of the precision leg
    ap.add_argument("--oracle-every", type=int, default=1000, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-dt", type=float, default=0.0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)  # child of the cpu_baseline leg
    ap.add_argument("--cpu-planning", action="store_true", help=argparse.SUPPRESS)  # child: planning CPU reference
    ap.add_argument("--cpu-parallel", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_trajectory:
        oracle_trajectory_child(args.workload, args.steps, args.oracle_every, args.oracle_dt, args.oracle_trajectory)
        return 0
    if args.cpu_planning:
        print(json.dumps(cpu_planning_sample(args.plan_scenarios, 8)))
        return 0
    if args.cpu_sample:
        print(json.dumps(cpu_oracle_sample(make_problem(args.workload), args.cpu_steps, seconds=args.cpu_seconds,
                                           warmup=3, parallel=args.cpu_parallel)))
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "liver_f2":
        return run_liver(args)
    if args.workload == "surrogate_inference":
        return run_surrogate_inference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
