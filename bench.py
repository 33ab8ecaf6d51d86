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
    if workload.startswith("block_h8_"):
        return W.block_h8(n=int(workload.split("_")[-1]))
    raise SystemExit(f"unknown workload {workload}")


def algorithmic_bytes(prob, n_prony):
    """Bytes the method must move per step in this library's layout: every
    element constant once, the Prony state read and written, and every nodal
    state array read and written once (see the design notes)."""
    npe = prob.npe
    elem = 2 * npe + 9 * 4 + 4 + 2 * 4 * 6 * n_prony  # local conn, J0^-1, V0, Prony R+W
    if prob.per_element:
        elem += 6 * 4  # mu, kappa, k1, k2, k, alpha
        if not np.allclose(prob.a0, prob.a0[0]):
            elem += 3 * 4  # fibres
    node = 5 * 16 + 3 * 16  # read u_hi/theta, X0/V, lo, v/Omega, m/C/mask; write hi, lo, v/Omega
    return elem * prob.ne + node * prob.nn


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


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


def cpu_oracle_sample(prob, steps, threads_note="1 (single-threaded C)"):
    """Time the FP64 oracle as it stands on a bounded sample of the workload."""
    import oracle

    t0 = time.perf_counter()
    m = oracle.OracleModel(prob)
    setup = time.perf_counter() - t0
    s = m.init_state()
    m.step(s, 1)  # warm caches
    t0 = time.perf_counter()
    m.step(s, steps)
    el = time.perf_counter() - t0
    return {"value": prob.ne * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{prob.name}: {steps} steps after 1 warm-up step ({el:.1f} s, setup {setup:.1f} s), "
                      f"FP64 C oracle, threads {threads_note}"}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    prob = make_problem(args.workload)
    steps = max(1, args.ref_steps)
    r = cpu_oracle_sample(prob, steps * max(1, args.steps) // max(1, args.steps))
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 0, "steps": steps,
            "warmup": 1, "ms_per_step": 1e3 * prob.ne / r["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": prob.name, "elements": prob.ne, "nodes": prob.nn},
            "cpu_baseline": r, "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


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
    s = tled.Solver.from_problem(prob, device=local, stream=stream)
    info = s.plan_info()
    dt = s.get_dt()[0]
    n_prony = len(prob.prony_g)

    # ---- warm-up (graphs captured here)
    s.step(args.warmup)
    s.sync()

    # ---- device-timed region: K steps, inputs resident in HBM (larger than L2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    s.sync()
    ms = ev0.elapsed_time(ev1)
    ms = reduce_max(ms, ws, f"cuda:{local}")
    value = ws * prob.ne * args.steps / (ms * 1e-3)
    launches_per_step = 1 + (1 if info["n_shared"] > 0 else 0)
    gpu_launches = args.steps * launches_per_step + (args.steps + 31) // 32

    # ---- live per-kernel timing for the roofline (CUDA events on the launching stream)
    k_tile, k_sh = s.step_timed(args.roofline_steps)
    s.sync()
    per_step_kernel_ms = (k_tile + k_sh) / args.roofline_steps
    alg = algorithmic_bytes(prob, n_prony)
    hbm, src = peaks()
    achieved = alg / (per_step_kernel_ms * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            traffic = json.load(open(tr_path)).get(prob.name)
        except Exception:
            traffic = None

    # ---- end to end through the C ABI with host buffers
    chunk = args.e2e_chunk
    n_calls = max(1, args.steps // chunk)
    T_host = torch.empty(prob.nn, dtype=torch.float64).pin_memory()
    D_host = torch.empty(prob.nn, dtype=torch.float64).pin_memory()
    src_rows = np.array(prob.sources)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n_calls):
        s.set_heat_sources(src_rows)          # H2D: this call's source settings
        s.step(chunk)
        s.temperature(out=T_host)             # D2H: temperature field (synchronises)
        s.damage(out=D_host)                  # D2H: damage field
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, ws, f"cuda:{local}")
    e2e_value = ws * prob.ne * chunk * n_calls / e2e_s
    s.sync()

    out = None
    if rank == 0:
        st = s.stats()
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            from paper_2009_10400_b300 import workloads as W

            cpu = cpu_oracle_sample(prob, args.cpu_steps)
        clocks = clk.summary()
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": prob.name, "elements": prob.ne, "nodes": prob.nn,
                       "element": "H8" if prob.npe == 8 else "T4", "dt_s": dt,
                       "tiles": info["n_tiles"], "shared_nodes": info["n_shared"],
                       "l2": "inputs larger than L2 (state + element data ~%.0f MB per step)" % (alg / 1e6),
                       "accumulation": "float-float compensated u and T", "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": "tile_step_kernel + shared_step_kernel (one step)",
                         "algorithmic_bytes_per_step": alg,
                         "kernel_ms_per_step": per_step_kernel_ms,
                         "tile_kernel_ms": k_tile / args.roofline_steps,
                         "shared_kernel_ms": k_sh / args.roofline_steps, "peak_source": src},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(src_rows.size * 8),
                    "d2h_bytes_per_step": int(2 * 8 * prob.nn), "steps_per_call": chunk,
                    "note": "per call: set_heat_sources from host, step(%d), temperature and damage to pinned host"
                            % chunk},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
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
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default="block_h8")
    ap.add_argument("--roofline-steps", type=int, default=50)
    ap.add_argument("--e2e-chunk", type=int, default=50)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--ref-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
