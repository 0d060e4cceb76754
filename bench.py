#!/usr/bin/env python
"""Throughput of the SALE hydro cycle on GB300: cell-updates per second.

Default workload: Sedov-Taylor blast in the octant [0, 1.2]^3 at 384^3
cells (56.6M) on a node-jittered mesh (+-10% of the spacing, seed 2209),
gamma = 1.4, Lagrange step plus Eulerian remap every cycle.  One step = one
full cycle (Lagrangian step + rezone/advection + EoS + CFL dt) of the whole
mesh.  The state (>= 8 GB) is far larger than the 129 MB L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64]
    python bench.py --impl reference     # the CPU oracle on a bounded sample

Under torchrun each rank runs its own replica of the workload on its GPU
(the workload has no exchange step on one mesh per GPU): weak scaling,
value = all ranks' cell-updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/sec per full Lagrange+remap cycle, FP64 vs FP32-mixed; % HBM roofline"
UNIT = "cell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--precision", default="fp64", choices=("fp64",))
    ap.add_argument("--n", type=int, default=384, help="cells per axis")
    ap.add_argument("--jitter", type=float, default=0.1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=64)
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 vector peak: 2 DFMA per clock per SM x 152 SMs x 2.07 GHz x 2 flop.
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_rate(n, jitter, steps, warmup):
    """Cell-updates/s of the CPU oracle on an n^3 sample of the workload."""
    import oracle
    from paper_2209_01983_gb300 import inputs
    oracle.build()
    md, pd = inputs.sedov_octant(n, jitter=jitter)
    o = oracle.Oracle.from_problem(md, pd)
    o.run(max_cycles=warmup, remap_every=1)
    t0 = time.perf_counter()
    rc, done = o.run(max_cycles=steps, remap_every=1)
    dt = time.perf_counter() - t0
    if rc != 0 or done != steps:
        raise RuntimeError(f"oracle run failed: rc={rc} done={done}")
    return md.ncell * steps / dt, dt, md.ncell


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.cpu_sample_n
    rate, secs, ncell = oracle_rate(n, args.jitter, args.steps, args.warmup)
    sample = (f"Sedov octant {n}^3 ({ncell} cells), jitter {args.jitter}, ALE every cycle, "
              f"{args.steps} cycles after {args.warmup}; serial FP64 C oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, "fp64"),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, precision):
    return {"workload": f"sedov-octant-{args.n}^3-jitter{args.jitter}-ale-every-cycle",
            "cells": args.n ** 3, "gamma": 1.4, "remap_every": 1, "precision": precision,
            "l2": "state larger than the 129 MB L2 (no flush)", "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def gpu_arm(args):
    import numpy as np
    import torch

    from paper_2209_01983_gb300 import costs, inputs, sale

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    def barrier():
        if dist is not None:
            dist.barrier()

    precision = args.precision
    md, pd = inputs.sedov_octant(args.n, jitter=args.jitter)
    st = sale.State(md, pd, precision=sale.SALE_FP64, device=f"cuda:{local}")
    st.run_to_time(max_cycles=args.warmup, remap_every=1)

    # ---- timed region: K full cycles, graph replays on the state's stream
    st.profile(True)
    st.profile_read(reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)  # let the sampler take a first reading
    ev0.record(st.stream)
    done = st.run_to_time(max_cycles=args.steps, remap_every=1)
    ev1.record(st.stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    prof = st.profile_read(reset=True)
    st.profile(False)
    if done != args.steps:
        raise RuntimeError(f"ran {done} of {args.steps} cycles")
    ms = ev0.elapsed_time(ev1)
    d = st.diagnostics()

    t_max = ms
    if dist is not None:
        t = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = world * md.ncell * args.steps / (t_max * 1e-3)

    # ---- roofline of the dominant kernel
    table = costs.table(precision, "ale")
    kern = {k: v for k, v in prof.items() if v[1] > 0}
    total_ms = sum(v[0] for v in kern.values())
    missing = [k for k in kern if k not in table]
    if missing:
        raise RuntimeError(f"no cost entry for kernels {missing}")
    top = max(kern, key=lambda k: kern[k][0])
    unit, bytes_u, flops_u = table[top]
    units = md.ncell if unit == "cell" else md.nnode
    avg_s = kern[top][0] / kern[top][1] * 1e-3
    peaks, peak_src = load_peaks()
    if precision == "fp64":
        achieved = flops_u * units / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": top,
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (FP64 vector pipe)",
                "hbm_achieved_gbs": bytes_u * units / avg_s / 1e9,
                "hbm_frac_of_measured": bytes_u * units / avg_s / 1e9 / peaks["hbm_gbs"]}
    def per_kernel(k, v):
        u_, b_, f_ = table[k]
        nunit = md.ncell if u_ == "cell" else md.nnode
        sec = v[0] / v[1] * 1e-3
        return {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / total_ms,
                "alg_gbs": b_ * nunit / sec / 1e9, "alg_tflops": f_ * nunit / sec / 1e12}
    kernels = {k: per_kernel(k, v) for k, v in sorted(kern.items(), key=lambda kv: -kv[1][0])}
    launches = sum(v[1] for v in kern.values())
    cycle_bytes = sum(table[k][1] * (md.ncell if table[k][0] == "cell" else md.nnode) for k in kern)
    cycle_flops = sum(table[k][2] * (md.ncell if table[k][0] == "cell" else md.nnode) for k in kern)
    full = {"cycle_algorithmic_bytes": cycle_bytes, "cycle_algorithmic_flops": cycle_flops,
            "cycle_tflops": cycle_flops * args.steps / (ms * 1e-3) / 1e12,
            "cycle_hbm_gbs": cycle_bytes * args.steps / (ms * 1e-3) / 1e9,
            "cycle_hbm_frac_of_measured": cycle_bytes * args.steps / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        names = ("u", "v", "w", "mn", "m", "e")
        host = {nm: torch.from_numpy(st.field(nm)).pin_memory() for nm in names}
        h2d = sum(t.numel() * 8 for t in host.values())
        d2h = 8 * 8 + 128  # diagnostics sums + device scalars
        e2e_steps = max(1, min(args.steps, 5))
        dd = sale.sale_diag()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for nm, t in host.items():
                sale.check(sale.sale_set_field(st._h, nm.encode(),
                                               sale.C.cast(t.data_ptr(), sale._dp), t.numel()))
            sale.check(sale.sale_refresh(st._h))
            sale.check(sale.sale_run_to_time(st._h, math.inf, 1, 1, None))
            sale.check(sale.sale_diagnostics(st._h, sale.C.byref(dd)))
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * md.ncell * e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        n = args.cpu_sample_n
        rate, secs, ncell = oracle_rate(n, args.jitter, 40, 5)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"same workload at {n}^3 ({ncell} cells), 40 cycles after 5, "
                         f"serial FP64 C oracle, {secs:.1f} s"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, precision),
        "roofline": roof, "full_cycle": full, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk, "kernels": kernels,
        "check": {"t": d["t"], "cycle": d["cycle"], "status": d["status"]},
        "peaks": {"hbm_gbs": peaks["hbm_gbs"], "source": peak_src},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
