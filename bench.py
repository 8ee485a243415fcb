#!/usr/bin/env python3
"""Benchmark of the GB300 particle-SMC path: SMC particle-steps/s.

One step = one complete SMC run of the workload (every checkpoint segment:
propagation, FP64 normaliser and scan, systematic resampling, gather, and
the outputs log Z / final log-weights / last ancestors / final states).
A particle-step is one particle advancing one checkpoint segment,
including its share of resampling.

Default workload (one GPU): the constant-rate birth-death model of
Listing 1 on a seeded 64-tip Yule tree of height 1, Gamma(1,1) /
Gamma(1,0.5) priors, N = 2^16 particles, FP64, 127 checkpoints.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload crbd64|lg|rateshift256]

With N > 1 (launched by torch.distributed.run) every rank runs its own
independent replica with a rank-specific seed (runs do not exchange data,
so there is no collective on the data path; scaling is weak).  Rank 0 prints
one JSON line.  `--impl reference` times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

import inputs  # noqa: E402

METRIC = "SMC particle-steps/s at fixed log-Z error vs plain GPU path; p50/p99 latency"
UNIT = "particle-steps/s"

WORKLOADS = {
    # Listing 1 CRBD, 64-tip Yule tree (seed 2), N = 2^16, FP64
    "crbd64": dict(kind="crbd", tips=64, tree_seed=2, N=1 << 16, precision="fp64"),
    # linear-Gaussian, T = 50 observations (seed 1), N = 1024, FP64
    "lg": dict(kind="lg", T=50, obs_seed=1, N=1024, precision="fp64"),
    # rate-shift, 256-tip Yule tree (seed 3), N = 2^20, FP32 particles / FP64 reductions
    "rateshift256": dict(kind="rateshift", tips=256, tree_seed=3, N=1 << 20, precision="fp32",
                         sigma=0.3),
}

# FP64 operations the step kernel executes per particle-step (2 x DFMA + DADD +
# DMUL from one ncu capture of the crbd64 workload; see the profiles folder).
FP64_FLOP_PER_PSTEP = {"crbd64": None}
# Per-launch DRAM traffic of the step kernel from the same capture, valid only
# for the kernel sources with this digest.
NCU_TRAFFIC = {"crbd64": dict(bytes_per_launch=None, src_digest=None)}

# 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM (2 DFMA) = the 1.25 TFLOP/s FP64 rate of GB300
FP64_PEAK_FLOPS = 152 * 2070e6 * 4


def src_digest() -> str:
    h = hashlib.sha256()
    for p in sorted((ROOT / "paper_2112_00364_gb300" / "csrc").glob("*")):
        h.update(p.read_bytes())
    return h.hexdigest()[:16]


def setup_inputs(w: dict):
    if w["kind"] == "lg":
        obs = inputs.lg_observations(w["T"], seed=w["obs_seed"])
        return dict(obs=obs), w["T"]
    tree = inputs.yule_tree(w["tips"], seed=w["tree_seed"])
    p = dict(tree=tree)
    if w["kind"] == "rateshift":
        p.update(sigma=w["sigma"], lam_stack_cap=tree.max_pending_right() + 1)
    return p, tree.n_nodes


def input_bytes(params: dict) -> int:
    if "obs" in params:
        return params["obs"].nbytes
    t = params["tree"]
    return 4 * 4 * t.n_nodes + 8 * t.n_nodes


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines: list[str] = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_throughput(w: dict, params: dict, n_seg: int, budget_s: float, n_particles: int,
                      max_runs: int = 50):
    """Time the CPU oracle on the host: full runs with seeds 1, 2, ... until
    `budget_s` seconds of work (at least one run)."""
    import oracle

    prec = oracle.FP64 if w["precision"] == "fp64" else oracle.FP32
    runs, t_tot = 0, 0.0
    while runs < max_runs and (runs == 0 or t_tot < budget_s):
        t0 = time.perf_counter()
        r = oracle.smc_run(w["kind"], n_particles, seed=runs + 1, precision=prec, **params)
        t_tot += time.perf_counter() - t0
        if r["status"] < 0:
            raise RuntimeError(f"oracle status {r['status']}")
        runs += 1
    return runs * n_particles * n_seg / t_tot, runs, t_tot


def run_reference(args, w, params, n_seg):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_sample = min(w["N"], 1 << 14)
    import oracle

    prec = oracle.FP64 if w["precision"] == "fp64" else oracle.FP32
    for s in range(args.warmup):
        oracle.smc_run(w["kind"], n_sample, seed=1000 + s, precision=prec, **params)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.smc_run(w["kind"], n_sample, seed=1 + s, precision=prec, **params)
        times.append(time.perf_counter() - t0)
        assert r["status"] >= 0
    total = sum(times)
    value = args.steps * n_sample * n_seg / total
    sample = (f"{args.steps} oracle runs of the {args.workload} workload with N={n_sample} "
              f"particles (of {w['N']}), {n_seg} checkpoints each, single-threaded")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if w["precision"] == "fp64" else "f32+f64", "data": "synthetic",
        "config": workload_config(args.workload, w, n_seg),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(name: str, w: dict, n_seg: int) -> dict:
    cfg = {"workload": name, "n_particles": w["N"], "checkpoints": n_seg,
           "precision": w["precision"], "l2": "flushed between timed steps (512 MiB write)",
           "parallelism": "replicas (one independent run per GPU)"}
    if w["kind"] == "lg":
        cfg.update(model="linear-Gaussian SSM x_t=0.9x+N(0,1), y~N(x,0.5^2)",
                   observations=f"T={w['T']} simulated, seed {w['obs_seed']}")
    else:
        cfg.update(model="CRBD (Listing 1), priors Gamma(1,1), Gamma(1,0.5), rho=1"
                   if w["kind"] == "crbd" else "rate-shift CRBD, lognormal multipliers sigma=0.3",
                   tree=f"Yule {w['tips']} tips seed {w['tree_seed']}, height 1.0")
    return cfg


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="crbd64", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    params, n_seg = setup_inputs(w)
    if args.impl == "reference":
        return run_reference(args, w, params, n_seg)

    import torch

    from paper_2112_00364_gb300 import smc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    N = w["N"]
    stream = torch.cuda.Stream()
    model = smc.Model(w["kind"], **params)
    outs = {
        "log_z": torch.zeros(1, dtype=torch.float64, device=dev),
        "final_logw": torch.zeros(N, dtype=torch.float64, device=dev),
        "ancestors": torch.zeros((1, N), dtype=torch.int32, device=dev),
        "int_fields": torch.zeros((model.n_int, N), dtype=torch.int32, device=dev),
    }
    if model.n_real:
        outs["real_fields"] = torch.zeros((model.n_real, N), dtype=torch.float64, device=dev)
    if model.stack_cap:
        outs["stack"] = torch.zeros((model.stack_cap, N), dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    seed0 = 1 + 100000 * rank

    def one(seed, timed_kernels):
        return smc.run(model, N, seed=seed, precision=w["precision"], where="device",
                       stream=stream, outputs=outs, time_kernels=timed_kernels)

    for s in range(args.warmup):
        one(seed0 + 50000 + s, False)
    torch.cuda.synchronize()
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms, kern_launches, logz = [], 0.0, 0, []
    statuses = []
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = one(seed0 + s, True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms += r["kernel_ms"]
        kern_launches += r["kernel_launches"]
        statuses.append(r["status"])
        logz.append(float(outs["log_z"].cpu()[0]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units_per_step = N * n_seg
    value = args.steps * units_per_step * ws / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # end to end through the public API: host inputs in, host results out
    h2d = input_bytes(params)
    pinned = {
        "log_z": torch.zeros(1, dtype=torch.float64).pin_memory(),
        "final_logw": torch.zeros(N, dtype=torch.float64).pin_memory(),
        "ancestors": torch.zeros((1, N), dtype=torch.int32).pin_memory(),
        "int_fields": torch.zeros((model.n_int, N), dtype=torch.int32).pin_memory(),
    }
    if model.n_real:
        pinned["real_fields"] = torch.zeros((model.n_real, N), dtype=torch.float64).pin_memory()
    if model.stack_cap:
        pinned["stack"] = torch.zeros((model.stack_cap, N), dtype=torch.float64).pin_memory()
    d2h = sum(t.numel() * t.element_size() for t in pinned.values())
    e2e_s = []
    for s in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = smc.Model(w["kind"], **params)
        smc.run(m2, N, seed=seed0 + s, precision=w["precision"], where="host", stream=stream,
                outputs=pinned)
        m2.close()
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_s)
    if dist:
        t = torch.tensor([e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = args.steps * units_per_step * ws / e2e_total

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    avg_launch_s = (kern_ms / kern_launches) * 1e-3 if kern_launches else None
    flop = FP64_FLOP_PER_PSTEP.get(args.workload)
    roof = None
    if avg_launch_s and flop:
        achieved = flop * N / avg_launch_s
        tr = NCU_TRAFFIC.get(args.workload, {})
        traffic = tr.get("bytes_per_launch") if tr.get("src_digest") == src_digest() else None
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_FLOPS, "traffic": traffic,
                "kernel": "step_kernel (fused segment kernel)",
                "avg_launch_us": avg_launch_s * 1e6, "launches": kern_launches,
                "peak_source": "derived: 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM"}
    cpu = None
    if ws == 1:
        v, runs, secs = oracle_throughput(w, params, n_seg, args.cpu_seconds, N)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{runs} full oracle runs of the workload (N={N}, seeds 1..{runs}), "
                         f"{secs:.1f} s single-threaded"}
    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if w["precision"] == "fp64" else "f32+f64", "data": "synthetic",
        "config": workload_config(args.workload, w, n_seg),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "log_z": {"mean": float(np.mean(logz)), "sd": float(np.std(logz))},
        "status": sorted(set(statuses)),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * (n_seg + 1),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
