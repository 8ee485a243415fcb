#!/usr/bin/env python3
"""Benchmark of the GB300 particle-SMC path: SMC particle-steps/s.

A particle-step is one particle advancing one checkpoint segment, including
its share of resampling.  One benchmark step is one complete piece of work:

  crbd64        one SMC run of the constant-rate birth-death model (Listing 1)
                on a seeded 64-tip Yule tree of height 1, Gamma(1,1) /
                Gamma(1,0.5) priors, N = 2^16, FP64, 127 checkpoints (default);
  lg            one run of the linear-Gaussian model, T = 50, N = 1024, FP64;
  rateshift256  one run of the rate-shift model on a 256-tip tree, N = 2^20,
                FP32 particles with FP64 reductions;
  batch512      one batched launch sequence of 512 independent runs (half
                linear-Gaussian with T log-uniform in 20..500, half CRBD with
                tips log-uniform in 16..256, N log-uniform in 256..65536),
                FP32 particles with FP64 reductions; the line also carries the
                same 512 runs timed one run per launch;
  serve2000     one second of a Poisson request stream (mean 2000 requests/s,
                request sizes drawn from the batch512 mix) served by the
                continuous-batching server, from the first submission to the
                last result on the host; p50/p99 request latency, beside the
                first requests of the stream served one run per launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload crbd64|lg|rateshift256|batch512|serve2000]

With N > 1 (launched by torch.distributed.run) every rank runs its own
independent replica with rank-specific seeds (runs exchange no data, so there
is no collective on the data path; scaling is weak).  Rank 0 prints one JSON
line.  `--impl reference` times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
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
    "crbd64": dict(kind="crbd", tips=64, tree_seed=2, N=1 << 16, precision="fp64"),
    "lg": dict(kind="lg", T=50, obs_seed=1, N=1024, precision="fp64"),
    # the same run with FP32 particles (the batched and served configurations' precision)
    "lg_fp32": dict(kind="lg", T=50, obs_seed=1, N=1024, precision="fp32"),
    # a small CRBD run (16 tiles of 32 particles), FP32 particles
    "crbd_small": dict(kind="crbd", tips=32, tree_seed=2, N=512, precision="fp32"),
    # the vector-borne disease SEIR model (Section 6.2), 26 weeks of synthetic reports
    "seir182": dict(kind="seir", days=182, obs_seed=7, N=1 << 16, precision="fp64"),
    # CRBD with static delayed sampling and ESS-triggered resampling (Section 6.3),
    # on a synthetic 128-tip tree standing in for the paper's larger phylogeny
    "crbd_ds128": dict(kind="crbd_ds", tips=128, tree_seed=6, N=100_000, precision="fp64",
                       ess=0.5),
    "rateshift256": dict(kind="rateshift", tips=256, tree_seed=3, N=1 << 20, precision="fp32",
                         sigma=0.3),
    "batch512": dict(kind="batch", n_runs=512, spec_seed=4, precision="fp32"),
    "serve2000": dict(kind="serve", n_runs=512, spec_seed=4, precision="fp32", rate=2000.0,
                      seconds_per_step=1.0, arrival_seed=5),
    # the standalone resampling steps (normaliser, scan, systematic search) and
    # the gather of a 2-field FP64 state, on a population larger than L2
    "resample24": dict(kind="resample", N=1 << 24, fields=2, logw_seed=24, logw_scale=2.0,
                       precision="fp64"),
}

HBM_PEAK_GBS = 6800.0  # fallback HBM bandwidth when MEASURED_PEAKS.json is absent
RS_BYTES = 20          # logw read twice (normaliser, scan) + ancestor written, per particle

# Per particle-step counts of the segment kernel from one ncu capture of the
# workload (profiles folder): warp instructions issued, FP64 flop (2 x DFMA +
# DADD + DMUL), DRAM traffic per launch and the FP64 pipe's busy fraction.  The
# roofline basis is the unit that bounds the kernel: instruction issue for the
# plain CRBD (latency-bound, most arithmetic on the integer pipes), the FP64
# rate for the delayed-sampling CRBD (FP64 pipe busy 36-44% of a launch).  The
# traffic holds only for the kernel sources with the recorded digest.
NCU = {"crbd64": dict(basis="issue", warp_inst_per_pstep=113.9, fp64_flop_per_pstep=18.8,
                      bytes_per_launch=2.963e6, fp64_pipe_elapsed=0.185,
                      src_digest="fc844398542168c5"),
       "crbd_ds128": dict(basis="fp64", warp_inst_per_pstep=110.2, fp64_flop_per_pstep=169.1,
                          bytes_per_launch=4.953e6, fp64_pipe_elapsed=0.353,
                          src_digest="fc844398542168c5"),
       # FP32 waves of 2^20 particles: bound by memory latency (long-scoreboard
       # stalls), reported against HBM; 72-75 warp instructions per particle-step
       "rateshift256": dict(basis="hbm", warp_inst_per_pstep=73.5, bytes_per_launch=1.182e8,
                            src_digest="fc844398542168c5")}

# 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM (2 DFMA/clk/SM) = GB300's FP64 rate
FP64_PEAK_FLOPS = 152 * 2070e6 * 4
# 152 SMs x 4 schedulers x 2070 MHz, one warp instruction per scheduler per clock
ISSUE_PEAK = 152 * 4 * 2070e6
# the compute-peak probe's steps per chain (about 5-20 ms a launch on GB300)
PROBE_ITERS = {0: 2000, 1: 100000, 2: 20000, 3: 50000, 4: 5000}


# the segment kernel's sources (the standalone resampling kernels are not among them)
KERNEL_SOURCES = ("smc_engine.cu", "smc_step.cuh", "smc_waves_kind.cu", "smc_engine.h",
                  "smc_models.cuh", "smc_device.cuh", "smc_combine.cuh")
# the standalone resampling kernels' sources
RS_SOURCES = ("smc_prims.cu", "smc_device.cuh", "smc_combine.cuh")

# DRAM traffic of one smc_resample call at 2^24 (the three kernels' dram__bytes
# read + write in one ncu capture, profiles folder), valid for the sources with
# the recorded digest.
RS_NCU = dict(bytes_per_call=2.353e8, src_digest="84e4a804f220f1c5")


def code_text(src: str) -> str:
    """A CUDA/C++ source without its comments and blank space, so that the digest
    changes with the code and not with its documentation (string literals in
    these files hold no comment markers)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


# Files that hold device and host code: only the part before the marker holds
# what the segment kernel executes (the kernels and the structures they read).
DEVICE_PART = {"smc_engine.cu": "// host side", "smc_engine.h": "struct Layout {"}


def device_part(name: str, text: str) -> str:
    mark = DEVICE_PART.get(name)
    if mark and mark in text:
        return text[: text.index(mark)]
    return text


def src_digest(sources=KERNEL_SOURCES, read=None) -> str:
    """Digest of the device code (comments and blank space stripped) of the sources."""
    read = read or (lambda name: (ROOT / "paper_2112_00364_gb300" / "csrc" / name).read_text())
    h = hashlib.sha256()
    for name in sources:
        h.update(code_text(device_part(name, read(name))).encode())
    return h.hexdigest()[:16]


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
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_rate(units_per_rank: float, seconds: float, dist=None, device="cpu") -> tuple:
    """Whole-job rate of independent replicas: every rank processed
    `units_per_rank` units; the job took as long as its slowest rank.  Returns
    (units of all ranks / slowest time, slowest time)."""
    ws = 1
    if dist is not None:
        import torch

        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds, ws = float(t.item()), dist.get_world_size()
    return units_per_rank * ws / seconds, seconds


# ------------------------------------------------------------------ workloads
class Work:
    """One workload: a list of runs (kind, params, N, seed, run_id)."""

    def __init__(self, name: str, seed_base: int):
        w = WORKLOADS[name]
        self.name, self.w, self.precision = name, w, w["precision"]
        self.runs = []
        if w["kind"] == "resample":
            self.units = w["N"]
            return
        if w["kind"] in ("batch", "serve"):
            for q, sp in enumerate(inputs.batch_specs(w["n_runs"], seed=w["spec_seed"])):
                if sp.kind == "lg":
                    p = dict(obs=inputs.lg_observations(sp.T, seed=sp.obs_seed))
                else:
                    p = dict(tree=inputs.yule_tree(sp.tips, seed=sp.tree_seed))
                self.runs.append(dict(kind=sp.kind, params=p, N=sp.n_particles,
                                      seed=seed_base + sp.seed, run_id=q,
                                      segments=sp.n_segments()))
        else:
            if w["kind"] == "lg":
                p = dict(obs=inputs.lg_observations(w["T"], seed=w["obs_seed"]))
                seg = w["T"]
            elif w["kind"] == "seir":
                p = dict(obs=inputs.seir_observations(w["days"], seed=w["obs_seed"]))
                seg = w["days"]
            else:
                tree = inputs.yule_tree(w["tips"], seed=w["tree_seed"])
                p = dict(tree=tree)
                if w["kind"] == "rateshift":
                    p.update(sigma=w["sigma"], lam_stack_cap=tree.max_pending_right() + 1)
                seg = tree.n_nodes
            self.runs.append(dict(kind=w["kind"], params=p, N=w["N"], seed=seed_base, run_id=0,
                                  segments=seg, ess=w.get("ess", 0.0)))
        self.units = sum(r["N"] * r["segments"] for r in self.runs)

    def config(self) -> dict:
        w = self.w
        cfg = {"workload": self.name, "precision": self.precision,
               "l2": "flushed between timed steps (512 MiB write)",
               "parallelism": "replicas (one independent workload per GPU)",
               "particle_steps_per_step": self.units}
        if w["kind"] == "resample":
            cfg.pop("particle_steps_per_step")
            cfg.update(n_particles=w["N"], state_fields=w["fields"],
                       step="smc_resample (FP64 normaliser, scan, systematic search) + smc_gather "
                            "of a 2-field f64 state",
                       logw=f"normal(0, {w['logw_scale']}) seed {w['logw_seed']}",
                       l2="inputs (384 MiB) larger than L2; L2 also flushed between steps")
            return cfg
        if w["kind"] == "serve":
            cfg.update(arrivals=f"Poisson, mean {w['rate']:.0f} requests/s, seed {w['arrival_seed']}+step",
                       stream_seconds_per_step=w["seconds_per_step"],
                       mix="request sizes drawn from the batch512 runs (spec seed 4)")
            cfg.pop("particle_steps_per_step")
        elif w["kind"] == "batch":
            cfg.update(runs=w["n_runs"], n_particles_total=sum(r["N"] for r in self.runs),
                       mix="half linear-Gaussian (T log-uniform 20..500), half CRBD (tips "
                           "log-uniform 16..256), N log-uniform 256..65536, seeded (spec seed 4)")
        elif w["kind"] == "seir":
            cfg.update(model="vector-borne disease SEIR (Listing 2), 7370 humans, Beta priors",
                       n_particles=w["N"], checkpoints=w["days"],
                       observations=f"{w['days']} days, weekly synthetic reports, seed {w['obs_seed']}")
        elif w["kind"] == "lg":
            cfg.update(model="linear-Gaussian SSM x_t=0.9x+N(0,1), y~N(x,0.5^2)",
                       n_particles=w["N"], checkpoints=w["T"],
                       observations=f"T={w['T']} simulated, seed {w['obs_seed']}")
        elif w["kind"] == "crbd_ds":
            cfg.update(model="CRBD (Listing 1) with lambda, mu integrated out (static delayed "
                             "sampling), priors Gamma(1,1), Gamma(1,0.5), rho=1",
                       n_particles=w["N"], checkpoints=self.runs[0]["segments"],
                       resampling=f"ESS-triggered, threshold {w['ess']} N",
                       tree=f"Yule {w['tips']} tips seed {w['tree_seed']}, height 1.0")
        else:
            cfg.update(model="CRBD (Listing 1), priors Gamma(1,1), Gamma(1,0.5), rho=1"
                       if w["kind"] == "crbd" else "rate-shift CRBD, lognormal multipliers sigma=0.3",
                       n_particles=w["N"], checkpoints=self.runs[0]["segments"],
                       tree=f"Yule {w['tips']} tips seed {w['tree_seed']}, height 1.0")
        return cfg

    def input_bytes(self) -> int:
        tot = 0
        for r in self.runs:
            p = r["params"]
            tot += p["obs"].nbytes if "obs" in p else 24 * p["tree"].n_nodes
        return tot


def oracle_throughput(work: Work, budget_s: float, max_runs: int, n_particles=None):
    """Time the CPU oracle on the host: the workload's runs in order (cycling),
    until `budget_s` seconds of work (at least one run)."""
    import oracle

    prec = oracle.FP64 if work.precision == "fp64" else oracle.FP32
    runs, t_tot, units = 0, 0.0, 0
    while runs < max_runs and (runs == 0 or t_tot < budget_s):
        r = work.runs[runs % len(work.runs)]
        N = n_particles or r["N"]
        t0 = time.perf_counter()
        o = oracle.smc_run(r["kind"], N, seed=r["seed"] + runs // len(work.runs), run_id=r["run_id"],
                           precision=prec, ess_threshold=r.get("ess", 0.0), **r["params"])
        t_tot += time.perf_counter() - t0
        if o["status"] < 0:
            raise RuntimeError(f"oracle status {o['status']}")
        units += N * r["segments"]
        runs += 1
    return units / t_tot, runs, t_tot, units


def equal_error_comparison(work: Work, smc, torch, stream, n_seeds: int = 16) -> dict:
    """Delayed sampling against the plain model at equal log-Z error (untimed
    by the bench's clock): the same tree, N and resampling rule run through the
    plain CRBD and the delayed-sampling CRBD for n_seeds seeds each; the log-Z
    standard deviations give the variance ratio, i.e. how many more particles
    the plain model needs for the same log-Z error (variance ~ 1/N), and the
    CUDA-event times give each model's particle-steps/s."""
    r = work.runs[0]
    out = {}
    for kind in ("crbd_ds", "crbd"):
        m = smc.Model(kind, **r["params"])
        lz, ms = [], 0.0
        for s in range(n_seeds):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = smc.run(m, r["N"], seed=70000 + s, run_id=0, precision=work.precision,
                          where="device", stream=stream, ess_threshold=r.get("ess", 0.0))
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            lz.append(float(res["log_z"].cpu()[0]))
        m.close()
        out[kind] = {"value": n_seeds * r["N"] * r["segments"] / (ms * 1e-3), "unit": UNIT,
                     "log_z_mean": float(np.mean(lz)), "log_z_sd": float(np.std(lz, ddof=1))}
    ratio = (out["crbd"]["log_z_sd"] / out["crbd_ds"]["log_z_sd"]) ** 2
    return {"seeds": n_seeds, "delayed_sampling": out["crbd_ds"], "plain_crbd": out["crbd"],
            "variance_ratio_plain_over_delayed": ratio,
            "delayed_value_at_plain_error": out["crbd_ds"]["value"] * ratio}


def run_reference(args, work: Work):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if work.w["kind"] == "resample":
        return run_reference_resample(args, work, ws)
    batch = work.w["kind"] in ("batch", "serve")
    n_sample = None if batch else min(work.runs[0]["N"], 1 << 14)
    max_runs = 32 if batch else 1
    for _ in range(args.warmup):
        oracle_throughput(work, 0.0, 1, n_sample)
    times, units = [], 0
    for _ in range(args.steps):
        v, runs, secs, u = oracle_throughput(work, 0.0 if not batch else 1e9, max_runs, n_sample)
        times.append(secs)
        units += u
    total = sum(times)
    value = units / total
    if batch:
        sample = (f"each step: the first {max_runs} of the 512 runs of the batch, run one after "
                  f"another by the single-threaded oracle")
    else:
        sample = (f"each step: one oracle run of the {args.workload} workload with N={n_sample} "
                  f"particles (of {work.runs[0]['N']}), single-threaded")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if work.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": work.config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_resample(args, work: Work, ws: int) -> int:
    """The oracle's systematic resampling on the host, a 2^20-particle sample per step."""
    import oracle

    w = work.w
    n_s = 1 << 20
    lw = inputs.random_logw(w["N"], seed=w["logw_seed"], scale=w["logw_scale"])[:n_s]
    for _ in range(args.warmup):
        oracle.resample(lw, 0.5)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.resample(lw, (k + 0.5) / (args.steps + 1))
    secs = time.perf_counter() - t0
    value = args.steps * n_s / secs
    sample = f"each step: oracle systematic resampling of {n_s} of the {w['N']} log-weights, no gather"
    line = {
        "impl": "reference", "metric": "standalone resample + gather throughput (particles/s)",
        "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": work.config(),
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serve_measure(steps: int, work: Work, smc, torch, dist, ws: int, local: int,
                  with_cpu: bool = True, n_plain: int = 300) -> dict:
    """Serve Poisson request streams through the continuous-batching server;
    returns the measurements (throughput, p50/p99 latency, the plain
    one-run-per-launch path on the first requests of the stream)."""
    w = work.w
    models = [smc.Model(r["kind"], **r["params"]) for r in work.runs]
    srv = smc.Server(96 << 30, precision=work.precision)
    pool: dict[int, list] = {}

    def take(q: int) -> dict:
        lst = pool.setdefault(q, [])
        if lst:
            return lst.pop()
        m, N = models[q], work.runs[q]["N"]
        o = {"log_z": torch.zeros(1, dtype=torch.float64).pin_memory(),
             "final_logw": torch.zeros(N, dtype=torch.float64).pin_memory(),
             "ancestors": torch.zeros((1, N), dtype=torch.int32).pin_memory(),
             "int_fields": torch.zeros((m.n_int, N), dtype=torch.int32).pin_memory()}
        if m.n_real:
            o["real_fields"] = torch.zeros((m.n_real, N), dtype=torch.float64).pin_memory()
        return o

    def stream_step(step: int, seconds: float):
        arr = inputs.poisson_arrivals(w["rate"], seconds, seed=w["arrival_seed"] + step)
        rng = np.random.Generator(np.random.PCG64(1000 + step))
        picks = rng.integers(0, len(work.runs), len(arr))
        tickets, used, units, d2h = [], [], 0, 0
        t0 = time.perf_counter()
        for a, q in zip(arr, picks):
            dt = t0 + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            r = work.runs[q]
            o = take(int(q))
            tickets.append(srv.submit(models[q], r["N"], seed=r["seed"] + 7919 * step,
                                      run_id=r["run_id"], outputs=o))
            used.append((int(q), o))
            units += r["N"] * r["segments"]
            d2h += sum(t.numel() * t.element_size() for t in o.values())
        res = [srv.wait(t, timeout=600.0) for t in tickets]
        span = time.perf_counter() - t0
        for q, o in used:
            pool.setdefault(q, []).append(o)
        lat = [r_["latency_s"] for r_ in res]
        lz = {(int(q), step): float(o["log_z"][0]) for (q, o) in used}
        return units, span, lat, len(arr), d2h, lz

    stream_step(10_000, 0.2)  # warm-up
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    units, span, lats, nreq, d2h = 0, 0.0, [], 0, 0
    served_lz = {}
    for s in range(steps):
        u, sp, la, n, b, lz = stream_step(s, w["seconds_per_step"])
        units, span, lats, nreq, d2h = units + u, span + sp, lats + la, nreq + n, d2h + b
        if s == 0:
            served_lz = lz
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    value, span = job_rate(units, span, dist, torch.device("cuda", local))
    # the first requests of the stream, served one run per launch in arrival order;
    # each also checks that the served result equals the plain one (equal log-Z error)
    arr = inputs.poisson_arrivals(w["rate"], w["seconds_per_step"], seed=w["arrival_seed"])
    rng = np.random.Generator(np.random.PCG64(1000))
    picks = rng.integers(0, len(work.runs), len(arr))
    n_plain = min(n_plain, len(arr))
    t_free, p_units, p_lat, same, compared = 0.0, 0, [], 0, 0
    for a, q in list(zip(arr, picks))[:n_plain]:
        r = work.runs[q]
        t_start = max(t_free, a)
        c0 = time.perf_counter()
        o = take(int(q))
        smc.run(models[q], r["N"], seed=r["seed"], run_id=r["run_id"], precision=work.precision,
                outputs=o)
        t_free = t_start + (time.perf_counter() - c0)
        p_lat.append(t_free - a)
        p_units += r["N"] * r["segments"]
        key = (int(q), 0)
        if key in served_lz:
            compared += 1
            same += int(served_lz[key] == float(o["log_z"][0]))
        pool.setdefault(int(q), []).append(o)
    plain = {"value": p_units / t_free, "unit": UNIT,
             "latency_ms": {"p50": 1e3 * float(np.percentile(p_lat, 50)),
                            "p99": 1e3 * float(np.percentile(p_lat, 99))},
             "what": f"the first {n_plain} requests of the stream, smc_run one after another in "
                     f"arrival order"}
    for m in models:
        m.close()
    cpu = None
    if ws == 1 and with_cpu:
        v, runs, secs, _ = oracle_throughput(work, 1e9, 32)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {runs} of the 512 request sizes, run one after another "
                         f"({secs:.1f} s single-threaded)"}
    return {"value": value, "unit": UNIT, "span_s": span, "requests": nreq,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lats, 50)),
                           "p99": 1e3 * float(np.percentile(lats, 99))},
            "d2h_bytes": d2h, "server": st, "cpu_baseline": cpu, "clocks": clk,
            "plain_one_run_per_launch": plain,
            "equal_log_z_error": {"served_equal_plain_log_z": same, "compared": compared,
                                  "rule": "a served request and the same request through smc_run "
                                          "give the same log Z bit for bit"}}


def run_serve(args, work: Work, smc, torch, dist, ws: int, rank: int, local: int) -> int:
    """The serve2000 workload as the benchmark line."""
    m = serve_measure(args.steps, work, smc, torch, dist, ws, local)
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": 1, "ms_per_step": 1e3 * m["span_s"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": work.config(), "requests": m["requests"], "latency_ms": m["latency_ms"],
        "e2e": {"value": m["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": m["d2h_bytes"] // args.steps},
        "gpu_launches": int(m["server"]["waves"]), "server": m["server"], "roofline": None,
        "cpu_baseline": m["cpu_baseline"], "clocks": m["clocks"],
        "plain_one_run_per_launch": m["plain_one_run_per_launch"],
        "equal_log_z_error": m["equal_log_z_error"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_resample(args, work: Work, smc, torch, dist, ws: int, rank: int, local: int) -> int:
    """The standalone resampling entry points on a 2^24-particle population."""
    w = work.w
    N = w["N"]
    dev = torch.device("cuda", local if dist else 0)
    lw_h = inputs.random_logw(N, seed=w["logw_seed"] + rank, scale=w["logw_scale"])
    lw = torch.from_numpy(lw_h).to(dev)
    wsb = torch.empty(smc.resample_workspace_bytes(N), dtype=torch.uint8, device=dev)
    anc = torch.empty(N, dtype=torch.int32, device=dev)
    o3 = torch.empty(3, dtype=torch.float64, device=dev)
    nn = torch.empty(1, dtype=torch.int64, device=dev)
    src = torch.randn(w["fields"], N, dtype=torch.float64, device=dev)
    dst = torch.empty_like(src)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    rng = np.random.default_rng(99 + rank)

    def step(u):
        smc.resample(lw, u, anc, o3, nn, wsb, stream=stream)
        smc.gather(src, dst, anc, stream=stream)

    for _ in range(args.warmup):
        step(float(rng.random() * 0.98 + 0.01))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    rs_ms, g_ms = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        u = float(rng.random() * 0.98 + 0.01)
        e[0].record(stream)
        smc.resample(lw, u, anc, o3, nn, wsb, stream=stream)
        e[1].record(stream)
        smc.gather(src, dst, anc, stream=stream)
        e[2].record(stream)
        e[2].synchronize()
        rs_ms.append(e[0].elapsed_time(e[1]))
        g_ms.append(e[1].elapsed_time(e[2]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_s = (sum(rs_ms) + sum(g_ms)) * 1e-3
    value, total_s = job_rate(args.steps * N, total_s, dist, dev)
    # end to end: host log-weights in (pinned), ancestors and the gathered state out
    lw_pin = torch.from_numpy(lw_h).pin_memory()
    anc_pin = torch.empty(N, dtype=torch.int32).pin_memory()
    dst_pin = torch.empty(w["fields"], N, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            lw.copy_(lw_pin, non_blocking=True)
        step(float(rng.random() * 0.98 + 0.01))
        with torch.cuda.stream(stream):
            anc_pin.copy_(anc, non_blocking=True)
            dst_pin.copy_(dst, non_blocking=True)
        stream.synchronize()
    e2e_value, _ = job_rate(e2e_steps * N, time.perf_counter() - t0, dist, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peaks = load_peaks()
    rs_s = float(np.mean(rs_ms)) * 1e-3
    g_s = float(np.mean(g_ms)) * 1e-3
    rs_gbs = RS_BYTES * N / rs_s / 1e9
    g_bytes = 4 + 2 * 8 * w["fields"]
    g_gbs = g_bytes * N / g_s / 1e9
    roof = {"bound": "hbm", "achieved": rs_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": rs_gbs / peaks["hbm_gbs"],
            "traffic": RS_NCU["bytes_per_call"] if RS_NCU["src_digest"] == src_digest(RS_SOURCES)
            else None,
            "kernel": "smc_resample (rs_tile_reduce + rs_combine + rs_ancestors<true>)",
            "bytes_per_particle": RS_BYTES, "avg_call_us": rs_s * 1e6,
            "peak_source": peaks["source"],
            "gather": {"achieved": g_gbs, "frac": g_gbs / peaks["hbm_gbs"], "avg_call_us": g_s * 1e6,
                       "bytes_per_particle": g_bytes}}
    cpu = None
    if ws == 1:
        import oracle

        n_s = 1 << 21
        t1 = time.perf_counter()
        oracle.resample(lw_h[:n_s], 0.5)
        secs = time.perf_counter() - t1
        cpu = {"value": n_s / secs, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle systematic resampling of the first {n_s} log-weights "
                         f"({secs:.2f} s single-threaded; no gather)"}
    line = {
        "metric": "standalone resample + gather throughput (particles/s)", "value": value,
        "unit": "particles/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": work.config(),
        "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 4 * N + 8 * w["fields"] * N},
        "gpu_launches": 4 * args.steps, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "n_near_last": int(nn.cpu()[0]),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def compute_peaks(smc) -> dict:
    """The arithmetic peaks measured on this GPU by the library's probe: FP64
    and FP32 fused multiply-add (TFLOP/s), the special function unit's ex2, the
    32-bit integer multiply-add and the 64-bit multiply-high (T ops/s)."""
    out = {}
    for k, (name, unit, flop) in smc.PEAK_KINDS.items():
        out[name] = {"value": smc.peak_probe(k, PROBE_ITERS[k]) * (flop or 1) / 1e12, "unit": unit}
    out["how"] = ("smc_peak_probe: 8 x 256 threads per SM, 8 independent chains of one "
                  "operation per thread, best of 3 launches timed with CUDA events")
    return out


def load_peaks() -> dict:
    """The HBM copy bandwidth the roofline divides by: the driver's measurement
    on the GB300s when its file is present, else the recipe's fallback."""
    f = ROOT / "MEASURED_PEAKS.json"
    try:
        d = json.loads(f.read_text())
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json)"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": HBM_PEAK_GBS, "source": "fallback (no MEASURED_PEAKS.json)"}


def rateshift_mean_sp(tree) -> float:
    """Mean pending-rate stack depth over a rate-shift run's checkpoints: the
    depth is a function of the traversal alone (a right child pops its parent's
    rate, an internal node pushes its own), the same for every particle."""
    sp, depths = 1, [1]  # the root's rate after the prior block
    for k in range(1, tree.n_nodes):
        v = int(tree.preorder[k])
        p = int(tree.parent[v])
        if int(tree.right[p]) == v:
            sp -= 1
        if int(tree.left[v]) >= 0:
            sp += 1
        depths.append(sp)
    return float(np.mean(depths))


def algorithmic_bytes(work: Work) -> tuple[float, str]:
    """Bytes per particle-step the method must move (the state read through the
    ancestor and written, the log-weight written and read, the ancestor written
    and read), in this library's layout."""
    kind = work.runs[0]["kind"]
    if kind == "lg":
        return 40.0, "x 8+8, logw 8+8, ancestor 4+4"
    if kind == "crbd":
        return 64.0, "lambda, mu 16+16, logw 8+8, ancestor 4+4, block index 4+4"
    if kind == "rateshift":
        sp = rateshift_mean_sp(work.runs[0]["params"]["tree"])
        b = (8 + 4 * sp + 8) * 2 + 4 + 4 + 4 + 4
        return b, (f"(lambda0, mu 8 + stack 4 sp + pc, sp 8) x 2 + logw 4+4 + ancestor 4+4, "
                   f"mean sp {sp:.2f} over the checkpoints")
    if kind == "seir":
        return (6 * 4 + 10 * 4) * 2 + 16 + 8, "6 reals + 10 ints read and written, logw, ancestor"
    return (4 * 8 + 4) * 2 + 16 + 8, "4 reals + block index read and written, logw, ancestor"


class DeviceBench:
    """A workload's runs with device-resident inputs and outputs, timed with CUDA
    events on the launching stream, L2 flushed between timed steps."""

    def __init__(self, work: Work, smc, torch, dev, launch: str = "auto"):
        self.work, self.smc, self.torch, self.dev = work, smc, torch, dev
        self.launch = launch
        self.stream = torch.cuda.Stream(device=dev)
        self.batch = work.w["kind"] == "batch"
        self.models = [smc.Model(r["kind"], **r["params"]) for r in work.runs]
        self.outs = [self._outputs(m, r["N"]) for m, r in zip(self.models, work.runs)]
        self.flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def _outputs(self, m, N):
        t = self.torch
        o = {"log_z": t.zeros(1, dtype=t.float64, device=self.dev),
             "final_logw": t.zeros(N, dtype=t.float64, device=self.dev),
             "ancestors": t.zeros((1, N), dtype=t.int32, device=self.dev),
             "resampled": t.zeros(1, dtype=t.int32, device=self.dev),
             "int_fields": t.zeros((m.n_int, N), dtype=t.int32, device=self.dev)}
        if m.n_real:
            o["real_fields"] = t.zeros((m.n_real, N), dtype=t.float64, device=self.dev)
        if m.stack_cap:
            o["stack"] = t.zeros((m.stack_cap, N), dtype=t.float64, device=self.dev)
        return o

    def step(self, seed_off: int, precision: str | None = None):
        w, smc = self.work, self.smc
        prec = precision or w.precision
        if self.batch:
            specs = [dict(N=r["N"], seed=r["seed"] + seed_off, run_id=r["run_id"], outputs=o)
                     for r, o in zip(w.runs, self.outs)]
            return smc.run_batch(self.models, specs, precision=prec, where="device",
                                 stream=self.stream, launch_graph=self.launch == "graph")
        r = w.runs[0]
        return [smc.run(self.models[0], r["N"], seed=r["seed"] + seed_off, run_id=r["run_id"],
                        precision=prec, where="device", stream=self.stream, outputs=self.outs[0],
                        ess_threshold=r.get("ess", 0.0), launch=self.launch)]

    def measure(self, steps: int, warmup: int, clocks=None, dist=None) -> dict:
        torch = self.torch
        for s in range(warmup):
            self.step(50000 + s)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        step_ms, logz, statuses, launches, segs = [], [], set(), 0, 0
        draws = blocks = 0
        for s in range(steps):
            with torch.cuda.stream(self.stream):
                self.flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            res = self.step(s)
            e1.record(self.stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            statuses.update(r["status"] for r in res)
            logz.append(float(self.outs[0]["log_z"].cpu()[0]))
            launches += res[0]["kernel_launches"]
            segs += res[0]["n_segments"]
            draws += sum(r["n_draws"] for r in res)
            blocks += sum(r["n_blocks"] for r in res)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        units = steps * self.work.units
        return {"step_ms": step_ms, "logz": logz, "statuses": sorted(statuses),
                "launches_per_step": launches // max(1, steps), "clocks": clk,
                "segments_per_step": segs / max(1, steps),
                "draws_per_pstep": draws / units, "blocks_per_pstep": blocks / units,
                "units": units}

    def close(self):
        for m in self.models:
            m.close()


def segment_roofline(work: Work, meas: dict, peaks: dict, name: str) -> dict:
    """The segment kernel's roofline from the timed steps themselves: a step is
    the run's waves (one wave_kernel launch per wave) plus a few small copies,
    so the mean wave time is at most ms_per_step / waves; the achieved rates
    below divide by that bound (never above the truth).  A small run launched as
    one kernel (one CTA or one cluster for all its segments) is divided by its
    segments instead."""
    r = work.runs[0]
    n_part = r["N"]
    waves = meas["launches_per_step"]
    one_launch = waves == 1 and meas.get("segments_per_step", 1) > 1
    per_step = meas["segments_per_step"] if one_launch else waves
    t_wave = float(np.mean(meas["step_ms"])) * 1e-3 / max(1, per_step)
    b_per, b_what = algorithmic_bytes(work)
    hbm = b_per * n_part / t_wave / 1e9
    info = NCU.get(name)
    traffic = None
    if info and info.get("src_digest") == src_digest():
        traffic = info["bytes_per_launch"]
    hbm_obj = {"achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": hbm / peaks["hbm_gbs"], "bytes_per_particle_step": b_per,
               "bytes_what": b_what, "peak_source": peaks["source"]}
    common = {"kernel": "wave_kernel (fused segment kernel)", "waves_per_step": waves,
              "wave_us": t_wave * 1e6, "traffic": traffic,
              "timing": "mean wave = ms_per_step / waves of the timed steps"}
    if one_launch:
        common = {"kernel": "small_run_kernel (every segment of the run in one launch)",
                  "segments_per_step": per_step, "segment_us": t_wave * 1e6, "traffic": None,
                  "timing": "mean segment = ms_per_step / segments of the timed steps"}
    if info and info["basis"] in ("issue", "fp64"):
        issue = info["warp_inst_per_pstep"] * n_part / t_wave
        fp64 = info["fp64_flop_per_pstep"] * n_part / t_wave
        issue_obj = {"achieved": issue / 1e12, "peak": ISSUE_PEAK / 1e12,
                     "unit": "T warp-instructions/s", "frac": issue / ISSUE_PEAK,
                     "per_unit": f"{info['warp_inst_per_pstep']} warp instructions per "
                                 f"particle-step (ncu)",
                     "peak_source": "derived: 152 SMs x 4 schedulers x 2070 MHz"}
        fp64_peak = peaks.get("fp64_flops", FP64_PEAK_FLOPS)
        fp64_obj = {"achieved": fp64 / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                    "frac": fp64 / fp64_peak,
                    "per_unit": f"{info['fp64_flop_per_pstep']} FP64 flop per particle-step (ncu)",
                    "peak_source": ("measured: the FP64 multiply-add probe (compute_peaks)"
                                    if "fp64_flops" in peaks else
                                    "derived: 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM"),
                    "derived_peak": FP64_PEAK_FLOPS / 1e12}
        main = issue_obj if info["basis"] == "issue" else fp64_obj
        return {"bound": "alu", **{k: main[k] for k in ("achieved", "peak", "unit", "frac")},
                "basis": "instruction issue" if info["basis"] == "issue" else "FP64 pipe",
                **common, "per_unit": main["per_unit"], "peak_source": main["peak_source"],
                "fp64": fp64_obj, "issue": issue_obj, "hbm": hbm_obj}
    return {"bound": "hbm", **{k: hbm_obj[k] for k in ("achieved", "peak", "unit", "frac")},
            **common, "per_unit": f"{b_per:.1f} algorithmic bytes per particle-step ({b_what})",
            "peak_source": peaks["source"]}


def e2e_measure(work: Work, smc, torch, stream, steps: int, dist, dev) -> tuple[float, int, int]:
    """The same metric end to end through the public API: every step registers
    the models from host data, runs, and copies the results to pinned host
    memory; returns (rate, host->device bytes, device->host bytes) per step."""
    batch = work.w["kind"] == "batch"
    pinned = []
    models0 = [smc.Model(r["kind"], **r["params"]) for r in work.runs]
    for m, r in zip(models0, work.runs):
        N = r["N"]
        o = {"log_z": torch.zeros(1, dtype=torch.float64).pin_memory(),
             "final_logw": torch.zeros(N, dtype=torch.float64).pin_memory(),
             "ancestors": torch.zeros((1, N), dtype=torch.int32).pin_memory(),
             "resampled": torch.zeros(1, dtype=torch.int32).pin_memory(),
             "int_fields": torch.zeros((m.n_int, N), dtype=torch.int32).pin_memory()}
        if m.n_real:
            o["real_fields"] = torch.zeros((m.n_real, N), dtype=torch.float64).pin_memory()
        if m.stack_cap:
            o["stack"] = torch.zeros((m.stack_cap, N), dtype=torch.float64).pin_memory()
        pinned.append(o)
    for m in models0:
        m.close()
    d2h = sum(t.numel() * t.element_size() for o in pinned for t in o.values())
    total = 0.0
    for s in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms2 = [smc.Model(r["kind"], **r["params"]) for r in work.runs]
        if batch:
            specs = [dict(N=r["N"], seed=r["seed"] + s, run_id=r["run_id"], outputs=o)
                     for r, o in zip(work.runs, pinned)]
            smc.run_batch(ms2, specs, precision=work.precision, where="host", stream=stream)
        else:
            r = work.runs[0]
            smc.run(ms2[0], r["N"], seed=r["seed"] + s, run_id=r["run_id"],
                    precision=work.precision, where="host", stream=stream, outputs=pinned[0],
                    ess_threshold=r.get("ess", 0.0))
        for m2 in ms2:
            m2.close()
        total += time.perf_counter() - t0
    value, _ = job_rate(steps * work.units, total, dist, dev)
    return value, work.input_bytes(), d2h


def config_lines(smc, torch, dev, peaks: dict) -> dict:
    """The metric's other configurations, measured in the same run on this GPU:
    C1 (lg), C3 (rateshift256, with its roofline and its FP32 log-Z error
    against the FP64 path on the same seeds), C4 (batch512 against the same
    runs one run per launch) and C5 (serve2000, p50/p99 against the plain path)."""
    out = {}
    # C1: one 1024-particle run of 50 segments (latency-bound)
    w = Work("lg", seed_base=1)
    b = DeviceBench(w, smc, torch, dev)
    m = b.measure(20, 3)
    b.close()
    ms = float(np.mean(m["step_ms"]))
    out["lg"] = {"value": w.units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                 "roofline": segment_roofline(w, m, peaks, "lg"), "status": m["statuses"],
                 "draws_per_particle_step": m["draws_per_pstep"],
                 "blocks_per_particle_step": m["blocks_per_pstep"]}
    # C3: rate-shift, 2^20 particles, FP32 particles / FP64 reductions
    w = Work("rateshift256", seed_base=1)
    b = DeviceBench(w, smc, torch, dev)
    m = b.measure(3, 2)
    ms = float(np.mean(m["step_ms"]))
    errs, lz32, lz64 = [], [], []
    for s in range(3):  # the same seeds at FP32 and FP64
        b.step(900 + s, "fp32")
        a = float(b.outs[0]["log_z"].cpu()[0])
        b.step(900 + s, "fp64")
        c = float(b.outs[0]["log_z"].cpu()[0])
        lz32.append(a)
        lz64.append(c)
        errs.append(abs(a - c))
    b.close()
    out["rateshift256"] = {
        "value": w.units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
        "roofline": segment_roofline(w, m, peaks, "rateshift256"), "status": m["statuses"],
        "draws_per_particle_step": m["draws_per_pstep"],
        "blocks_per_particle_step": m["blocks_per_pstep"],
        "log_z_error_vs_fp64": {"per_result": errs, "fp32": lz32, "fp64": lz64,
                                "what": "|log Z(FP32) - log Z(FP64)| for the same seed, run id "
                                        "and N (the FP64 path equals the FP64 oracle to 1e-9 "
                                        "relative; FP32 uniforms are the FP64 ones to 2^-24)",
                                "monte_carlo_sd_fp64": float(np.std(lz64, ddof=1))}}
    # C4: 512 uneven runs in one sequence of waves, against one run per launch
    w = Work("batch512", seed_base=1)
    b = DeviceBench(w, smc, torch, dev)
    m = b.measure(2, 1)
    ms = float(np.mean(m["step_ms"]))
    batch_lz = [float(o["log_z"].cpu()[0]) for o in b.outs]  # the last timed step's seeds
    seed_off = 1
    t_plain, same = 0.0, 0
    for q, (mo, r, o) in enumerate(zip(b.models, w.runs, b.outs)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        smc.run(mo, r["N"], seed=r["seed"] + seed_off, run_id=r["run_id"], precision=w.precision,
                where="device", stream=b.stream, outputs=o)
        e1.record(b.stream)
        e1.synchronize()
        t_plain += e0.elapsed_time(e1)
        same += int(float(o["log_z"].cpu()[0]) == batch_lz[q])
    b.close()
    plain_v = w.units / (t_plain * 1e-3)
    out["batch512"] = {"value": w.units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                       "status": m["statuses"], "launches_per_step": m["launches_per_step"],
                       "plain_one_run_per_launch": {"value": plain_v, "unit": UNIT,
                                                    "ms": t_plain},
                       "speedup_vs_plain": (w.units / (ms * 1e-3)) / plain_v,
                       "equal_log_z_error": {"runs_with_identical_log_z": same, "runs": len(w.runs),
                                             "rule": "each batched run and the same run through "
                                                     "smc_run give the same log Z bit for bit"}}
    # C5: one second of a Poisson stream at 2000 requests/s
    w = Work("serve2000", seed_base=1)
    sm = serve_measure(1, w, smc, torch, None, 1, 0, with_cpu=False, n_plain=200)
    out["serve2000"] = {k: sm[k] for k in ("value", "unit", "requests", "latency_ms",
                                            "plain_one_run_per_launch", "equal_log_z_error")}
    out["serve2000"]["speedup_vs_plain"] = sm["value"] / sm["plain_one_run_per_launch"]["value"]
    return out


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="crbd64", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the other configurations' sub-objects of the default line")
    ap.add_argument("--launch", default="auto",
                    choices=["auto", "waves", "graph", "one_cta", "cluster"],
                    help="launch form of the segments (results are the same bits)")
    ap.add_argument("--launch-graph", action="store_true", help="the same as --launch graph")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    work = Work(args.workload, seed_base=1 + 100000 * rank)
    if args.impl == "reference":
        return run_reference(args, work)

    import torch

    from paper_2112_00364_gb300 import smc

    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if work.w["kind"] == "serve":
        return run_serve(args, work, smc, torch, dist, ws, rank, local)
    if work.w["kind"] == "resample":
        return run_resample(args, work, smc, torch, dist, ws, rank, local)
    peaks = load_peaks()
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    launch = "graph" if args.launch_graph else args.launch
    bench = DeviceBench(work, smc, torch, dev, launch=launch)
    meas = bench.measure(args.steps, args.warmup, ClockSampler(gpu_index), dist)
    value, total_s = job_rate(meas["units"], sum(meas["step_ms"]) * 1e-3, dist, dev)
    total_ms = total_s * 1e3

    # the same runs one run per launch (plain path), timed once
    plain = None
    if bench.batch:
        torch.cuda.synchronize()
        t_plain = 0.0
        for m, r, o in zip(bench.models, work.runs, bench.outs):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(bench.stream)
            smc.run(m, r["N"], seed=r["seed"], run_id=r["run_id"], precision=work.precision,
                    where="device", stream=bench.stream, outputs=o)
            e1.record(bench.stream)
            e1.synchronize()
            t_plain += e0.elapsed_time(e1)
        plain = {"value": work.units / (t_plain * 1e-3), "unit": UNIT,
                 "what": "the same 512 runs through smc_run, one run after another"}
    e2e_steps = args.steps if not bench.batch else max(1, min(args.steps, 3))
    e2e_value, h2d, d2h = e2e_measure(work, smc, torch, bench.stream, e2e_steps, dist, dev)

    if rank != 0:
        bench.close()
        if dist:
            dist.destroy_process_group()
        return 0

    cpk = compute_peaks(smc)
    peaks["fp64_flops"] = cpk["fp64_fma"]["value"] * 1e12
    equal_error = None
    if work.w["kind"] == "crbd_ds":
        equal_error = equal_error_comparison(work, smc, torch, bench.stream)
    roof = None if bench.batch else segment_roofline(work, meas, peaks, args.workload)
    bench.close()
    cpu = None
    if ws == 1:
        if bench.batch:
            v, runs, secs, _ = oracle_throughput(work, 1e9, 32)
            sample = (f"the first {runs} of the 512 runs of the batch, run one after another "
                      f"({secs:.1f} s single-threaded)")
        else:
            n_s = min(work.runs[0]["N"], 1 << 16)
            v, runs, secs, _ = oracle_throughput(work, args.cpu_seconds, 50, n_particles=n_s)
            sample = (f"{runs} oracle runs of the workload with N={n_s} particles "
                      f"(of {work.runs[0]['N']}), seeds from {work.runs[0]['seed']}, "
                      f"{secs:.1f} s single-threaded")
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    configs = None
    if ws == 1 and args.workload == "crbd64" and not args.no_configs:
        configs = config_lines(smc, torch, dev, peaks)
    lat = sorted(meas["step_ms"])
    cfg_line = work.config()
    cfg_line["launch"] = {"auto": "the library's choice: every segment of a small run in "
                                  "one thread-block cluster, else one launch per wave",
                          "graph": "one captured CUDA graph per step",
                          "one_cta": "every segment of a small run in one CTA (else waves)",
                          "cluster": "every segment of a small run in one thread-block "
                                     "cluster (else waves)",
                          "waves": "one launch per wave and CTA size, chained by dependent "
                                   "launch"}[launch]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if work.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": cfg_line,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "log_z_run0": {"mean": float(np.mean(meas["logz"])), "sd": float(np.std(meas["logz"]))},
        "status": meas["statuses"],
        "work": {"draws_per_particle_step": meas["draws_per_pstep"],
                 "blocks_per_particle_step": meas["blocks_per_pstep"],
                 "what": "Philox blocks drawn by SAMPLE statements and basic blocks executed, "
                         "per particle-step, from the run's device counters"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * (meas["launches_per_step"] + len(work.runs)),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": meas["clocks"],
        "compute_peaks": cpk,
    }
    if plain:
        line["plain_one_run_per_launch"] = plain
    if equal_error:
        line["equal_log_z_error"] = equal_error
    if configs:
        line["configs"] = configs
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
