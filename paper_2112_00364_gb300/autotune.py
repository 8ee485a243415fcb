"""Autotuner of the library's tile table (run on the GPU the library serves).

A run of N particles is cut into tiles, one CTA per tile and wave; the tile
size must be a function of N alone (it fixes how the weights are rounded, so a
run gives the same bits alone, batched and served).  The library reads it from
a table of N bands (csrc/smc_tile_table.inc): the band with the smallest
n_max >= N gives tiles of clamp(ceil(N / slots), tile_min, tile_max).

For every band this script times each candidate rule on a representative N:
  - a batch of 48 runs of that N (half linear-Gaussian with T = 50, half CRBD
    on a 32-tip tree, FP32 particles: the batched configuration's work),
  - one linear-Gaussian run and one CRBD run alone (FP64: the latency of a
    single run),
each the median of repeated CUDA-event timings, and scores a candidate by the
mean of log(throughput / best throughput) over the three.  The best candidate
of each band is written to csrc/smc_tile_table.inc (adjacent bands with the
same choice merged), and the whole sweep to the file given by --report.

    python -m paper_2112_00364_gb300.autotune [--report FILE] [--table FILE] [--dry-run]

It needs a CUDA device; the library must be built (python -c "import
__graft_entry__ as g; g.build()").  Rebuild the library afterwards to compile
the new table in.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
TABLE = PKG / "csrc" / "smc_tile_table.inc"

# band upper edges (particles); the last band reaches the largest run
EDGES = [256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536, 131072, 0x7FFFFFFF]
SLOTS = [152, 304, 456, 608, 912]
TILE_MIN = [32, 64]
TILE_MAX = 256
BATCH_RUNS = 48


def representative(i: int) -> int:
    lo = EDGES[i - 1] if i > 0 else 128
    hi = EDGES[i] if i + 1 < len(EDGES) else 1 << 18
    return int(round(math.sqrt(lo * hi)))


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--report", default=None, help="write the sweep (JSON) here")
    ap.add_argument("--dry-run", action="store_true", help="do not write the table")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--table", default=str(TABLE), help="where to write the table")
    args = ap.parse_args()
    sys.path.insert(0, str(ROOT))
    import numpy as np
    import torch

    import inputs
    from paper_2112_00364_gb300 import smc

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    obs = inputs.lg_observations(50, seed=1)
    tree = inputs.yule_tree(32, seed=2)
    m_lg = smc.Model("lg", obs=obs)
    m_crbd = smc.Model("crbd", tree=tree)

    def timed(fn, reps):
        fn()  # warm-up (also sizes the cached workspace)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return float(np.median(ts))

    def measure(N: int) -> dict:
        models = [m_lg if q % 2 == 0 else m_crbd for q in range(BATCH_RUNS)]
        specs = [dict(N=N, seed=10 + q, run_id=q) for q in range(BATCH_RUNS)]
        units_b = sum(N * (50 if q % 2 == 0 else tree.n_nodes) for q in range(BATCH_RUNS))
        tb = timed(lambda: smc.run_batch(models, specs, precision="fp32", where="device",
                                         stream=stream), args.reps)
        tl = timed(lambda: smc.run(m_lg, N, 3, where="device", stream=stream), 2 * args.reps)
        tc = timed(lambda: smc.run(m_crbd, N, 4, where="device", stream=stream), 2 * args.reps)
        return {"batch": units_b / tb, "lg": N * 50 / tl, "crbd": N * tree.n_nodes / tc}

    report = {"gpu": torch.cuda.get_device_name(0), "when": time.strftime("%Y-%m-%d %H:%M:%S"),
              "batch_runs": BATCH_RUNS, "bands": []}
    chosen = []
    for i, n_max in enumerate(EDGES):
        N = representative(i)
        rows = []
        for slots in SLOTS:
            for tmin in TILE_MIN:
                smc.set_tile_bands([(0x7FFFFFFF, slots, tmin, TILE_MAX)])
                tile = smc.tile_size(N)
                if any(r["tile"] == tile for r in rows):  # the same tiling: reuse its timing
                    same = next(r for r in rows if r["tile"] == tile)
                    rows.append(dict(same, slots=slots, tile_min=tmin))
                    continue
                rows.append({"slots": slots, "tile_min": tmin, "tile": tile, **measure(N)})
        best = {k: max(r[k] for r in rows) for k in ("batch", "lg", "crbd")}
        for r in rows:
            r["score"] = float(np.mean([math.log(r[k] / best[k]) for k in best]))
        win = max(rows, key=lambda r: (r["score"], -r["slots"]))
        chosen.append((n_max, win["slots"], win["tile_min"], TILE_MAX))
        report["bands"].append({"n_max": n_max, "N": N, "chosen": win, "candidates": rows})
        print(f"band <= {n_max}: N={N} -> slots {win['slots']} tile_min {win['tile_min']} "
              f"(tile {win['tile']}, score {win['score']:.3f})", flush=True)
    smc.set_tile_bands(None)
    m_lg.close()
    m_crbd.close()
    merged = []
    for b in chosen:
        if merged and merged[-1][1:] == b[1:]:
            merged[-1] = b
        else:
            merged.append(b)
    report["table"] = merged
    if args.report:
        Path(args.report).write_text(json.dumps(report, indent=1) + "\n")
    if not args.dry_run:
        lines = ["// Tile bands {n_max, slots, tile_min, tile_max, pad}: a run of N <= n_max",
                 "// particles gets tiles of clamp(ceil(N / slots), tile_min, tile_max).",
                 f"// Written by autotune.py on {report['gpu']} ({report['when']}): per band the",
                 "// candidate with the best mean log-throughput over a 48-run batch (FP32) and",
                 "// single linear-Gaussian and CRBD runs (FP64)."]
        for n_max, slots, tmin, tmax in merged:
            lines.append(f"{{{n_max:#x}ll, {slots}, {tmin}, {tmax}, 0}},")
        Path(args.table).write_text("\n".join(lines) + "\n")
        print(f"wrote {args.table}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
