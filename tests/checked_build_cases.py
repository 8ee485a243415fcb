"""Parity cases run against the library's checking build (test infrastructure).

Run as a script in its own process with SMC_LIB_VARIANT=debug (one library
variant per process): every case is compared with the oracle as the parity
tests compare it, and every run's checking counters must show no out-of-range
access.  Prints one line per case and "ALL OK" at the end.
"""
import os
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parent))
sys.path.insert(0, str(HERE))

import inputs  # noqa: E402
from parity import assert_parity_exact, assert_parity_fp64, run_pair  # noqa: E402


def check_counters(res, name):
    assert res["debug_code"] == 0 and res["debug_count"] == 0, (name, res["debug_code"],
                                                                res["debug_index"], res["debug_count"])


def main():
    assert os.environ.get("SMC_LIB_VARIANT") == "debug"
    from paper_2112_00364_gb300 import build, smc

    assert Path(smc.lib()._name) == build.LIB_DEBUG
    tree = inputs.yule_tree(24, seed=5)
    rs = dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    cases = [
        ("lg fp64", "lg", 3000, 1, "fp64", 0.0, dict(obs=inputs.lg_observations(40, seed=2))),
        ("crbd fp64", "crbd", 4097, 2, "fp64", 0.0, dict(tree=tree)),
        ("crbd fp32 last-CTA combine", "crbd", 300_001, 3, "fp32", 0.0,
         dict(tree=inputs.yule_tree(8, seed=4))),
        ("rateshift fp32", "rateshift", 5000, 4, "fp32", 0.0, rs),
        ("rateshift fp64 ess", "rateshift", 3001, 5, "fp64", 0.5, rs),
        ("crbd_ds fp64 ess", "crbd_ds", 4000, 6, "fp64", 0.5, dict(tree=tree)),
        ("seir fp32", "seir", 1500, 7, "fp32", 0.0, dict(obs=inputs.seir_observations(35, seed=7))),
        ("geometric fp64", "geometric", 2000, 8, "fp64", 0.0, {}),
    ]
    for name, kind, N, seed, prec, ess, p in cases:
        g, o = run_pair(kind, N, seed, precision=prec, ess_threshold=ess, **p)
        check_counters(g, name)
        (assert_parity_exact if prec == "fp32" else assert_parity_fp64)(g, o)
        print("ok", name, flush=True)
    # a batch and served requests through the same checked kernels
    specs = inputs.batch_specs(16, seed=8)
    models = [smc.Model(sp.kind, **(dict(obs=inputs.lg_observations(sp.T, seed=sp.obs_seed))
                                    if sp.kind == "lg" else
                                    dict(tree=inputs.yule_tree(sp.tips, seed=sp.tree_seed))))
              for sp in specs]
    runs = [dict(N=sp.n_particles, seed=sp.seed, run_id=q) for q, sp in enumerate(specs)]
    for r in smc.run_batch(models, runs, precision="fp32"):
        check_counters(r, "batch")
    srv = smc.Server(2 << 30, precision="fp32")
    tickets = [srv.submit(m, r["N"], r["seed"], run_id=r["run_id"]) for m, r in zip(models, runs)]
    for t in tickets:
        check_counters(srv.wait(t), "server")
    srv.close()
    print("ok batch and server", flush=True)
    print("ALL OK", flush=True)


if __name__ == "__main__":
    main()
