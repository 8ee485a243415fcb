"""Write the oracle regression fixtures of this folder.

The paper prints no numeric worked example whose inputs are available (its
normalising-constant estimates, Appendix "Normalizing Constant Experiment
Estimates", are box plots over the Alcedinidae, SSM and Tyrant-flycatcher data,
which are not public here), so the oracle is pinned by closed forms and
statistical tests (tests/test_oracle_*.py, tests/closed_forms.py).  These
fixtures are a regression record on top of those pins: fixed small runs of each
oracle model and a few Philox4x32-10 blocks, written by this script from the
oracle alone.  tests/test_golden.py checks that the oracle still reproduces
them; a change to the oracle's arithmetic must regenerate them in a commit that
names the passage or reading that justifies it.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
ROOT = HERE.parents[1]
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

import inputs  # noqa: E402
import oracle  # noqa: E402

# (name, model kind, N, seed, precision, parameters as a recipe of inputs)
CASES = [
    ("lg_t50_n1024", "lg", 1024, 1, "fp64", {"obs": ("lg_observations", 50, 1)}),
    ("crbd_16tips_n3000", "crbd", 3000, 1, "fp64", {"tree": ("yule_tree", 16, 2)}),
    ("crbd_16tips_n3000_fp32", "crbd", 3000, 1, "fp32", {"tree": ("yule_tree", 16, 2)}),
    ("crbd_fixed_rates_8tips", "crbd", 2000, 3, "fp64",
     {"tree": ("yule_tree", 8, 4), "rates": (1.5, 0.5)}),
    ("rateshift_12tips", "rateshift", 1500, 2, "fp64", {"tree": ("yule_tree", 12, 3)}),
    ("geometric_n1024", "geometric", 1024, 5, "fp64", {}),
    ("seir_28days_n500", "seir", 500, 4, "fp64", {"obs": ("seir_observations", 28, 7)}),
    ("crbd_ds_16tips_ess", "crbd_ds", 2000, 6, "fp64",
     {"tree": ("yule_tree", 16, 5), "ess_threshold": 0.5}),
]

PHILOX_COUNTERS = [[0, 0, 0, 0], [1, 2, 3, 4], [0xFFFFFFFF, 0, 7, 1], [12345, 678, 9, 2]]
PHILOX_KEYS = [[0, 0], [1, 0], [0xDEADBEEF, 0x12345678], [7, 0xFFFFFFFF]]


def build_params(recipe: dict) -> tuple[dict, float]:
    params, ess = {}, 0.0
    for k, v in recipe.items():
        if k == "ess_threshold":
            ess = v
        elif k == "rates":
            params[k] = tuple(v)
        elif k == "obs":
            fn, n, seed = v
            params[k] = getattr(inputs, fn)(n, seed=seed)
        elif k == "tree":
            fn, n, seed = v
            params[k] = getattr(inputs, fn)(n, seed=seed)
    return params, ess


def run_case(kind: str, N: int, seed: int, prec: str, recipe: dict) -> dict:
    params, ess = build_params(recipe)
    if kind == "rateshift":
        params["lam_stack_cap"] = params["tree"].max_pending_right() + 1
    r = oracle.smc_run(kind, N, seed, precision=oracle.FP64 if prec == "fp64" else oracle.FP32,
                       ess_threshold=ess, record_ancestors=True, **params)
    anc = r.get("ancestors")
    last = anc[-1] if anc is not None and len(anc) else np.arange(N, dtype=np.int32)
    return {
        "log_z": float(r["log_z"]).hex(),
        "n_segments": int(r["n_segments"]),
        "n_resamples": int(r["n_resamples"]),
        "status": int(r["status"]),
        "final_logw_sum": float(np.sum(r["final_logw"][np.isfinite(r["final_logw"])])).hex(),
        "last_ancestors_head": [int(a) for a in last[:16]],
        "last_ancestors_sum": int(np.sum(last.astype(np.int64))),
    }


def philox_blocks() -> list:
    ctr = np.array(PHILOX_COUNTERS, dtype=np.uint32)
    key = np.array(PHILOX_KEYS, dtype=np.uint32)
    out = oracle.philox(ctr, key)
    return [[int(w) for w in row] for row in out]


def main() -> None:
    cases = {}
    for name, kind, N, seed, prec, recipe in CASES:
        cases[name] = {"kind": kind, "N": N, "seed": seed, "precision": prec,
                       "recipe": {k: list(v) if isinstance(v, tuple) else v
                                  for k, v in recipe.items()},
                       "expected": run_case(kind, N, seed, prec, recipe)}
    doc = {"source": "oracle/ via tests/golden/make_golden.py",
           "philox": {"counters": PHILOX_COUNTERS, "keys": PHILOX_KEYS,
                      "blocks": philox_blocks()},
           "runs": cases}
    (HERE / "oracle_runs.json").write_text(json.dumps(doc, indent=1) + "\n")
    print(f"wrote {len(cases)} runs and {len(PHILOX_COUNTERS)} Philox blocks")


if __name__ == "__main__":
    main()
