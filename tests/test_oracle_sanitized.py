"""The oracle runs clean under AddressSanitizer and UndefinedBehaviorSanitizer
(CPU only).

A copy of the oracle package is built with -fsanitize=address,undefined (any
undefined behaviour aborts) and a quick subset of its tests runs against it in
a child process with the sanitizer runtimes preloaded: the regression runs of
every model, the resampling pins, the rate-shift stack, the kill rules, a SEIR
transition day, the ESS rule and snapshot / resume.  An out-of-bounds access, a use after free,
a signed overflow or an invalid shift in the oracle fails the child.
"""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import sys
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent
ORACLE = ROOT / "oracle"

SUBSET = [
    "test_golden.py",
    "test_oracle_resample.py",
    "test_oracle_models.py::test_rateshift_stack_depth_and_final_state",
    "test_oracle_models.py::test_depth_cap_and_call_limit_kill",
    "test_oracle_models.py::test_step_limit",
    "test_oracle_seir.py::test_one_day_transition_law",
    "test_oracle_ess.py::test_threshold_above_one_equals_every_checkpoint",
    "test_oracle_crbd_ds.py::test_crbd_ds_posterior_bookkeeping",
    "test_oracle_resume.py",
]


def _runtime(name: str) -> str | None:
    try:
        p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True,
                           check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc sanitizer runtimes not installed")
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    for name in ("__init__.py", "smc_oracle.c", "smc_oracle.h", "smc_oracle_prec.inc"):
        shutil.copy(ORACLE / name, pkg / name)
    lib = pkg / "liboracle.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-fsanitize=address,undefined",
                    "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-o", str(lib),
                    str(pkg / "smc_oracle.c"), "-lm"], check=True)
    os.utime(lib)  # newer than the sources: the package loads it instead of rebuilding
    env = dict(os.environ, SMC_ORACLE_UNDER_TEST=str(tmp_path), PYTHONDONTWRITEBYTECODE="1",
               LD_PRELOAD=f"{asan} {ubsan}", ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    # -s: a sanitizer report is written to stderr as the child aborts, which
    # pytest's output capture would swallow
    cmd = [sys.executable, "-m", "pytest", "-s", "-x", "-q", "-m", "not gpu",
           "-p", "no:cacheprovider", "--keep-duplicates", *[str(HERE / s) for s in SUBSET]]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    hits = [out.find(m) for m in ("runtime error", "AddressSanitizer",
                                  "UndefinedBehaviorSanitizer") if m in out]
    if hits:  # the report's first lines name the file and line
        start = min(hits)
        pytest.fail(out[max(0, start - 300):start + 2500])
    assert r.returncode == 0, out[-4000:]
    m = re.search(r"(\d+) passed", out)
    assert m and int(m.group(1)) >= 30, out[-2000:]  # the subset ran
