"""The library's checking build on the parity cases (GPU).

libsmc_debug.so is the same sources compiled with SMC_DEBUG_CHECKS: every
ancestor index is checked against [0, N), every gathered block index against
the model's blocks and every gathered stack pointer against the stack
capacity; an access found out of range is recorded in the run's counters and
skipped (no trap).  The parity cases of every model (both precisions, ESS,
more than one combining CTA, a batch and served requests) run in a process of
their own on the checking build: results equal the oracle as in the release
build's tests, and no run records a violation.
"""
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

HERE = Path(__file__).resolve().parent


def test_parity_cases_on_the_checking_build_record_no_violation():
    env = dict(os.environ, SMC_LIB_VARIANT="debug")
    p = subprocess.run([sys.executable, str(HERE / "checked_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900, cwd=str(HERE.parent))
    assert p.returncode == 0 and "ALL OK" in p.stdout, (p.stdout[-3000:], p.stderr[-3000:])
