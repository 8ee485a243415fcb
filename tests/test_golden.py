"""The oracle against its regression fixtures (tests/golden/oracle_runs.json).

The fixtures were written by tests/golden/make_golden.py from the oracle alone
(the paper prints no numeric worked example whose inputs are available): fixed
small runs of every oracle model and a few Philox4x32-10 blocks.  The oracle must
reproduce them exactly (log Z and weight sums to the bit, segment and
resampling counts, the last ancestors); a change to its arithmetic shows up here
and has to be regenerated with the passage or reading that justifies it.
"""
import json
from pathlib import Path

import numpy as np
import pytest

import oracle

GOLDEN = Path(__file__).resolve().parent / "golden"
DOC = json.loads((GOLDEN / "oracle_runs.json").read_text())


def _make():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden",
                                                  GOLDEN / "make_golden.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_philox_blocks():
    ph = DOC["philox"]
    out = oracle.philox(np.array(ph["counters"], dtype=np.uint32),
                        np.array(ph["keys"], dtype=np.uint32))
    np.testing.assert_array_equal(out.astype(np.int64), np.array(ph["blocks"], dtype=np.int64))


@pytest.mark.parametrize("name", sorted(DOC["runs"]))
def test_oracle_run_reproduces_fixture(name):
    mg = _make()
    case = DOC["runs"][name]
    recipe = {k: tuple(v) if isinstance(v, list) else v for k, v in case["recipe"].items()}
    got = mg.run_case(case["kind"], case["N"], case["seed"], case["precision"], recipe)
    assert got == case["expected"], (name, got, case["expected"])
