"""Snapshot and resume of the oracle's runs (CPU only).

Between checkpoints a run is its particles' states and log-weights, the log Z
closed so far and the segment index; every draw comes from a counter keyed by
(seed, run, particle, segment, draw).  So a run stopped by the step limit after
k segments (a snapshot) and resumed from its outputs must end exactly as the
uninterrupted run: the same log Z, final states and log-weights bit for bit,
and the same ancestors from checkpoint k - 1 on.  Checked for every model, at
FP64 and FP32, with resampling at every checkpoint and ESS-triggered, and for
a snapshot resumed twice in a chain.
"""
import numpy as np
import pytest

import inputs
import oracle


def _params(kind):
    if kind == "lg":
        return dict(obs=inputs.lg_observations(30, seed=2))
    if kind == "seir":
        return dict(obs=inputs.seir_observations(28, seed=7))
    if kind == "geometric":
        return {}
    tree = inputs.yule_tree(12, seed=3)
    if kind == "rateshift":
        return dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    return dict(tree=tree)


def _same(a, b, from_row):
    assert a["status"] == b["status"]
    assert a["log_z"] == b["log_z"]
    assert a["n_segments"] == b["n_segments"]
    np.testing.assert_array_equal(a["final_logw"], b["final_logw"])
    np.testing.assert_array_equal(a["real_fields"], b["real_fields"])
    np.testing.assert_array_equal(a["int_fields"], b["int_fields"])
    if a["stack"] is not None:
        np.testing.assert_array_equal(a["stack"], b["stack"])
    np.testing.assert_array_equal(a["ancestors"][from_row:], b["ancestors"][from_row:])
    np.testing.assert_array_equal(a["resampled"][from_row:], b["resampled"][from_row:])


@pytest.mark.parametrize("kind", ["lg", "crbd", "rateshift", "geometric", "seir", "crbd_ds"])
@pytest.mark.parametrize("ess", [0.0, 0.5])
@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_resume_equals_uninterrupted_run(kind, ess, prec):
    p = _params(kind)
    kw = dict(precision=prec, ess_threshold=ess, record_ancestors=True, **p)
    N, seed = 700, 5
    full = oracle.smc_run(kind, N, seed, **kw)
    assert full["status"] == 0 and full["n_segments"] >= 4
    for k in (1, 2, full["n_segments"] // 2, full["n_segments"] - 1):
        snap = oracle.smc_run(kind, N, seed, max_segments=k, **kw)
        assert snap["status"] == oracle.ESTEPLIMIT and snap["n_segments"] == k
        res = oracle.smc_run(kind, N, seed, resume_from=snap, **kw)
        _same(res, full, k - 1)


def test_resume_chain_and_unclosed_weights():
    # ESS-triggered: a snapshot may hold weights accumulated over several
    # segments; log_z_closed leaves them out (log_z adds them, as the run ended)
    p = _params("lg")
    kw = dict(ess_threshold=0.3, record_ancestors=True, **p)
    full = oracle.smc_run("lg", 600, 9, **kw)
    k1, k2 = 6, 17
    s1 = oracle.smc_run("lg", 600, 9, max_segments=k1, **kw)
    s2 = oracle.smc_run("lg", 600, 9, max_segments=k2, resume_from=s1, **kw)
    assert s2["status"] == oracle.ESTEPLIMIT and s2["n_segments"] == k2
    res = oracle.smc_run("lg", 600, 9, resume_from=s2, **kw)
    _same(res, full, k2 - 1)
    # some snapshot along the run carried unclosed weights
    opened = [oracle.smc_run("lg", 600, 9, max_segments=k, **kw) for k in range(2, 12)]
    assert any(s["log_z_closed"] != s["log_z"] for s in opened)


def test_resume_argument_checks():
    p = _params("crbd")
    snap = oracle.smc_run("crbd", 100, 1, max_segments=3, **p)
    # a snapshot taken at segment 3 cannot be resumed under a limit of 2
    r = oracle.smc_run("crbd", 100, 1, max_segments=2, resume_from=snap, **p)
    assert r["status"] == oracle.EINVAL
