"""Pins for the oracle's ESS-triggered resampling (CPU only).

With a threshold tau the population is resampled after a checkpoint only when
ESS = (sum w)^2 / sum w^2 < tau N; otherwise the weights accumulate and log Z
gains log((1/N) sum W) of the accumulated weights W when they are next closed
(at a resampling, the end or the step limit).  Pinned by:
  * tau above 1 (ESS <= N always): identical, bit for bit, to resampling at
    every checkpoint;
  * tau N below 1 (ESS >= 1 always): never resampled, ancestors the identity,
    and log Z equals the importance-sampling estimate logsumexp(W) - log N of
    the final accumulated weights (a dropped or doubled increment breaks it);
  * unbiasedness of Zhat at tau = 0.5 against the Kalman likelihood and the
    closed-form CRBD likelihood, and of the importance-sampling estimate;
  * the decision record: rows without resampling are the identity, the others
    non-decreasing, and at tau = 0.5 the population is resampled sometimes but
    not always.
"""
import numpy as np
import pytest
from scipy.special import logsumexp

import closed_forms as cf
import inputs
import oracle


def _run(model, N, seed, **kw):
    r = oracle.smc_run(model, N, seed, record_ancestors=True, **kw)
    assert r["status"] == 0, r["status"]
    return r


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_threshold_above_one_equals_every_checkpoint(prec):
    y = inputs.lg_observations(30, seed=2)
    tree = inputs.yule_tree(12, seed=3)
    for model, kw in [("lg", dict(obs=y)), ("crbd", dict(tree=tree))]:
        a = _run(model, 700, 5, precision=prec, **kw)
        b = _run(model, 700, 5, precision=prec, ess_threshold=1.5, **kw)
        assert a["log_z"] == b["log_z"]
        np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
        np.testing.assert_array_equal(a["final_logw"], b["final_logw"])
        np.testing.assert_array_equal(a["real_fields"], b["real_fields"])
        assert b["n_resamples"] == b["n_segments"] - 1
        assert np.all(b["resampled"] == 1)


def test_tiny_threshold_is_importance_sampling():
    y = inputs.lg_observations(20, seed=4)
    N = 500
    r = _run("lg", N, 3, obs=y, ess_threshold=1e-9)
    assert r["n_resamples"] == 0 and np.all(r["resampled"] == 0)
    np.testing.assert_array_equal(r["ancestors"], np.tile(np.arange(N), (r["n_segments"] - 1, 1)))
    # the only increment is the final one, over the weights accumulated along
    # the whole run
    assert abs(r["log_z"] - (logsumexp(r["final_logw"]) - np.log(N))) <= 1e-12 * abs(r["log_z"])
    tree = inputs.yule_tree(8, seed=5)
    c = _run("crbd", N, 3, tree=tree, rates=(2.0, 0.5), ess_threshold=1e-9)
    assert c["n_resamples"] == 0
    assert abs(c["log_z"] - (logsumexp(c["final_logw"]) - np.log(N))) <= 1e-12 * abs(c["log_z"])


def test_decision_record():
    y = inputs.lg_observations(50, seed=1)
    r = _run("lg", 1024, 7, obs=y, ess_threshold=0.5)
    n_tr = r["n_segments"] - 1
    assert 0 < r["n_resamples"] < n_tr
    assert r["resampled"].sum() == r["n_resamples"]
    for k in range(n_tr):
        row = r["ancestors"][k]
        if r["resampled"][k]:
            assert np.all(np.diff(row) >= 0)
        else:
            np.testing.assert_array_equal(row, np.arange(1024))


def test_ess_resampling_unbiased_lg():
    y = inputs.lg_observations(50, seed=1)
    lz = np.array([_run("lg", 1024, s, obs=y, ess_threshold=0.5)["log_z"] for s in range(1, 101)])
    ok, mean, se = cf.unbiased_check(lz, cf.kalman_loglik(y))
    assert ok, (mean, se)


def test_ess_resampling_unbiased_crbd_fixed_rates():
    tree = inputs.yule_tree(16, seed=2)
    lz = np.array([_run("crbd", 2048, s, tree=tree, rates=(3.0, 1.0), ess_threshold=0.5)["log_z"]
                   for s in range(1, 101)])
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_log_z(tree, 3.0, 1.0))
    assert ok, (mean, se)


def test_importance_sampling_unbiased_lg():
    y = inputs.lg_observations(5, seed=6)
    lz = np.array([_run("lg", 2048, s, obs=y, ess_threshold=1e-9)["log_z"] for s in range(1, 101)])
    ok, mean, se = cf.unbiased_check(lz, cf.kalman_loglik(y))
    assert ok, (mean, se)


def test_follow_mode_adopts_decisions():
    y = inputs.lg_observations(50, seed=1)
    a = _run("lg", 1024, 7, obs=y, ess_threshold=0.5)
    fake = a["resampled"].copy()
    k = int(np.flatnonzero(fake)[0])
    fake[k] = 0  # keep the population where the run resampled
    b = _run("lg", 1024, 7, obs=y, ess_threshold=0.5, follow_resampled=fake)
    np.testing.assert_array_equal(b["resampled"][: k + 1], fake[: k + 1])
    assert b["n_dec_hard_mismatch"] + b["n_dec_flag_mismatch"] >= 1
    assert b["log_z"] != a["log_z"]


def test_ess_near_band_is_relative():
    # geometric program: after segment 0 the weights are 1.5 (heads) or 1
    # (tails); a snapshot there gives them exactly, so the threshold can be put
    # 1e-7 above the ESS: inside the band 1e-9 tau N (about 5e-7), outside an
    # absolute 1e-9
    N = 1000
    snap = oracle.smc_run("geometric", N, 4, max_segments=1)
    lw = snap["final_logw"]
    w = np.exp(lw - lw.max())
    ess = w.sum() ** 2 / (w * w).sum()
    assert 0.3 * N < ess < N
    above = oracle.smc_run("geometric", N, 4, ess_threshold=(ess + 1e-7) / N)
    below = oracle.smc_run("geometric", N, 4, ess_threshold=(ess - 1e-7) / N)
    assert above["n_ess_flagged"] >= 1 and below["n_ess_flagged"] >= 1
    # and the decision at checkpoint 0 falls on the side the threshold says
    assert above["resampled"][0] == 1 and below["resampled"][0] == 0
