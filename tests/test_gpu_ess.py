"""ESS-triggered resampling on the GPU against the oracle (Section 3.3).

The oracle runs in follow mode: it adopts the GPU's ancestors and its
resample / keep decisions, and a decision may differ only where the oracle's
ESS lies within 1e-9 of the threshold; everything else as in the FP64 parity
tests.  Plus: a threshold above 1 is resampling after every checkpoint, bit
for bit; the estimate stays unbiased; batched runs equal single runs.
"""
import numpy as np
import pytest

import closed_forms as cf
import inputs
from parity import assert_parity_exact, assert_parity_fp64, run_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,tau", [(1024, 0.5), (3001, 0.3), (257, 0.15)])
def test_lg_ess_parity(N, tau):
    y = inputs.lg_observations(50, seed=1)
    g, o = run_pair("lg", N, 7, obs=y, ess_threshold=tau)
    assert 0 < g["n_resamples"] < g["n_segments"] - 1
    np.testing.assert_array_equal(g["resampled"], o["resampled"])
    assert_parity_fp64(g, o)


def test_crbd_ess_parity():
    tree = inputs.yule_tree(16, seed=2)
    g, o = run_pair("crbd", 3000, 4, tree=tree, ess_threshold=0.5)
    np.testing.assert_array_equal(g["resampled"], o["resampled"])
    assert_parity_fp64(g, o)


def test_rateshift_ess_parity():
    tree = inputs.yule_tree(24, seed=3)
    g, o = run_pair("rateshift", 2500, 4, tree=tree, sigma=0.3,
                    lam_stack_cap=tree.max_pending_right() + 1, ess_threshold=0.7)
    assert_parity_fp64(g, o)
    np.testing.assert_allclose(g["stack"], o["stack"], rtol=1e-12, atol=0)


def test_large_population_ess_parity():
    """One-CTA combine path (1,172 tiles)."""
    y = inputs.lg_observations(12, seed=3)
    g, o = run_pair("lg", 300_001, 5, obs=y, ess_threshold=0.5)
    assert_parity_fp64(g, o)


def test_threshold_above_one_is_every_checkpoint():
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(32, seed=5)
    m = smc.Model("crbd", tree=tree)
    a = smc.run(m, 20_000, 3, record_all_ancestors=True)
    b = smc.run(m, 20_000, 3, record_all_ancestors=True, ess_threshold=1.5)
    assert a["log_z_value"] == b["log_z_value"]
    np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
    np.testing.assert_array_equal(a["final_logw"], b["final_logw"])
    assert b["n_resamples"] == b["n_segments"] - 1 and np.all(b["resampled"] == 1)


def test_ess_unbiased_crbd_64_tips():
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(64, seed=2)
    m = smc.Model("crbd", tree=tree, rates=(4.0, 1.0))
    runs = [smc.run(m, 1 << 16, s, ess_threshold=0.5) for s in range(1, 61)]
    assert all(0 < r["n_resamples"] < r["n_segments"] - 1 for r in runs)
    ok, mean, se = cf.unbiased_check(np.array([r["log_z_value"] for r in runs]),
                                     cf.crbd_log_z(tree, 4.0, 1.0))
    assert ok, (mean, se)


def test_ess_batch_equals_single_runs():
    from paper_2112_00364_gb300 import smc

    y = inputs.lg_observations(40, seed=8)
    tree = inputs.yule_tree(20, seed=9)
    models = [smc.Model("lg", obs=y), smc.Model("crbd", tree=tree), smc.Model("lg", obs=y)]
    specs = [dict(N=2000, seed=3, ess_threshold=0.5), dict(N=5000, seed=4, ess_threshold=0.6),
             dict(N=700, seed=5)]
    batch = smc.run_batch(models, specs, record_all_ancestors=True)
    for m, sp, b in zip(models, specs, batch):
        a = smc.run(m, sp["N"], sp["seed"], record_all_ancestors=True,
                    ess_threshold=sp.get("ess_threshold", 0.0))
        assert a["log_z_value"] == b["log_z_value"]
        np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
        np.testing.assert_array_equal(a["resampled"], b["resampled"])


def test_rateshift_fp32_ess_follows_oracle():
    tree = inputs.yule_tree(24, seed=3)
    g, o = run_pair("rateshift", 3000, 6, precision="fp32", tree=tree, sigma=0.3,
                    lam_stack_cap=tree.max_pending_right() + 1, ess_threshold=0.5)
    assert_parity_exact(g, o)
