"""Full SMC runs through the C ABI vs the oracle, element by element (GPU).

Sizes span several 256-particle tiles with a ragged last tile, plus the full
linear-Gaussian (N=1024, T=50) and CRBD (64-tip tree, N=2^16) workloads in the
launch configuration the benchmark times.
"""

import numpy as np
import pytest

import closed_forms as cf
import inputs
from parity import assert_parity_fp64, run_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [1, 2, 255, 257, 1024, 3001])
def test_lg_parity(N):
    y = inputs.lg_observations(50, seed=1)
    g, o = run_pair("lg", N, seed=7, obs=y)
    assert_parity_fp64(g, o)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lg_full_config_parity(seed):
    y = inputs.lg_observations(50, seed=1)
    g, o = run_pair("lg", 1024, seed=seed, obs=y)
    assert_parity_fp64(g, o)


@pytest.mark.parametrize("N,seed", [(1, 1), (300, 2), (2049, 3), (5000, 4)])
def test_crbd_parity_small_tree(N, seed):
    tree = inputs.yule_tree(16, seed=2)
    g, o = run_pair("crbd", N, seed=seed, tree=tree)
    assert_parity_fp64(g, o)


def test_crbd_fixed_rates_parity():
    tree = inputs.yule_tree(24, seed=5)
    g, o = run_pair("crbd", 4099, seed=11, tree=tree, rates=(3.0, 1.5))
    assert_parity_fp64(g, o)


def test_crbd_full_config_parity():
    # 64-tip tree, N = 2^16, FP64, priors: the benchmark workload
    tree = inputs.yule_tree(64, seed=2)
    g, o = run_pair("crbd", 1 << 16, seed=1, tree=tree)
    assert_parity_fp64(g, o)
    assert g["n_segments"] == 127 and g["n_resamples"] == 126


@pytest.mark.parametrize("kind", ["lg", "crbd"])
def test_large_population_parity(kind):
    """N = 300,001: 1,172 tiles of 256, more than a CTA combines for itself, so
    the run's last tile of each segment forms the offsets for the next wave."""
    if kind == "lg":
        g, o = run_pair("lg", 300_001, seed=5, obs=inputs.lg_observations(12, seed=3))
    else:
        g, o = run_pair("crbd", 300_001, seed=5, tree=inputs.yule_tree(6, seed=4))
    assert_parity_fp64(g, o)


def test_crbd_kill_rules_parity():
    tree = inputs.yule_tree(8, seed=8)
    g, o = run_pair("crbd", 2000, seed=3, tree=tree, rates=(6.0, 5.0), depth_cap=2)
    assert o["n_overflow"] > 0
    assert_parity_fp64(g, o)
    g, o = run_pair("crbd", 2000, seed=3, tree=tree, rates=(6.0, 5.0), call_limit=3)
    assert o["n_limit"] > 0
    assert_parity_fp64(g, o)


def test_geometric_parity_divergent_termination():
    g, o = run_pair("geometric", 3000, seed=5)
    assert g["n_segments"] > 3
    assert_parity_fp64(g, o)


def test_rateshift_fp64_parity():
    tree = inputs.yule_tree(32, seed=3)
    cap = tree.max_pending_right() + 1
    g, o = run_pair("rateshift", 2500, seed=4, tree=tree, sigma=0.3, lam_stack_cap=cap)
    assert_parity_fp64(g, o)
    np.testing.assert_allclose(g["stack"], o["stack"], rtol=1e-12, atol=0)


def test_crbd_gpu_unbiased_vs_closed_form():
    # unbiasedness at the benchmark size: 100 seeds, 64-tip tree, N = 2^16, fixed rates
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(64, seed=2)
    lam, mu = 4.0, 1.0
    m = smc.Model("crbd", tree=tree, rates=(lam, mu))
    lz = [smc.run(m, 1 << 16, seed=s)["log_z_value"] for s in range(1, 101)]
    ok, mean, se = cf.unbiased_check(np.array(lz), cf.crbd_log_z(tree, lam, mu))
    assert ok, (mean, se)


def test_lg_gpu_unbiased_vs_kalman():
    from paper_2112_00364_gb300 import smc

    y = inputs.lg_observations(50, seed=1)
    m = smc.Model("lg", obs=y)
    lz = [smc.run(m, 1024, seed=s)["log_z_value"] for s in range(1, 101)]
    ok, mean, se = cf.unbiased_check(np.array(lz), cf.kalman_loglik(y))
    assert ok, (mean, se)


def test_device_outputs_match_host_outputs():
    import torch
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(16, seed=2)
    m = smc.Model("crbd", tree=tree)
    h = smc.run(m, 3000, seed=9, record_all_ancestors=True)
    d = smc.run(m, 3000, seed=9, record_all_ancestors=True, where="device")
    torch.cuda.synchronize()
    assert float(d["log_z"].cpu()[0]) == h["log_z_value"]
    np.testing.assert_array_equal(d["ancestors"].cpu().numpy(), h["ancestors"])
    np.testing.assert_array_equal(d["real_fields"].cpu().numpy(), h["real_fields"])


def test_step_limit_status():
    from paper_2112_00364_gb300 import smc

    m = smc.Model("geometric")
    r = smc.run(m, 512, seed=1, max_segments=2)
    assert r["status"] == smc.ESTEPLIMIT
