"""CRBD with static delayed sampling on the GPU (Section 6.3).

The two predictive samplers against the oracle's, draw by draw on the same
Philox counters; runs against the oracle in follow mode (FP64 element-wise, FP32
to single-precision rounding, with and without ESS-triggered resampling); the
GPU estimate unbiased against the 2-D quadrature of the closed-form likelihood
over the priors; and the workload of the benchmark (128-tip tree, N = 100,000,
ESS threshold 0.5) in full against the oracle, plus its bookkeeping invariants.
"""
import numpy as np
import pytest

import closed_forms as cf
import inputs
import oracle
from parity import assert_parity_exact, assert_parity_fp64, run_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("alpha,ratio", [(1.0, 0.5), (3.5, 2.0), (1.0, 9.0), (2.0, 8.0),
                                         (20.0, 0.9)])
def test_negative_binomial_matches_oracle(alpha, ratio, prec):
    from paper_2112_00364_gb300 import smc

    g, gb = smc.sample("neg_binomial", 200_000, alpha, ratio, seed=31, precision=prec)
    g, gb = g.cpu().numpy(), gb.cpu().numpy()
    o, ob = oracle.sample("neg_binomial", 200_000, alpha, ratio, seed=31, return_blocks=True,
                          precision=oracle.FP64 if prec == "fp64" else oracle.FP32)
    diff = g != o
    if prec == "fp32":  # the same single-precision operations on both sides
        assert diff.sum() == 0
    assert diff.mean() < 1e-5, diff.sum()
    np.testing.assert_array_equal(gb[~diff], ob[~diff])


@pytest.mark.parametrize("alpha,beta", [(1.0, 2.0), (4.0, 1.5), (30.0, 12.0)])
def test_lomax_matches_oracle(alpha, beta):
    from paper_2112_00364_gb300 import smc

    g, gb = smc.sample("lomax", 100_000, alpha, beta, seed=33)
    g, gb = g.cpu().numpy(), gb.cpu().numpy()
    o, ob = oracle.sample("lomax", 100_000, alpha, beta, seed=33, return_blocks=True)
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_allclose(g, o, rtol=1e-13, atol=0)


@pytest.mark.parametrize("tips,N,seed", [(16, 1000, 1), (32, 4097, 2), (8, 300, 3)])
def test_crbd_ds_parity(tips, N, seed):
    tree = inputs.yule_tree(tips, seed=seed)
    g, o = run_pair("crbd_ds", N, seed, tree=tree)
    assert_parity_fp64(g, o)


def test_crbd_ds_ess_parity():
    tree = inputs.yule_tree(32, seed=4)
    g, o = run_pair("crbd_ds", 3001, 5, tree=tree, ess_threshold=0.5)
    assert 0 < g["n_resamples"] < g["n_segments"] - 1
    assert_parity_fp64(g, o)


def test_crbd_ds_fp32_follows_oracle():
    tree = inputs.yule_tree(32, seed=3)
    g, o = run_pair("crbd_ds", 4000, 5, precision="fp32", tree=tree)
    assert_parity_exact(g, o)
    g, o = run_pair("crbd_ds", 3001, 6, precision="fp32", tree=tree, ess_threshold=0.5)
    assert_parity_exact(g, o)


def test_crbd_ds_gpu_unbiased_vs_quadrature():
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(8, seed=4)
    m = smc.Model("crbd_ds", tree=tree)
    lz = np.array([smc.run(m, 4096, seed=s)["log_z_value"] for s in range(1, 101)])
    m.close()
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_marginal_log_z(tree))
    assert ok, (mean, se)


def test_crbd_ds_rejects_fixed_rates():
    from paper_2112_00364_gb300 import smc

    with pytest.raises(Exception):
        smc.Model("crbd_ds", tree=inputs.yule_tree(8, seed=4), rates=(1.0, 0.5))


def test_crbd_ds_benchmark_workload_parity():
    """The benchmark's workload (128-tip Yule tree, N = 100,000, ESS-triggered
    resampling at 0.5) in full against the oracle in follow mode, and the
    posterior bookkeeping of its final particles."""
    tree = inputs.yule_tree(128, seed=6)
    g, o = run_pair("crbd_ds", 100_000, 1, tree=tree, ess_threshold=0.5)
    assert_parity_fp64(g, o)
    a_l, b_l, a_m, b_m = g["real_fields"]
    alive = np.isfinite(g["final_logw"])
    par, age = np.asarray(tree.parent), np.asarray(tree.age)
    nonroot = np.flatnonzero(par >= 0)
    length = float(np.sum(age[par[nonroot]] - age[nonroot]))
    n_int = int(np.sum(np.asarray(tree.left)[nonroot] >= 0))
    assert np.all(a_l[alive] == np.round(a_l[alive])) and np.all(a_l[alive] >= 1 + n_int)
    assert np.all(b_l[alive] >= 1.0 + length * (1 - 1e-12))
    assert np.all(b_m[alive] >= 2.0 + length * (1 - 1e-12))
