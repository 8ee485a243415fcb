"""Pins for the oracle's delayed-sampling CRBD (Section 6.3: CRBD with the
rates' Gamma priors integrated out) and its two predictive samplers.

  * negative binomial (Poisson(lambda tau) with lambda ~ Gamma(alpha, rate beta)
    integrated out): chi-square against scipy's nbinom pmf in the inversion
    range (mean below 10) and in the Gamma-Poisson mixture range;
  * Lomax (Exponential(mu) with mu ~ Gamma(alpha, rate beta) integrated out):
    Kolmogorov-Smirnov against scipy's lomax;
  * the model estimates the same marginal likelihood as the plain CRBD with
    its Gamma priors: mean Zhat / Z within 3 standard errors of 1 against the
    2-D quadrature of the closed-form CRBD likelihood over the priors, on an
    8-tip and on a 2-tip tree;
  * integrating the rates out lowers the variance of log Zhat against the
    plain model at the same N;
  * the same with a general rate (exposure 1): chi-square against nbinom with
    p = beta / (beta + 1), in both ranges;
  * the quadrature check also with rho = 1/2 and with other prior scales;
  * posterior bookkeeping: every finished particle's shapes are integers,
    a_lambda >= 1 + the internal non-root nodes, and b_lambda - 1/s_lambda and
    b_mu - 1/s_mu both count every observed branch length once (>= the tree
    length, equal for a particle that drew no hidden lineage); with rho = 1
    a_mu - 1 = a_lambda - 1 - (internal non-root nodes) (one hidden lineage per
    hidden speciation) and b_mu - 1/s_mu = b_lambda - 1/s_lambda (every hidden
    lifetime ended before the present and counts once in each).
"""
import math

import numpy as np
import pytest
from scipy import stats

import closed_forms as cf
import inputs
import oracle


def _chi2_pvalue(x, pmf_vals, support):
    counts = np.array([(x == k).sum() for k in support], dtype=float)
    exp = pmf_vals * len(x)
    keep = exp >= 5
    obs_k, exp_k = list(counts[keep]), list(exp[keep])
    obs_k.append(len(x) - sum(obs_k))
    exp_k.append(len(x) - sum(exp_k))
    obs_k, exp_k = np.array(obs_k), np.array(exp_k)
    m = exp_k > 1e-9
    chi2 = (((obs_k - exp_k) ** 2)[m] / exp_k[m]).sum()
    return stats.chi2.sf(chi2, m.sum() - 1)


@pytest.mark.parametrize("alpha,ratio", [(1.0, 0.5), (3.5, 2.0), (1.0, 9.0), (7.0, 0.05),
                                         (2.0, 8.0), (20.0, 0.9), (1.0, 40.0)])
@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_negative_binomial_exact_pmf(alpha, ratio, prec):
    # beta = 1, tau = ratio: p = 1 / (1 + ratio), mean alpha ratio
    x = oracle.sample("neg_binomial", 200_000, alpha, ratio, seed=int(alpha * 10 + ratio * 7),
                      precision=prec)
    assert np.all(x == np.round(x)) and x.min() >= 0
    p = 1.0 / (1.0 + ratio)
    support = np.arange(int(x.max()) + 1)
    assert _chi2_pvalue(x, stats.nbinom.pmf(support, alpha, p), support) > 1e-3


@pytest.mark.parametrize("alpha,beta", [(3.0, 2.0), (1.0, 0.25), (30.0, 0.5), (2.0, 0.1)])
def test_negative_binomial_rate_exact_pmf(alpha, beta):
    # exposure 1, rate beta: p = beta / (beta + 1), mean alpha / beta (inversion
    # below 10, the Gamma-Poisson mixture from 10 up)
    x = oracle.sample("neg_binomial_rate", 200_000, alpha, beta, seed=int(alpha * 3 + beta * 11))
    assert np.all(x == np.round(x)) and x.min() >= 0
    support = np.arange(int(x.max()) + 1)
    pmf = stats.nbinom.pmf(support, alpha, beta / (beta + 1.0))
    assert _chi2_pvalue(x, pmf, support) > 1e-3


@pytest.mark.parametrize("alpha,beta", [(1.0, 2.0), (1.0, 0.3), (4.0, 1.5), (30.0, 12.0)])
def test_lomax_ks(alpha, beta):
    x = oracle.sample("lomax", 100_000, alpha, beta, seed=int(alpha + 13 * beta))
    assert x.min() > 0
    assert stats.kstest(x, stats.lomax(c=alpha, scale=beta).cdf).pvalue > 1e-3


def _many(kind, N, seeds, **params):
    return np.array([oracle.smc_run(kind, N, seed=s, **params)["log_z"] for s in seeds])


# Zhat / Z is right-skewed, so 100 seeds can understate its standard error;
# the rho = 1/2 case with internal nodes takes 400
@pytest.mark.parametrize("tips,tree_seed,N,rho,ls,ms,n_seeds", [(8, 4, 4096, 1.0, 1.0, 0.5, 100),
                                                             (2, 0, 512, 1.0, 1.0, 0.5, 100),
                                                             (2, 0, 512, 0.5, 2.0, 0.25, 100),
                                                             (4, 1, 1024, 0.5, 1.0, 0.5, 400)])
def test_crbd_ds_unbiased_vs_quadrature(tips, tree_seed, N, rho, ls, ms, n_seeds):
    tree = inputs.two_tip_tree(1.0) if tips == 2 else inputs.yule_tree(tips, seed=tree_seed)
    lz = _many("crbd_ds", N, range(1, n_seeds + 1), tree=tree, rho=rho, lambda_scale=ls,
               mu_scale=ms)
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_marginal_log_z(tree, rho, ls, ms))
    assert ok, (mean, se)


def test_crbd_ds_lowers_log_z_variance():
    tree = inputs.yule_tree(8, seed=4)
    ds = _many("crbd_ds", 1024, range(1, 41), tree=tree)
    plain = _many("crbd", 1024, range(101, 141), tree=tree)
    assert ds.var(ddof=1) < plain.var(ddof=1), (ds.var(ddof=1), plain.var(ddof=1))


@pytest.mark.parametrize("ls,ms", [(1.0, 0.5), (2.0, 0.25)])
def test_crbd_ds_posterior_bookkeeping(ls, ms):
    tree = inputs.yule_tree(16, seed=5)
    r = oracle.smc_run("crbd_ds", 4096, seed=3, tree=tree, lambda_scale=ls, mu_scale=ms)
    assert r["status"] == 0 and np.all(r["int_fields"][0] == -1)
    # at these rates no hidden recursion comes near the depth cap (64) or the
    # call limit (65,536 calls per branch)
    assert r["n_overflow"] == 0 and r["n_limit"] == 0
    a_l, b_l, a_m, b_m = r["real_fields"]
    par = np.asarray(tree.parent)
    age = np.asarray(tree.age)
    nonroot = np.flatnonzero(par >= 0)
    length = float(np.sum(age[par[nonroot]] - age[nonroot]))
    n_internal_nonroot = int(np.sum(np.asarray(tree.left)[nonroot] >= 0))
    alive = np.isfinite(r["final_logw"])
    assert alive.any()
    for a in (a_l[alive], a_m[alive]):
        assert np.all(a == np.round(a))
    assert np.all(a_l[alive] >= 1 + n_internal_nonroot)
    assert np.all(a_m[alive] >= 1)
    assert np.all(b_l[alive] >= 1 / ls + length * (1 - 1e-12))
    assert np.all(b_m[alive] >= 1 / ms + length * (1 - 1e-12))
    # a particle with no hidden lineage (a_mu = 1) added exactly the tree's
    # branch lengths to both rates, and a_lambda = 1 + internal nodes
    none = alive & (a_m == 1.0)
    assert none.any()
    np.testing.assert_allclose(b_l[none], 1 / ls + length, rtol=1e-12)
    np.testing.assert_allclose(b_m[none], 1 / ms + length, rtol=1e-12)
    assert np.all(a_l[none] == 1 + n_internal_nonroot)
    # every hidden speciation event starts one hidden lineage, whose lifetime
    # is drawn once (a_mu += 1); with rho = 1 a surviving particle's hidden
    # lineages all ended before the present, so each added the same lifetime
    # to b_mu and, as its exposure, to b_lambda
    some = alive & (a_m > 1.0)
    assert some.any()
    np.testing.assert_array_equal(a_m[alive] - 1, a_l[alive] - 1 - n_internal_nonroot)
    np.testing.assert_allclose(b_m[alive] - 1 / ms, b_l[alive] - 1 / ls, rtol=1e-12)


def test_crbd_ds_rejects_fixed_rates():
    tree = inputs.yule_tree(8, seed=4)
    r = oracle.smc_run("crbd_ds", 64, seed=1, tree=tree, rates=(1.0, 0.5))
    assert r["status"] == oracle.EINVAL


def test_crbd_ds_fp32_close_to_fp64():
    tree = inputs.yule_tree(8, seed=4)
    lz64 = oracle.smc_run("crbd_ds", 4096, seed=9, tree=tree)["log_z"]
    lz32 = oracle.smc_run("crbd_ds", 4096, seed=9, tree=tree, precision=oracle.FP32)["log_z"]
    assert math.isfinite(lz32) and abs(lz32 - lz64) < 0.5
