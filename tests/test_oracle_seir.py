"""Pins for the oracle's SEIR model (Section 6.2, Listing 2) and its samplers.

  * Binomial(n, p): chi-square against the exact pmf, in the inversion range
    (n p < 10), the transformed-rejection range, for p > 1/2 (drawn as n minus
    the draw for 1 - p), and the degenerate cases;
  * Gamma(shape) (Marsaglia-Tsang) and Beta(a, b): Kolmogorov-Smirnov against
    scipy's distributions, for the shapes the model's priors use;
  * a one-day run (one report at day 0): Z = sum_k P(hI = k) 1{y <= k} / (k + 1),
    the reporting probability integrated out under its uniform prior;
  * a two-day run (no report at day 0, one at day 1): z = hI + d with
    d ~ Binomial(hE, hDelta), so Z = sum_{k,e} P(hI = k) P(hE = e) sum_d
    BetaBinomial(d | e, a, b) 1{y <= k + d} / (k + d + 1) with hDelta's Beta(a, b)
    prior; mean Zhat / Z within 3 standard errors of 1 in both;
  * invariants of a full run: the human compartments sum to 7,370, every count
    is non-negative, every particle finishes.
"""
import numpy as np
import pytest
from scipy import stats

import closed_forms as cf
import inputs
import oracle

N_HUMANS = 7370


def _chi2_pvalue(x, pmf_vals, support):
    counts = np.array([(x == k).sum() for k in support], dtype=float)
    exp = pmf_vals * len(x)
    # merge the tails so that every cell expects at least 5
    keep = exp >= 5
    obs_k, exp_k = list(counts[keep]), list(exp[keep])
    obs_k.append(len(x) - sum(obs_k))
    exp_k.append(len(x) - sum(exp_k))
    obs_k, exp_k = np.array(obs_k), np.array(exp_k)
    m = exp_k > 1e-9
    chi2 = (((obs_k - exp_k) ** 2)[m] / exp_k[m]).sum()
    return stats.chi2.sf(chi2, m.sum() - 1)


@pytest.mark.parametrize("n,p", [(20, 0.3), (40, 0.1), (1000, 0.02), (100, 0.4), (7370, 0.12),
                                 (300, 0.9), (50, 0.99), (5, 0.5)])
@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_binomial_exact_pmf(n, p, prec):
    x = oracle.sample("binomial", 200_000, n, p, seed=n + 1, precision=prec)
    assert np.all(x == np.round(x)) and x.min() >= 0 and x.max() <= n
    support = np.arange(n + 1)
    assert _chi2_pvalue(x, stats.binom.pmf(support, n, p), support) > 1e-3


def test_binomial_degenerate():
    for n, p, want in [(0, 0.4, 0), (50, 0.0, 0), (50, 1.0, 50), (1, 1e-300, 0)]:
        x = oracle.sample("binomial", 1000, n, p, seed=3)
        assert np.all(x == want)


@pytest.mark.parametrize("shape", [1.0, 1.0 + 2 / 4.4, 3 - 2 / 4.4, 10.0])
def test_gamma_marsaglia_tsang(shape):
    x = oracle.sample("gamma", 100_000, shape, seed=11)
    assert stats.kstest(x, stats.gamma(shape).cdf).pvalue > 1e-3


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1 + 2 / 4.4, 3 - 2 / 4.4), (1 + 2 / 6.5, 3 - 2 / 6.5)])
def test_beta(a, b):
    x = oracle.sample("beta", 100_000, a, b, seed=13)
    assert stats.kstest(x, stats.beta(a, b).cdf).pvalue > 1e-3


def _many(N, obs, seeds):
    out = []
    for s in seeds:
        r = oracle.smc_run("seir", N, s, obs=obs)
        assert r["status"] == 0
        out.append(r["log_z"])
    return np.array(out)


def test_one_day_closed_form():
    y0 = 4
    k = np.arange(1, 80)
    pk = stats.poisson.pmf(k - 1, 5.0)
    Z = float((pk * (y0 <= k) / (k + 1)).sum())
    lz = _many(500, np.array([float(y0)]), range(1, 101))
    ok, mean, se = cf.unbiased_check(lz, np.log(Z))
    assert ok, (mean, se)


def test_two_day_closed_form():
    y1 = 7
    a, b = 1 + 2 / 4.4, 3 - 2 / 4.4
    Z = 0.0
    for k in range(1, 60):
        pk = stats.poisson.pmf(k - 1, 5.0)
        for e in range(0, 60):
            pe = stats.poisson.pmf(e, 5.0)
            d = np.arange(e + 1)
            bb = stats.betabinom.pmf(d, e, a, b)
            Z += pk * pe * float((bb * (y1 <= k + d) / (k + d + 1)).sum())
    lz = _many(2000, np.array([-1.0, float(y1)]), range(1, 101))
    ok, mean, se = cf.unbiased_check(lz, np.log(Z))
    assert ok, (mean, se)


def test_full_run_invariants():
    y = inputs.seir_observations(84, seed=7)
    r = oracle.smc_run("seir", 600, 3, obs=y)
    assert r["status"] == 0 and r["n_segments"] == 84 and np.isfinite(r["log_z"])
    f = r["int_fields"]
    assert np.all(f[0] == -1)  # every particle at b_stop
    np.testing.assert_array_equal(f[1] + f[2] + f[3] + f[4], N_HUMANS)
    assert f[1:].min() >= 0
    th = r["real_fields"]
    assert np.all((th > 0) & (th < 1))
