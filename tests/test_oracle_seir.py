"""Pins for the oracle's SEIR model (Section 6.2, Listing 2) and its samplers.

  * Binomial(n, p): chi-square against the exact pmf, in the inversion range
    (n p < 10), the transformed-rejection range, for p > 1/2 (drawn as n minus
    the draw for 1 - p), and the degenerate cases;
  * Gamma(shape) (Marsaglia-Tsang) and Beta(a, b): Kolmogorov-Smirnov against
    scipy's distributions, for the shapes the model's priors use;
  * day 0's draws: the parameters against their Beta priors (KS), the initial
    human compartments (Poisson chi-square, uniform recovered count) and the
    log-uniform mosquito population;
  * a one-day run (one report at day 0): Z = sum_k P(hI = k) 1{y <= k} / (k + 1),
    the reporting probability integrated out under its uniform prior;
  * a two-day run (no report at day 0, one at day 1): z = hI + d with
    d ~ Binomial(hE, hDelta), so Z = sum_{k,e} P(hI = k) P(hE = e) sum_d
    BetaBinomial(d | e, a, b) 1{y <= k + d} / (k + d + 1) with hDelta's Beta(a, b)
    prior; mean Zhat / Z within 3 standard errors of 1 in both;
  * invariants of a full run: the human compartments sum to 7,370, every count
    is non-negative, every particle finishes;
  * the one-day transition law, particle by particle: two runs that never
    resample (ESS threshold below 1/N) end one day apart on the same draws, so
    every particle's state before and after day t is known.  Given the state
    before, each flow is a sum of independent binomials by binomial thinning
    (new exposed humans ~ Bin(hS, (1 - e^{-mI/hN}) hLambda), new infectious ~
    Bin(hE, hDelta), recoveries ~ Bin(hI, hGamma); mosquitoes: susceptible ~
    Bin(mS, (1 - pm) 6/7) + Bin(mN, 1/7) with pm = (1 - e^{-hI/hN}) mLambda,
    exposed ~ Bin(mE, (1 - mDelta) 6/7) + Bin(mS, pm 6/7), infectious ~
    Bin(mI, 6/7) + Bin(mE, mDelta 6/7)); the sums over particles of the
    standardised residuals and of their squares must match the exact first,
    second and fourth moments.  The unreported cases and the log-weight change
    exactly as the condition step says: z += new infectious, and on a report
    day the weight gains log Binomial(y | z, rho) (scipy) and z restarts at 0.
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


def test_day_zero_draws():
    """Day 0 of Listing 2: the six parameters from their Beta priors, hI - 1 and
    hE ~ Poisson(5), hR uniform on {0, ..., n - hI - hE}, hS the rest,
    floor(n 10^u) susceptible mosquitoes with u ~ U(-1, 2) and no others, the
    day's new infectious cases z = hI; a day without a report leaves the weight
    at 0."""
    N = 20_000
    r = oracle.smc_run("seir", N, 5, obs=np.array([-1.0]))
    assert r["status"] == 0 and r["log_z"] == 0.0
    assert np.all(r["final_logw"] == 0.0)
    th = r["real_fields"]
    priors = [(1.0, 1.0), (1 + 2 / 4.4, 3 - 2 / 4.4), (1 + 2 / 4.5, 3 - 2 / 4.5), (1.0, 1.0),
              (1 + 2 / 6.5, 3 - 2 / 6.5), (1.0, 1.0)]
    for k, (a, b) in enumerate(priors):
        assert stats.kstest(th[k], stats.beta(a, b).cdf).pvalue > 1e-4, k
    pc, hS, hE, hI, hR, mS, mE, mI, mR, z = r["int_fields"].astype(np.int64)
    assert np.all(pc == -1)
    for x in (hI - 1, hE):
        support = np.arange(int(x.max()) + 1)
        assert _chi2_pvalue(x, stats.poisson.pmf(support, 5.0), support) > 1e-4
    np.testing.assert_array_equal(hS, N_HUMANS - hE - hI - hR)
    assert np.all((hR >= 0) & (hR <= N_HUMANS - hI - hE))
    assert stats.kstest((hR + 0.5) / (N_HUMANS - hI - hE + 1), "uniform").pvalue > 1e-4
    # mS = floor(n 10^u): u lies within 1/(n/10) of log10(mS / n)
    u_hat = np.log10((mS + 0.5) / N_HUMANS)
    assert stats.kstest(u_hat, stats.uniform(-1.0, 3.0).cdf).pvalue > 1e-4
    assert np.all(mE == 0) and np.all(mI == 0) and np.all(mR == 0)
    np.testing.assert_array_equal(z, hI)


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


def _binom_moments(n, p):
    """mean, variance and fourth central moment of Binomial(n, p), elementwise"""
    n = np.asarray(n, dtype=float)
    p = np.asarray(p, dtype=float)
    v = n * p * (1.0 - p)
    return n * p, v, v * (1.0 + 3.0 * (n - 2.0) * p * (1.0 - p))


def _sum_moments(*parts):
    """moments of a sum of independent variables from their (mean, var, mu4)"""
    m = sum(q[0] for q in parts)
    v = sum(q[1] for q in parts)
    m4 = sum(q[2] for q in parts)
    for i in range(len(parts)):
        for j in range(i + 1, len(parts)):
            m4 = m4 + 6.0 * parts[i][1] * parts[j][1]
    return m, v, m4


def _check_flow(name, x, moments, n_sd=6.0):
    mean, var, mu4 = moments
    r = np.asarray(x, dtype=float) - mean
    fixed = var <= 0
    assert np.all(r[fixed] == 0), name  # a flow with no randomness is exact
    z1 = r.sum() / np.sqrt(var.sum())
    z2 = ((r * r).sum() - var.sum()) / np.sqrt(np.sum(mu4 - var * var))
    assert abs(z1) < n_sd and abs(z2) < n_sd, (name, z1, z2)


@pytest.mark.parametrize("day", [19, 20])  # day 20 carries a weekly report
def test_one_day_transition_law(day):
    y = inputs.seir_observations(day + 1, seed=7)
    assert (y[day] == -1) == (day == 19)
    N = 20_000
    before = oracle.smc_run("seir", N, 11, obs=y[:day], ess_threshold=1e-9)
    after = oracle.smc_run("seir", N, 11, obs=y[:day + 1], ess_threshold=1e-9)
    assert before["n_resamples"] == 0 and after["n_resamples"] == 0
    th = before["real_fields"]
    np.testing.assert_array_equal(th, after["real_fields"])  # drawn once, on day 0
    hS, hE, hI, hR, mS, mE, mI, mR, z = before["int_fields"][1:].astype(np.int64)
    hS1, hE1, hI1, hR1, mS1, mE1, mI1, mR1, z1 = after["int_fields"][1:].astype(np.int64)
    hN = hS + hE + hI + hR
    assert np.all(hS1 + hE1 + hI1 + hR1 == hN)
    assert np.all(mR == 0) and np.all(mR1 == 0)  # mosquitoes never recover
    dE = hS - hS1
    dR = hR1 - hR
    dI = hI1 - hI + dR
    s = 6.0 / 7.0
    _check_flow("new exposed humans", dE,
                _binom_moments(hS, (1.0 - np.exp(-mI / hN)) * th[0]))
    _check_flow("new infectious humans", dI, _binom_moments(hE, th[1]))
    _check_flow("recovered humans", dR, _binom_moments(hI, th[2]))
    pm = (1.0 - np.exp(-hI / hN)) * th[3]
    mN = mS + mE + mI + mR
    _check_flow("susceptible mosquitoes", mS1,
                _sum_moments(_binom_moments(mS, (1.0 - pm) * s), _binom_moments(mN, 1.0 / 7.0)))
    _check_flow("exposed mosquitoes", mE1,
                _sum_moments(_binom_moments(mE, (1.0 - th[4]) * s), _binom_moments(mS, pm * s)))
    _check_flow("infectious mosquitoes", mI1,
                _sum_moments(_binom_moments(mI, s), _binom_moments(mE, th[4] * s)))
    if y[day] == -1:
        np.testing.assert_array_equal(z1, z + dI)
        np.testing.assert_array_equal(after["final_logw"], before["final_logw"])
    else:
        assert np.all(z1 == 0)
        inc = stats.binom.logpmf(int(y[day]), z + dI, th[5])
        lw0, lw1 = before["final_logw"], after["final_logw"]
        live = np.isfinite(lw0)
        assert live.sum() > N // 10
        np.testing.assert_array_equal(np.isfinite(lw1[live]), np.isfinite(inc[live]))
        ok = live & np.isfinite(inc)
        np.testing.assert_allclose(lw1[ok] - lw0[ok], inc[ok], rtol=1e-9, atol=1e-9)
