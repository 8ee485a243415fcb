"""Exact quantities that pin the oracle (test infrastructure).

Each function here is an *independent* route to a number the SMC estimate
must be unbiased for; none of them runs SMC.

* Kalman filter: exact log p(y_1:T) of the linear-Gaussian model (the Eq. 2
  family used by Fig. 3).
* CRBD at fixed rates: the likelihood of Listing 1's model in closed form.
  The hidden-lineage simulation (crbdGoesUndetected / simBranch) makes each
  branch contribute E[exp(lnProb1 + lnProb3)] = p1(t_parent) / p1(t_child),
  with p1 the standard birth-death "one sampled descendant" probability, so
  the product over branches telescopes.
* A brute-force route for the same branch factor that does not use p1: the
  extinction probability from an RK4 solve of its ODE and an explicit sum
  over the Poisson number of hidden events.
* mu = 0 special case: every hidden lineage survives to the present and is
  detected (rho = 1), so the likelihood is just P(no hidden events).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special, stats


# ----------------------------- Kalman ---------------------------------
def kalman_filter(y, a=0.9, b=0.0, q_sd=1.0, r_sd=0.5, x0_mean=0.0, x0_sd=1.0):
    """log p(y_1..T) and the mean and variance of p(x_T | y_1..T)."""
    m, P = x0_mean, x0_sd ** 2
    ll = 0.0
    for yt in y:
        m = a * m + b
        P = a * a * P + q_sd ** 2
        S = P + r_sd ** 2
        ll += stats.norm.logpdf(yt, loc=m, scale=math.sqrt(S))
        K = P / S
        m = m + K * (yt - m)
        P = (1.0 - K) * P
    return float(ll), float(m), float(P)


def kalman_loglik(y, a=0.9, b=0.0, q_sd=1.0, r_sd=0.5, x0_mean=0.0, x0_sd=1.0) -> float:
    return kalman_filter(y, a, b, q_sd, r_sd, x0_mean, x0_sd)[0]


# ------------------------ birth-death closed form ----------------------
def log_p1(t, lam, mu, rho=1.0):
    """log of p1(t) = rho r^2 e^{-rt} / (rho lam + (lam(1-rho) - mu) e^{-rt})^2,
    written as rho e^{-rt} / (rho lam g + e^{-rt})^2 with g = (1 - e^{-rt}) / r
    (g = t at r = 0) so that lam = mu needs no special case."""
    t = np.asarray(t, dtype=np.float64)
    r = lam - mu
    if abs(r) < 1e-300:
        g = t
    else:
        g = -np.expm1(-r * t) / r
    e = np.exp(-r * t)
    return math.log(rho) - r * t - 2.0 * np.log(rho * lam * g + e)


def crbd_corr(n_tips: int) -> float:
    return (n_tips - 1) * math.log(2.0) - special.gammaln(n_tips + 1)


def crbd_log_z(tree, lam, mu, rho=1.0) -> float:
    """Exact log-likelihood of Listing 1's CRBD model at fixed (lam, mu)."""
    n = tree.n_tips
    tot = crbd_corr(n)
    for v in range(1, tree.n_nodes):
        p = tree.parent[v]
        tot += float(log_p1(tree.age[p], lam, mu, rho) - log_p1(tree.age[v], lam, mu, rho))
        tot += math.log(lam) if tree.left[v] >= 0 else math.log(rho)
    return tot


def crbd_log_z_rates(tree, lam_branch, mu, rho=1.0) -> float:
    """Same model with a per-branch birth rate lam_branch[v] (v = child node)."""
    tot = crbd_corr(tree.n_tips)
    for v in range(1, tree.n_nodes):
        p = tree.parent[v]
        lv = lam_branch[v]
        tot += float(log_p1(tree.age[p], lv, mu, rho) - log_p1(tree.age[v], lv, mu, rho))
        tot += math.log(lv) if tree.left[v] >= 0 else math.log(rho)
    return tot


def crbd_log_z_mu0(tree, lam) -> float:
    """mu = 0, rho = 1: Z = e^{corr} lam^{n-2} exp(-lam * total branch length)."""
    L = sum(tree.age[tree.parent[v]] - tree.age[v] for v in range(1, tree.n_nodes))
    return crbd_corr(tree.n_tips) + (tree.n_tips - 2) * math.log(lam) - lam * L


def crbd_log_z_depth1(tree, lam, mu) -> float:
    """rho = 1 and a hidden-lineage depth cap of 1: a lineage started on an
    observed branch may not itself speciate (its first event would be a call at
    depth 2, which kills the particle), so it must die before the present with
    no event: q(t) = int_0^t mu e^{-(lam + mu) s} ds for a lineage born t before
    the present.  With Poisson(lam dt) events uniform on a branch [stop, start]
    each weighted 2 q(t), the branch factor is
    e^{-mu dt} exp(-lam dt + 2 lam int_stop^start q(t) dt)."""
    r = lam + mu
    tot = crbd_corr(tree.n_tips)
    for v in range(tree.n_nodes):
        p = tree.parent[v]
        if p < 0:
            continue
        start, stop = float(tree.age[p]), float(tree.age[v])
        dt = start - stop
        int_q = mu / r * (dt - (math.exp(-r * stop) - math.exp(-r * start)) / r)
        tot += -mu * dt - lam * dt + 2.0 * lam * int_q
        if tree.left[v] >= 0:
            tot += math.log(lam)
    return tot


def extinction_rk4(lam, mu, rho, t_lo, t_hi, steps=4000):
    """E(t) = P(a lineage alive at age t leaves no sampled descendant):
    dE/dt = mu - (lam + mu) E + lam E^2, E(0) = 1 - rho, integrated by RK4
    together with I(t) = int_{t_lo}^t E.  Returns I(t_hi)."""
    def f(y):
        e = y[0]
        return np.array([mu - (lam + mu) * e + lam * e * e, e])

    y = np.array([1.0 - rho, 0.0])
    # first run to t_lo (no integral), then integrate over the branch
    for a, b in ((0.0, t_lo), (t_lo, t_hi)):
        if b <= a:
            continue
        h = (b - a) / steps
        for _ in range(steps):
            k1 = f(y)
            k2 = f(y + 0.5 * h * k1)
            k3 = f(y + 0.5 * h * k2)
            k4 = f(y + h * k3)
            y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if b == t_lo:
            y[1] = 0.0  # the integral starts at the branch's lower end
    return y[1]


def branch_factor_bruteforce(lam, mu, rho, t_lo, t_hi) -> float:
    """E[exp(lnProb1 + lnProb3)] for one observed branch from age t_hi down to
    t_lo: e^{-mu dt} * sum_k Pois(k; lam dt) (2 pbar0)^k, where pbar0 is the
    mean extinction probability over the branch (events are uniform on it)."""
    dt = t_hi - t_lo
    pbar0 = extinction_rk4(lam, mu, rho, t_lo, t_hi, steps=2000) / dt
    m = lam * dt
    tot = 0.0
    k = 0
    while True:
        term = stats.poisson.pmf(k, m) * (2.0 * pbar0) ** k
        tot += term
        if k > m and term < 1e-18 * max(tot, 1e-300):
            break
        k += 1
    return math.exp(-mu * dt) * tot


def crbd_marginal_log_z(tree, rho=1.0, lambda_scale=1.0, mu_scale=0.5) -> float:
    """log of the integral of Z(lam, mu) against the Gamma(1, scale) priors,
    by adaptive 2-D quadrature in (lam, mu)."""
    ref = crbd_log_z(tree, 1.0, 0.5, rho)

    def f(mu, lam):
        lz = crbd_log_z(tree, lam, mu, rho) - ref
        return math.exp(lz - lam / lambda_scale - mu / mu_scale) / (lambda_scale * mu_scale)

    val, err = integrate.dblquad(f, 0.0, 60.0 * lambda_scale, 0.0, 60.0 * mu_scale,
                                 epsabs=0.0, epsrel=1e-9)
    return ref + math.log(val)


def unbiased_check(log_zhat, log_z, n_se=3.0):
    """For an unbiased estimator Zhat of Z: mean(Zhat / Z) is within n_se
    standard errors of 1.  Returns (ok, mean, se)."""
    ratio = np.exp(np.asarray(log_zhat) - log_z)
    mean = float(ratio.mean())
    se = float(ratio.std(ddof=1) / math.sqrt(len(ratio)))
    return abs(mean - 1.0) <= n_se * se + 1e-12, mean, se
