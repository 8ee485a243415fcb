"""The closed forms that pin the oracle, checked against independent routes
(CPU only): brute-force numerical integration for the Kalman likelihood, an
RK4 + Poisson-sum computation for the birth-death branch factor, the
mu = 0 special case, and a direct simulation for the depth-capped branch
factor."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import closed_forms as cf
import inputs


def test_kalman_matches_numerical_integration_T2():
    y = np.array([0.7, -0.4])
    a, q, r, s0 = 0.9, 1.0, 0.5, 1.0
    # p(y1, y2) = int int int N(x0;0,s0) N(x1; a x0, q) N(y1; x1, r) N(x2; a x1, q) N(y2; x2, r)
    # integrate x0 and x2 analytically-free by nesting 1-D quadratures on x1 only:
    # p(y1,y2) = int N(x1; 0, a^2 s0^2 + q^2) N(y1; x1, r) N(y2; a x1, q^2 + r^2) dx1
    f = lambda x1: (stats.norm.pdf(x1, 0, math.sqrt(a * a * s0 * s0 + q * q))
                    * stats.norm.pdf(y[0], x1, r)
                    * stats.norm.pdf(y[1], a * x1, math.sqrt(q * q + r * r)))
    val, _ = integrate.quad(f, -30, 30, epsabs=0, epsrel=1e-12)
    assert abs(cf.kalman_loglik(y, a=a, q_sd=q, r_sd=r, x0_sd=s0) - math.log(val)) < 1e-9


def test_kalman_filter_moments_match_numerical_integration_T2():
    """Mean and variance of p(x2 | y1, y2) by 2-D integration over (x1, x2) of
    N(x1; 0, a^2 s0^2 + q^2) N(y1; x1, r) N(x2; a x1, q) N(y2; x2, r): the
    trapezoid rule on a fine grid, spectrally accurate for this smooth,
    Gaussian-decaying integrand."""
    y = np.array([0.7, -0.4])
    a, q, r, s0 = 0.9, 1.0, 0.5, 1.0
    g = np.linspace(-12.0, 12.0, 2401)
    h = g[1] - g[0]
    x1, x2 = np.meshgrid(g, g, indexing="ij")
    joint = (stats.norm.pdf(x1, 0, math.sqrt(a * a * s0 * s0 + q * q))
             * stats.norm.pdf(y[0], x1, r) * stats.norm.pdf(x2, a * x1, q)
             * stats.norm.pdf(y[1], x2, r))
    mom = [float((x2 ** k * joint).sum() * h * h) for k in range(3)]
    mean = mom[1] / mom[0]
    var = mom[2] / mom[0] - mean * mean
    ll, m, P = cf.kalman_filter(y, a=a, q_sd=q, r_sd=r, x0_sd=s0)
    assert abs(ll - math.log(mom[0])) < 1e-8
    assert abs(m - mean) < 1e-8 and abs(P - var) < 1e-8


@pytest.mark.parametrize("lam,mu,rho", [(2.0, 0.5, 1.0), (1.0, 1.0, 1.0), (0.7, 1.9, 1.0),
                                        (3.0, 1.0, 0.5)])
def test_branch_factor_closed_form_vs_bruteforce(lam, mu, rho):
    for lo, hi in [(0.0, 1.0), (0.3, 0.8)]:
        bf = cf.branch_factor_bruteforce(lam, mu, rho, lo, hi)
        closed = math.exp(float(cf.log_p1(hi, lam, mu, rho) - cf.log_p1(lo, lam, mu, rho)))
        assert abs(bf - closed) < 1e-10 * max(1.0, closed), (lo, hi, bf, closed)


@pytest.mark.parametrize("lam,mu,rho", [(2.0, 0.5, 1.0), (1.2, 1.2, 1.0), (3.0, 1.0, 0.5)])
def test_two_tip_likelihood(lam, mu, rho):
    tree = inputs.two_tip_tree(1.0)
    lz = cf.crbd_log_z(tree, lam, mu, rho)
    brute = 2 * math.log(rho) + 2 * math.log(cf.branch_factor_bruteforce(lam, mu, rho, 0.0, 1.0))
    assert abs(lz - brute) < 1e-9


def test_mu_zero_special_case():
    tree = inputs.yule_tree(12, seed=5)
    for lam in (0.5, 2.0, 4.0):
        assert abs(cf.crbd_log_z(tree, lam, 0.0) - cf.crbd_log_z_mu0(tree, lam)) < 1e-9
    # the two-tip instance: Z = exp(-2 lam t_root)
    t2 = inputs.two_tip_tree(0.8)
    assert abs(cf.crbd_log_z_mu0(t2, 1.7) - (-2 * 1.7 * 0.8)) < 1e-12


def test_depth_one_branch_factor_vs_simulation():
    """crbd_log_z_depth1's branch factor against a direct simulation of the
    hidden events on one branch with numpy's generator: Poisson(lam dt) events
    uniform on the branch, each starting a lineage with an Exp(mu) lifetime that
    must end before the present and hold no Poisson(lam x) event of its own."""
    lam, mu, start, stop = 2.0, 1.3, 0.9, 0.35
    rng = np.random.Generator(np.random.PCG64(17))
    M = 400_000
    n = rng.poisson(lam * (start - stop), size=M)
    fac = np.exp(-mu * (start - stop)) * np.ones(M)
    for k in range(1, int(n.max()) + 1):
        sel = n >= k
        t = rng.uniform(stop, start, size=sel.sum())
        x = rng.exponential(1.0 / mu, size=sel.sum())
        ok = (x < t) & (rng.poisson(lam * np.minimum(x, t)) == 0)
        fac[sel] *= np.where(ok, 2.0, 0.0)
    r = lam + mu
    int_q = mu / r * ((start - stop) - (math.exp(-r * stop) - math.exp(-r * start)) / r)
    exact = math.exp(-(lam + mu) * (start - stop) + 2 * lam * int_q)
    assert abs(fac.mean() - exact) < 4 * fac.std() / math.sqrt(M)
    # the two-tip tree (root age `start`): corr + two branches from the root to 0
    tree = inputs.two_tip_tree(start)
    int_q0 = mu / r * (start - (1.0 - math.exp(-r * start)) / r)
    lz = cf.crbd_corr(2) + 2 * (-(lam + mu) * start + 2 * lam * int_q0)
    assert abs(cf.crbd_log_z_depth1(tree, lam, mu) - lz) < 1e-12


def test_lambda_equals_mu_is_continuous():
    tree = inputs.yule_tree(8, seed=6)
    a = cf.crbd_log_z(tree, 1.5, 1.5)
    b = cf.crbd_log_z(tree, 1.5, 1.5 - 1e-7)
    assert abs(a - b) < 1e-5


def test_yule_tree_shape():
    for n in (2, 3, 16, 64, 256):
        t = inputs.yule_tree(n, seed=n)
        assert t.n_nodes == 2 * n - 1 and t.n_tips == n
        assert abs(t.age[0] - 1.0) < 1e-15
        tips = t.left < 0
        assert tips.sum() == n and np.all(t.age[tips] == 0.0)
        for v in range(1, t.n_nodes):
            assert t.age[t.parent[v]] > t.age[v]
        assert sorted(t.preorder.tolist()) == list(range(t.n_nodes)) and t.preorder[0] == 0
