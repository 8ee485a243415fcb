"""Pins for the oracle's SMC runs (CPU only).

SMC's likelihood estimate Zhat is unbiased for Z (log Zhat is not), so for
each model with an exact Z the mean of Zhat / Z over independent seeds must
lie within 3 standard errors of 1:
  * linear-Gaussian (Fig. 3's model family): Z from the Kalman filter;
  * CRBD (Listing 1) at fixed rates: closed-form birth-death likelihood;
  * CRBD with mu = 0: Z = P(no hidden events), no p1 involved;
  * CRBD on a two-tip tree;
  * CRBD with its Gamma priors: Z from 2-D quadrature;
  * the weighted geometric program of Fig. 2a: Z = 2 (Section 2.2);
  * rate-shift with fixed per-branch multipliers: per-branch closed form.
Plus structural invariants: the b_stop rule, sigma = 0 reducing the
rate-shift model to CRBD exactly, and the depth-cap / call-limit kill rules.
"""
import math

import numpy as np
import pytest

import closed_forms as cf
import inputs
import oracle


def _many(model, N, seeds, **kw):
    out = []
    for s in seeds:
        r = oracle.smc_run(model, N, seed=s, **kw)
        assert r["status"] == 0, r["status"]
        out.append(r["log_z"])
    return np.array(out)


def test_lg_unbiased_vs_kalman():
    y = inputs.lg_observations(50, seed=1)
    lz = _many("lg", 1024, range(1, 101), obs=y)
    ok, mean, se = cf.unbiased_check(lz, cf.kalman_loglik(y))
    assert ok, (mean, se)
    # consistency: log Zhat concentrates on log Z
    assert abs(np.mean(lz) - cf.kalman_loglik(y)) < 0.1


@pytest.mark.parametrize("second_is_sd", [True, False])
def test_eq2_ssm_unbiased_vs_kalman(second_is_sd):
    # Eq. 2: X0 ~ N(0, 100), X_t ~ N(X_{t-1} + 2, 1), Y_t ~ N(X_t, 5); both
    # readings of the second argument (sd or variance) are checked.
    f = (lambda v: v) if second_is_sd else math.sqrt
    par = dict(a=1.0, b=2.0, q_sd=f(1.0), r_sd=f(5.0), x0_mean=0.0, x0_sd=f(100.0))
    y = inputs.lg_observations(20, seed=3, **par)
    lz = _many("lg", 512, range(1, 81), obs=y, **par)
    ok, mean, se = cf.unbiased_check(lz, cf.kalman_loglik(y, **par))
    assert ok, (mean, se)


def test_lg_single_particle_is_importance_sampling():
    y = inputs.lg_observations(5, seed=2)
    lz = _many("lg", 1, range(1, 4001), obs=y)
    ok, mean, se = cf.unbiased_check(lz, cf.kalman_loglik(y))
    assert ok, (mean, se)


@pytest.mark.parametrize("rho", [1.0, 0.5])
def test_crbd_fixed_rates_unbiased(rho):
    tree = inputs.yule_tree(16, seed=2)
    lam, mu = 2.5, 0.8
    lz = _many("crbd", 2048, range(1, 101), tree=tree, rates=(lam, mu), rho=rho)
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_log_z(tree, lam, mu, rho))
    assert ok, (mean, se)


def test_crbd_mu_zero_unbiased():
    tree = inputs.yule_tree(16, seed=3)
    lam = 2.0
    lz = _many("crbd", 1024, range(1, 101), tree=tree, rates=(lam, 0.0))
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_log_z_mu0(tree, lam))
    assert ok, (mean, se)


def test_crbd_two_tip_unbiased():
    tree = inputs.two_tip_tree(1.0)
    lam, mu = 1.5, 1.0
    lz = _many("crbd", 512, range(1, 201), tree=tree, rates=(lam, mu))
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_log_z(tree, lam, mu))
    assert ok, (mean, se)


def test_crbd_priors_unbiased_vs_quadrature():
    tree = inputs.yule_tree(8, seed=4)
    lz = _many("crbd", 4096, range(1, 101), tree=tree)
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_marginal_log_z(tree))
    assert ok, (mean, se)


def test_geometric_z_equals_two_and_posterior():
    lz = _many("geometric", 1024, range(1, 201))
    ok, mean, se = cf.unbiased_check(lz, math.log(2.0))
    assert ok, (mean, se)
    # weighted posterior over the flip count: P(n) = 0.25 * 0.75^(n-1)
    r = oracle.smc_run("geometric", 1 << 16, seed=7)
    w = np.exp(r["final_logw"] - r["final_logw"].max())
    cnt = r["int_fields"][1]
    assert np.all(r["int_fields"][0] == -1)  # everyone ended at b_stop
    for n in range(1, 5):
        p = w[cnt == n].sum() / w.sum()
        assert abs(p - 0.25 * 0.75 ** (n - 1)) < 0.02


def test_bstop_particles_keep_participating():
    # with few particles some finish segments before others; the run must
    # still end with everyone at b_stop and resample the finished ones
    r = oracle.smc_run("geometric", 64, seed=3, record_ancestors=True)
    assert r["status"] == 0 and r["n_segments"] > 1
    assert r["n_resamples"] == r["n_segments"] - 1


def test_rateshift_sigma_zero_is_crbd():
    tree = inputs.yule_tree(16, seed=5)
    cap = tree.max_pending_right() + 1
    for prec in (oracle.FP64, oracle.FP32):
        a = oracle.smc_run("crbd", 2048, seed=9, tree=tree, precision=prec, record_ancestors=True)
        b = oracle.smc_run("rateshift", 2048, seed=9, tree=tree, sigma=0.0, lam_stack_cap=cap,
                           precision=prec, record_ancestors=True)
        assert a["log_z"] == b["log_z"]
        np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
        np.testing.assert_array_equal(a["real_fields"], b["real_fields"])


def test_rateshift_fixed_multipliers_unbiased():
    tree = inputs.yule_tree(12, seed=6)
    cap = tree.max_pending_right() + 1
    rng = np.random.default_rng(1)
    mult = np.exp(0.3 * rng.standard_normal(tree.n_nodes))
    lam0, mu = 2.0, 0.6
    lam_b = np.empty(tree.n_nodes)
    lam_b[0] = lam0
    for v in tree.preorder[1:]:
        lam_b[v] = lam_b[tree.parent[v]] * mult[v]
    lz = _many("rateshift", 2048, range(1, 101), tree=tree, rates=(lam0, mu), fixed_mult=mult,
               lam_stack_cap=cap)
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_log_z_rates(tree, lam_b, mu))
    assert ok, (mean, se)


def test_rateshift_stack_depth_and_final_state():
    tree = inputs.yule_tree(32, seed=7)
    cap = tree.max_pending_right() + 1
    r = oracle.smc_run("rateshift", 256, seed=2, tree=tree, lam_stack_cap=cap)
    assert r["status"] == 0 and r["n_overflow"] == 0
    # at the end of the preorder walk no right child is pending
    assert np.all(r["int_fields"][1] == 0)


def test_depth_cap_and_call_limit_kill():
    tree = inputs.yule_tree(8, seed=8)
    r = oracle.smc_run("crbd", 512, seed=3, tree=tree, rates=(6.0, 5.0), depth_cap=1)
    assert r["n_overflow"] > 0
    r2 = oracle.smc_run("crbd", 512, seed=3, tree=tree, rates=(6.0, 5.0), call_limit=1)
    assert r2["n_limit"] > 0
    r3 = oracle.smc_run("crbd", 512, seed=3, tree=tree, rates=(6.0, 5.0))
    assert r3["n_overflow"] == 0 and r3["n_limit"] == 0
    # a tighter cap can only remove weight
    assert r["log_z"] <= r3["log_z"] + 1.0


def test_ancestor_follow_mode_adopts():
    y = inputs.lg_observations(10, seed=4)
    a = oracle.smc_run("lg", 256, seed=5, obs=y, record_ancestors=True)
    b = oracle.smc_run("lg", 256, seed=5, obs=y, follow=a["ancestors"], record_ancestors=True)
    assert b["n_hard_mismatch"] == 0 and b["log_z"] == a["log_z"]
    fake = a["ancestors"].copy()
    fake[-1, 10] = (fake[-1, 10] + 7) % 256  # last resampling: nothing downstream changes
    c = oracle.smc_run("lg", 256, seed=5, obs=y, follow=fake, record_ancestors=True)
    assert c["n_hard_mismatch"] == 1
    np.testing.assert_array_equal(c["ancestors"], fake)


def test_depth_cap_one_closed_form():
    # with depth_cap = 1 a hidden lineage may start on an observed branch but
    # not speciate itself: Z has the closed form of closed_forms.crbd_log_z_depth1
    tree = inputs.yule_tree(8, seed=8)
    lam, mu = 2.0, 1.0
    lz = _many("crbd", 2048, range(1, 101), tree=tree, rates=(lam, mu), depth_cap=1)
    ok, mean, se = cf.unbiased_check(lz, cf.crbd_log_z_depth1(tree, lam, mu))
    assert ok, (mean, se)


def test_step_limit():
    r = oracle.smc_run("geometric", 256, seed=1, max_segments=2)
    assert r["status"] == oracle.ESTEPLIMIT
    assert r["n_segments"] == 2  # the limit counts segments run
