"""Model constants away from their defaults, through the C ABI vs the oracle,
element by element (GPU).

The other parity tests run each model at its default constants (rho = 1, the
Gamma(1, 1) / Gamma(1, 0.5) priors, the linear-Gaussian model of the
benchmark, Fig. 2a's p = 1/2).  Here the same kernels run with the sampling
probability rho = 1/2 (the tips' log rho and the hidden lineages' detection
draw of Listing 1), other prior scales (also for the delayed-sampling
posteriors of Section 6.3), depth cap 1 (a hidden lineage may start on an
observed branch but not speciate), other linear-Gaussian coefficients, another
geometric program, and a step limit that ends the run early.
"""
import numpy as np
import pytest

import inputs
import oracle
from parity import assert_parity_fp64, run_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["crbd", "crbd_ds"])
@pytest.mark.parametrize("rho,ls,ms", [(0.5, 1.0, 0.5), (1.0, 2.0, 0.25), (0.5, 0.7, 1.5)])
def test_tree_models_rho_and_prior_scales(kind, rho, ls, ms):
    tree = inputs.yule_tree(16, seed=7)
    g, o = run_pair(kind, 3001, seed=5, tree=tree, rho=rho, lambda_scale=ls, mu_scale=ms)
    assert_parity_fp64(g, o)


def test_crbd_fixed_rates_rho_half():
    tree = inputs.yule_tree(24, seed=5)
    g, o = run_pair("crbd", 2049, seed=8, tree=tree, rates=(3.0, 1.5), rho=0.5)
    assert_parity_fp64(g, o)


def test_rateshift_rho_half():
    tree = inputs.yule_tree(32, seed=3)
    cap = tree.max_pending_right() + 1
    g, o = run_pair("rateshift", 1500, seed=6, tree=tree, sigma=0.3, lam_stack_cap=cap, rho=0.5)
    assert_parity_fp64(g, o)
    np.testing.assert_allclose(g["stack"], o["stack"], rtol=1e-12, atol=0)


def test_crbd_ds_rho_half_with_ess():
    tree = inputs.yule_tree(16, seed=5)
    g, o = run_pair("crbd_ds", 2500, seed=9, tree=tree, rho=0.5, lambda_scale=2.0, mu_scale=0.25,
                    ess_threshold=0.5)
    assert_parity_fp64(g, o)
    assert 0 < g["n_resamples"] < g["n_segments"] - 1


@pytest.mark.parametrize("kind", ["crbd", "crbd_ds"])
def test_depth_cap_one(kind):
    tree = inputs.yule_tree(8, seed=8)
    params = dict(rates=(2.0, 1.0)) if kind == "crbd" else dict(lambda_scale=2.0)
    g, o = run_pair(kind, 2000, seed=3, tree=tree, depth_cap=1, **params)
    assert o["n_overflow"] > 0
    assert_parity_fp64(g, o)


def test_lg_other_coefficients():
    y = inputs.lg_observations(30, seed=2)
    kw = dict(obs=y, a=0.5, b=0.3, q_sd=0.7, r_sd=1.3, x0_mean=2.0, x0_sd=0.4)
    g, o = run_pair("lg", 1500, seed=4, **kw)
    assert_parity_fp64(g, o)


def test_geometric_other_program():
    g, o = run_pair("geometric", 2000, seed=6, geo_p=0.8, geo_logw=-0.3)
    assert g["n_segments"] > 5
    assert_parity_fp64(g, o)


@pytest.mark.parametrize("kind,limit", [("geometric", 2), ("lg", 7), ("crbd", 5)])
def test_step_limit(kind, limit):
    from paper_2112_00364_gb300 import smc

    params = {"geometric": {}, "lg": dict(obs=inputs.lg_observations(20, seed=1)),
              "crbd": dict(tree=inputs.yule_tree(16, seed=2))}[kind]
    m = smc.Model(kind, **params)
    g = smc.run(m, 1000, 3, max_segments=limit, record_all_ancestors=True)
    m.close()
    o = oracle.smc_run(kind, 1000, 3, max_segments=limit, follow=g["ancestors"],
                       record_ancestors=True, **params)
    assert g["status"] == smc.ESTEPLIMIT and o["status"] == oracle.ESTEPLIMIT
    assert g["n_segments"] == o["n_segments"] == limit
    assert_parity_fp64(g, o)
