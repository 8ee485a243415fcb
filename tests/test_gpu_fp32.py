"""FP32-particle / FP64-reduction mode against the oracle (GPU).

In FP32 mode the particle arithmetic and log-weights are single precision while
the normaliser, scan and log Z stay FP64.  The GPU and the oracle perform the
same single-precision operations, the mode's own log / exp / cos(2 pi u) /
log1p / expm1 / log k! included, so an FP32 run is compared with the FP32
oracle in follow mode exactly as an FP64 one: no unflagged ancestor difference,
every final log-weight and state bit-identical, log Z to the FP64 tolerance.
The statistical checks compare FP32 estimates with exact likelihoods, and the
per-result log-Z error of FP32 against the FP64 oracle on the same seeds (an
FP32 uniform is the FP64 uniform of the same counter to within 2^-24).
"""
import math

import numpy as np
import pytest

import closed_forms as cf
import inputs
import oracle
from parity import assert_parity_exact, run_pair

pytestmark = pytest.mark.gpu


def _check_fp32(g, o):
    assert_parity_exact(g, o)


@pytest.mark.parametrize("N,seed", [(1000, 1), (5000, 2)])
def test_lg_fp32_follows_oracle(N, seed):
    y = inputs.lg_observations(50, seed=1)
    g, o = run_pair("lg", N, seed, precision="fp32", obs=y)
    _check_fp32(g, o)


@pytest.mark.parametrize("kind", ["crbd", "rateshift"])
def test_tree_fp32_follows_oracle(kind):
    tree = inputs.yule_tree(32, seed=3)
    p = dict(tree=tree)
    if kind == "rateshift":
        p.update(sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    g, o = run_pair(kind, 4000, 5, precision="fp32", **p)
    _check_fp32(g, o)


def test_rateshift_fp32_unbiased_fixed_multipliers():
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(24, seed=6)
    cap = tree.max_pending_right() + 1
    rng = np.random.default_rng(1)
    mult = np.exp(0.3 * rng.standard_normal(tree.n_nodes))
    lam0, mu = 2.0, 0.6
    lam_b = np.empty(tree.n_nodes)
    lam_b[0] = lam0
    for v in tree.preorder[1:]:
        lam_b[v] = lam_b[tree.parent[v]] * mult[v]
    m = smc.Model("rateshift", tree=tree, rates=(lam0, mu), fixed_mult=mult, lam_stack_cap=cap)
    lz = [smc.run(m, 1 << 14, seed=s, precision="fp32")["log_z_value"] for s in range(1, 101)]
    ok, mean, se = cf.unbiased_check(np.array(lz), cf.crbd_log_z_rates(tree, lam_b, mu))
    assert ok, (mean, se)


def test_crbd_fp32_unbiased_fixed_rates_64_tips():
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(64, seed=2)
    m = smc.Model("crbd", tree=tree, rates=(4.0, 1.0))
    lz = [smc.run(m, 1 << 16, seed=s, precision="fp32")["log_z_value"] for s in range(1, 101)]
    ok, mean, se = cf.unbiased_check(np.array(lz), cf.crbd_log_z(tree, 4.0, 1.0))
    assert ok, (mean, se)


def test_rateshift_fp32_matches_fp64_oracle_in_distribution():
    """The log-Z error of FP32 particles against the FP64 oracle (the FP32
    mode's precision statement): over 24 seeds the two means of log Zhat agree within
    3 combined standard errors, and the mean difference is reported."""
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(48, seed=3)
    p = dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    m = smc.Model("rateshift", **p)
    g = np.array([smc.run(m, 4096, seed=s, precision="fp32")["log_z_value"] for s in range(1, 25)])
    o = np.array([oracle.smc_run("rateshift", 4096, seed=100 + s, **p)["log_z"]
                  for s in range(1, 25)])
    se = math.sqrt(g.var(ddof=1) / len(g) + o.var(ddof=1) / len(o))
    assert abs(g.mean() - o.mean()) <= 3 * se, (g.mean(), o.mean(), se)


def test_rateshift_full_config_properties():
    """C3 at full size (256-tip tree, N = 2^20, FP32 particles): every particle
    ends at b_stop with an empty pending-rate stack, log Z is finite, the
    recorded last ancestors are a valid systematic resampling (non-decreasing,
    in range), and no particle hit the stack or depth caps."""
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(256, seed=3)
    m = smc.Model("rateshift", tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    r = smc.run(m, 1 << 20, seed=1, precision="fp32")
    assert r["status"] == 0 and r["n_segments"] == 511
    assert np.isfinite(r["log_z_value"])
    assert np.all(r["int_fields"][0] == -1) and np.all(r["int_fields"][1] == 0)
    a = r["ancestors"][0]
    assert a.min() >= 0 and a.max() < (1 << 20) and np.all(np.diff(a) >= 0)
    assert r["n_overflow"] == 0 and r["n_limit"] == 0


def test_rateshift_benchmark_tree_fp32_follows_oracle():
    """The benchmark's rate-shift tree (256 tips, 511 checkpoints, sigma = 0.3)
    in FP32 at N = 2^14 against the FP32 oracle in follow mode, to FP32 rounding
    (the full N = 2^20 is checked by its invariants above)."""
    tree = inputs.yule_tree(256, seed=3)
    g, o = run_pair("rateshift", 1 << 14, 1, precision="fp32", tree=tree, sigma=0.3,
                    lam_stack_cap=tree.max_pending_right() + 1)
    assert g["n_segments"] == 511
    _check_fp32(g, o)


def test_fp32_last_cta_combine_parity():
    """N = 300,001 particles (1,172 tiles of 256: more than one combining CTA
    can hold, so every segment is combined by the run's last CTA) in FP32,
    element-wise against the FP32 oracle, for the plain and the rate-shift CRBD."""
    tree = inputs.yule_tree(16, seed=8)
    g, o = run_pair("crbd", 300_001, 3, precision="fp32", tree=tree)
    _check_fp32(g, o)
    g, o = run_pair("rateshift", 300_001, 4, precision="fp32", tree=tree, sigma=0.3,
                    lam_stack_cap=tree.max_pending_right() + 1)
    _check_fp32(g, o)


def test_rateshift_benchmark_config_fp32_element_wise():
    """The rate-shift benchmark workload itself (256-tip tree, 511 checkpoints,
    N = 2^20, sigma = 0.3, FP32), launched as the benchmark launches it, against
    the FP32 oracle in follow mode: every ancestor row, log Z and every final
    state bit for bit."""
    tree = inputs.yule_tree(256, seed=3)
    g, o = run_pair("rateshift", 1 << 20, 1, precision="fp32", tree=tree, sigma=0.3,
                    lam_stack_cap=tree.max_pending_right() + 1)
    assert g["n_segments"] == 511
    _check_fp32(g, o)


def test_fp32_log_z_error_against_fp64_oracle_per_result():
    """The FP32 mode's log-Z error, result by result: the GPU's FP32 runs
    against the FP64 oracle on the same seeds (the same Philox counters, FP32
    uniforms within 2^-24 of the FP64 ones), rate-shift on a 48-tip tree.  Once
    a resampling decision differs the two runs go separate ways, so a paired
    difference is of the order of the Monte Carlo spread; what precision must
    not add is a bias: the mean paired difference lies within 3 standard errors
    of zero, and the paired differences spread no wider than two independent
    estimates would (sd below sqrt(2) times the FP64 estimates' sd)."""
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(48, seed=3)
    p = dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    m = smc.Model("rateshift", **p)
    seeds = range(1, 33)
    g = np.array([smc.run(m, 4096, seed=s, precision="fp32")["log_z_value"] for s in seeds])
    o = np.array([oracle.smc_run("rateshift", 4096, seed=s, **p)["log_z"] for s in seeds])
    m.close()
    d = g - o
    se = d.std(ddof=1) / math.sqrt(len(d))
    assert abs(d.mean()) <= 3 * se, (d.mean(), se)
    assert d.std(ddof=1) <= math.sqrt(2.0) * o.std(ddof=1), (d.std(ddof=1), o.std(ddof=1))
