"""The vector-borne disease SEIR model on the GPU (Section 6.2, Listing 2).

Its samplers against the oracle's, draw by draw on the same Philox counters
(integers exact; the rare draw whose accept test lies within the last place of
the two sides' log / exp may differ), a full run against the oracle in follow
mode (element-wise, FP64), the closed-form likelihood of a two-day run, and the
run's invariants at the benchmark size.
"""
import numpy as np
import pytest
from scipy import stats

import closed_forms as cf
import inputs
import oracle
from parity import assert_parity_exact, assert_parity_fp64, run_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p", [(20, 0.3), (1000, 0.02), (7370, 0.12), (300, 0.9), (0, 0.5)])
def test_binomial_matches_oracle(n, p, prec):
    from paper_2112_00364_gb300 import smc

    g, gb = smc.sample("binomial", 200_000, n, p, seed=21, precision=prec)
    g, gb = g.cpu().numpy(), gb.cpu().numpy()
    o, ob = oracle.sample("binomial", 200_000, n, p, seed=21, return_blocks=True,
                          precision=oracle.FP64 if prec == "fp64" else oracle.FP32)
    diff = g != o
    if prec == "fp32":  # the same single-precision operations on both sides
        assert diff.sum() == 0
    assert diff.mean() < 1e-5, diff.sum()
    np.testing.assert_array_equal(gb[~diff], ob[~diff])


@pytest.mark.parametrize("dist,p1,p2", [("beta", 1.0, 1.0), ("beta", 1 + 2 / 4.4, 3 - 2 / 4.4),
                                        ("gamma", 1 + 2 / 6.5, 0.0), ("gamma", 10.0, 0.0)])
def test_beta_gamma_match_oracle(dist, p1, p2):
    from paper_2112_00364_gb300 import smc

    g, gb = smc.sample(dist, 100_000, p1, p2, seed=23)
    g, gb = g.cpu().numpy(), gb.cpu().numpy()
    o, ob = oracle.sample(dist, 100_000, p1, p2, seed=23, return_blocks=True)
    same = gb == ob
    assert same.mean() > 0.9999
    np.testing.assert_allclose(g[same], o[same], rtol=1e-12, atol=0)


@pytest.mark.parametrize("N,seed", [(1000, 1), (3001, 2)])
def test_seir_parity(N, seed):
    y = inputs.seir_observations(63, seed=7)
    g, o = run_pair("seir", N, seed, obs=y)
    assert_parity_fp64(g, o)


def test_seir_fp32_parity():
    y = inputs.seir_observations(63, seed=7)
    g, o = run_pair("seir", 2000, 3, precision="fp32", obs=y)
    assert_parity_exact(g, o)


def test_seir_two_day_closed_form_gpu():
    from paper_2112_00364_gb300 import smc

    y1 = 7
    a, b = 1 + 2 / 4.4, 3 - 2 / 4.4
    Z = 0.0
    for k in range(1, 60):
        pk = stats.poisson.pmf(k - 1, 5.0)
        for e in range(0, 60):
            pe = stats.poisson.pmf(e, 5.0)
            d = np.arange(e + 1)
            Z += pk * pe * float((stats.betabinom.pmf(d, e, a, b) * (y1 <= k + d) / (k + d + 1)).sum())
    m = smc.Model("seir", obs=np.array([-1.0, float(y1)]))
    lz = np.array([smc.run(m, 20_000, s)["log_z_value"] for s in range(1, 101)])
    ok, mean, se = cf.unbiased_check(lz, np.log(Z))
    assert ok, (mean, se)


def test_seir_full_size_invariants():
    from paper_2112_00364_gb300 import smc

    y = inputs.seir_observations(182, seed=7)
    m = smc.Model("seir", obs=y)
    r = smc.run(m, 1 << 16, 1)
    assert r["status"] == 0 and r["n_segments"] == 182 and np.isfinite(r["log_z_value"])
    f = r["int_fields"]
    assert np.all(f[0] == -1)
    np.testing.assert_array_equal(f[1] + f[2] + f[3] + f[4], 7370)
    assert f[1:].min() >= 0
    th = r["real_fields"]
    assert np.all((th > 0) & (th < 1))


def test_seir_benchmark_workload_parity():
    """The benchmark's SEIR workload in full (N = 2^16, 182 days of synthetic
    weekly reports, FP64) against the oracle in follow mode, element by element."""
    y = inputs.seir_observations(182, seed=7)
    g, o = run_pair("seir", 1 << 16, 1, obs=y)
    assert_parity_fp64(g, o)
    assert g["n_segments"] == 182
