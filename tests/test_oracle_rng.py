"""Pins for the oracle's random numbers (CPU only).

* Philox4x32-10 against an independent implementation: Triton's
  ``tl.philox`` run by Triton's CPU interpreter (the published Random123
  known-answer vectors are not available to copy).
* Each variate recipe against its closed-form distribution (KS tests,
  exact pmf chi-square for the Poisson sampler in both of its regimes).
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle


def _triton_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def kern(c0p, c1p, c2p, c3p, outp, k0, k1, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        c0 = tl.load(c0p + i).to(tl.uint32, bitcast=True)
        c1 = tl.load(c1p + i).to(tl.uint32, bitcast=True)
        c2 = tl.load(c2p + i).to(tl.uint32, bitcast=True)
        c3 = tl.load(c3p + i).to(tl.uint32, bitcast=True)
        seed = (k1.to(tl.uint64) << 32) | k0.to(tl.uint64)
        r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
        tl.store(outp + i * 4 + 0, r0.to(tl.int32, bitcast=True))
        tl.store(outp + i * 4 + 1, r1.to(tl.int32, bitcast=True))
        tl.store(outp + i * 4 + 2, r2.to(tl.int32, bitcast=True))
        tl.store(outp + i * 4 + 3, r3.to(tl.int32, bitcast=True))

    n = ctr.shape[0]
    out = np.empty((n, 4), dtype=np.uint32)
    for kk in np.unique(key, axis=0):
        sel = np.where((key == kk).all(axis=1))[0]
        cols = [torch.from_numpy(np.ascontiguousarray(ctr[sel, j]).view(np.int32)) for j in range(4)]
        o = torch.zeros(len(sel) * 4, dtype=torch.int32)
        kern[(1,)](*cols, o, int(kk[0]), int(kk[1]), BLOCK=len(sel))
        out[sel] = o.numpy().view(np.uint32).reshape(-1, 4)
    return out


def test_philox_matches_independent_implementation():
    rng = np.random.Generator(np.random.PCG64(7))
    n = 256
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    keys = rng.integers(0, 2 ** 32, size=(4, 2), dtype=np.uint64).astype(np.uint32)
    keys[0] = 0
    key = keys[np.arange(n) % 4]
    ours = oracle.philox(ctr, key)
    theirs = _triton_philox(ctr, key)
    np.testing.assert_array_equal(ours, theirs)


def test_philox_counter_sensitivity():
    base = np.zeros((1, 4), dtype=np.uint32)
    key = np.array([[1, 2]], dtype=np.uint32)
    ref = oracle.philox(base, key)
    for j in range(4):
        c = base.copy()
        c[0, j] = 1
        assert not np.array_equal(oracle.philox(c, key), ref)


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_uniform_open_interval_and_ks(prec):
    u = oracle.sample("uniform", 200_000, seed=11, precision=prec)
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, stats.uniform().cdf).pvalue > 1e-3


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_normal(prec):
    z = oracle.sample("normal", 200_000, 1.5, 2.0, seed=12, precision=prec)
    assert stats.kstest(z, stats.norm(1.5, 2.0).cdf).pvalue > 1e-3


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_exponential_and_gamma1(prec):
    e = oracle.sample("exponential", 200_000, 2.5, seed=13, precision=prec)
    assert stats.kstest(e, stats.expon(0, 1 / 2.5).cdf).pvalue > 1e-3
    g = oracle.sample("gamma1", 200_000, 0.5, seed=14, precision=prec)
    assert stats.kstest(g, stats.gamma(1.0, 0, 0.5).cdf).pvalue > 1e-3


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_uniform_ab_bernoulli_lognormal(prec):
    x = oracle.sample("uniform_ab", 200_000, -1.0, 3.0, seed=15, precision=prec)
    assert x.min() >= -1.0 and x.max() <= 3.0
    assert stats.kstest(x, stats.uniform(-1.0, 4.0).cdf).pvalue > 1e-3
    b = oracle.sample("bernoulli", 400_000, 0.3, seed=16, precision=prec)
    assert set(np.unique(b)) <= {0.0, 1.0}
    assert abs(b.mean() - 0.3) < 4 * math.sqrt(0.3 * 0.7 / b.size)
    ln = oracle.sample("lognormal", 200_000, 0.3, seed=17, precision=prec)
    assert stats.kstest(ln, stats.lognorm(0.3).cdf).pvalue > 1e-3


def _poisson_chi2(x, m):
    kmax = int(max(x.max(), m + 10 * math.sqrt(m) + 10))
    obs = np.bincount(x.astype(np.int64), minlength=kmax + 1).astype(float)
    pmf = stats.poisson.pmf(np.arange(kmax + 1), m)
    pmf[-1] += stats.poisson.sf(kmax, m)
    exp = pmf * x.size
    # pool cells with small expectation
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] < 5:
        o[-2] += o[-1]
        e[-2] += e[-1]
        o, e = o[:-1], e[:-1]
    chi2 = ((o - e) ** 2 / e).sum()
    return stats.chi2.sf(chi2, len(o) - 1)


@pytest.mark.parametrize("m", [0.1, 3.0, 9.99, 10.0, 50.0])
@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32])
def test_poisson_exact_pmf(m, prec):
    x, blocks = oracle.sample("poisson", 300_000, m, seed=18, precision=prec, return_blocks=True)
    assert np.all(x == np.floor(x)) and x.min() >= 0
    assert _poisson_chi2(x, m) > 1e-4
    if m < 10:
        assert np.all(blocks == 1)  # inversion: one uniform
    else:
        assert blocks.mean() < 1.45  # PTRS accepts most first trials


def test_streams_independent_of_run_id_and_seed():
    a = oracle.sample("uniform", 1000, seed=1, run_id=0)
    b = oracle.sample("uniform", 1000, seed=1, run_id=1)
    c = oracle.sample("uniform", 1000, seed=2, run_id=0)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15
