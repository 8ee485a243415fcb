"""Pins for the oracle's FP64 normaliser and systematic resampling (CPU only).

Properties that any correct systematic resampler has, independent of how the
running sum is formed: equal weights give the identity map, offspring counts
are floor or ceil of N w_j and sum to N, ancestors are non-decreasing, and
averaged over the uniform offset the offspring count equals N w_j exactly.
The log-Z increment is checked against scipy's logsumexp.
"""
import math

import numpy as np
import pytest
from scipy.special import logsumexp

import inputs
import oracle


@pytest.mark.parametrize("N", [1, 2, 3, 4, 33, 1024])
@pytest.mark.parametrize("u", [1e-9, 0.25, 0.5, 0.999999])
def test_equal_weights_identity(N, u):
    anc, flag, incr, m, S, rc = oracle.resample(np.full(N, -2.5), u)
    assert rc == 0
    np.testing.assert_array_equal(anc, np.arange(N))
    assert incr == -2.5  # constant log-weight c gives increment exactly c
    assert m == -2.5 and S == N


@pytest.mark.parametrize("N", [1, 2, 3, 33, 1000])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_systematic_offspring_properties(N, seed):
    lw = inputs.random_logw(N, seed, scale=2.0, dead_frac=0.1 if N > 3 else 0.0)
    if not np.isfinite(lw).any():
        lw[0] = 0.0
    rng = np.random.default_rng(seed)
    w = np.exp(lw - logsumexp(lw))
    for u in rng.random(20):
        anc, flag, incr, m, S, rc = oracle.resample(lw, float(u))
        assert rc == 0
        assert np.all(np.diff(anc) >= 0) and anc.min() >= 0 and anc.max() < N
        o = np.bincount(anc, minlength=N)
        assert o.sum() == N
        assert np.all(o >= np.floor(N * w - 1e-9)) and np.all(o <= np.ceil(N * w + 1e-9))
        assert np.all(o[~np.isfinite(lw)] == 0)  # killed particles never chosen
        assert abs(incr - (logsumexp(lw) - math.log(N))) < 1e-12 * max(1.0, abs(incr))


def test_systematic_unbiased_over_offset():
    N = 7
    lw = np.log(np.array([0.05, 0.3, 0.01, 0.2, 0.14, 0.25, 0.05]))
    w = np.exp(lw - logsumexp(lw))
    us = (np.arange(20000) + 0.5) / 20000
    tot = np.zeros(N)
    for u in us:
        anc, *_ = oracle.resample(lw, float(u))
        tot += np.bincount(anc, minlength=N)
    np.testing.assert_allclose(tot / len(us), N * w, atol=5e-4)


def test_all_dead_is_degenerate():
    anc, flag, incr, m, S, rc = oracle.resample(np.full(5, -np.inf), 0.3)
    assert rc == oracle.EDEGENERATE and incr == -np.inf


def test_boundary_flag():
    # weights 1,1,1,1 -> q = 1,2,3,4; with u = 0.5 no offset is near a boundary
    _, flag, *_ = oracle.resample(np.zeros(4), 0.5)
    assert flag.sum() == 0
    # an offset within 1e-12 N of q_0 = 1: i = 0, u = 1 - 1e-15
    _, flag, *_ = oracle.resample(np.zeros(4), 1.0 - 1e-15)
    assert flag[0] == 1


def test_boundary_flag_band_scales_with_n_and_covers_both_sides():
    # equal weights: q_j = j + 1 exactly (S = N, N / S = 1), offsets y_i = i + u.
    # The band is 1e-12 N = 1e-9 at N = 1000.
    N = 1000
    # y_i sits 5e-10 below q_i (the boundary of its own ancestor a_i = i)
    anc, flag, *_ = oracle.resample(np.zeros(N), 1.0 - 5e-10)
    np.testing.assert_array_equal(anc, np.arange(N))
    assert flag.all()
    # y_i sits 5e-10 above q_{i-1} (the boundary below its ancestor)
    anc, flag, *_ = oracle.resample(np.zeros(N), 5e-10)
    np.testing.assert_array_equal(anc, np.arange(N))
    assert flag[1:].all() and flag[0] == 0  # no boundary below particle 0
    # 2e-9 away from every boundary: outside the band
    _, flag, *_ = oracle.resample(np.zeros(N), 2e-9)
    assert flag.sum() == 0


def test_single_particle():
    anc, flag, incr, m, S, rc = oracle.resample(np.array([-3.25]), 0.7)
    assert anc.tolist() == [0] and incr == -3.25
