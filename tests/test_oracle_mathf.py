"""Pins of the oracle's FP32 elementary functions (CPU).

In FP32-particle mode every logarithm, exponential and Box-Muller cosine of a
run is one of the oracle's own single-precision functions (log, exp,
cos(2 pi u), log1p, expm1, log k!), not the C library's, so that the GPU can
perform the same operations and reproduce every bit.  Each function is pinned
here against float64 reference values from numpy / scipy: within its ulp bound
everywhere it is sampled, exhaustively over the 2^23 odd points of the FP32
uniform grid ((n | 1) 2^-24) where the samplers evaluate log and cos(2 pi u),
and exact at its special points.
"""
import numpy as np
import pytest
from scipy.special import gammaln

import oracle


def _ulps(y, ref):
    """|y - ref| in units of the float32 spacing at ref."""
    ref = np.asarray(ref, dtype=np.float64)
    sp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    return np.abs(np.asarray(y, dtype=np.float64) - ref) / sp


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def grid():
    """Every FP32 uniform: (2j + 1) 2^-24, j = 0 .. 2^23 - 1."""
    return (np.arange(1 << 23, dtype=np.float64) * 2.0 + 1.0) * 2.0 ** -24


def test_log_on_the_uniform_grid_and_wide(grid):
    assert _ulps(oracle.mathf("log", grid), np.log(grid)).max() <= 1.0
    x = _f32(np.exp(np.random.default_rng(2).uniform(-87, 88, 1_000_000)))
    assert _ulps(oracle.mathf("log", x), np.log(x)).max() <= 1.5
    sub = _f32([1e-40, 3e-45, 1.1754942e-38])  # subnormals and the largest one
    assert _ulps(oracle.mathf("log", sub), np.log(sub)).max() <= 1.0
    y = oracle.mathf("log", [1.0, 0.0, -1.0, np.inf, 2.0])
    assert y[0] == 0.0 and y[1] == -np.inf and np.isnan(y[2]) and y[3] == np.inf
    assert _ulps(y[4], np.log(2.0)) <= 0.5


def test_exp_accuracy_and_range():
    x = _f32(np.random.default_rng(1).uniform(-87.3, 88.7, 2_000_000))
    assert _ulps(oracle.mathf("exp", x), np.exp(x)).max() <= 1.5
    x = _f32(np.random.default_rng(3).uniform(-1e-3, 1e-3, 100_000))
    assert _ulps(oracle.mathf("exp", x), np.exp(x)).max() <= 1.5
    y = oracle.mathf("exp", [0.0, -np.inf, np.inf, 89.5, -200.0, 88.72])
    assert y[0] == 1.0 and y[1] == 0.0 and y[2] == np.inf and y[3] == np.inf and y[4] == 0.0
    assert np.isfinite(y[5])
    # subnormal results: within one subnormal spacing (2^-149)
    xs = _f32(np.linspace(-103.5, -88.0, 2001))
    assert np.abs(oracle.mathf("exp", xs) - np.exp(xs)).max() <= 2.0 ** -149


def test_cos2pi_on_the_uniform_grid(grid):
    c = oracle.mathf("cos2pi", grid)
    ref = np.cos(2.0 * np.pi * grid)
    assert _ulps(c, ref).max() <= 1.5
    # the quadrant points are exact
    y = oracle.mathf("cos2pi", [0.0, 0.25, 0.5, 0.75, 1.0])
    np.testing.assert_array_equal(np.abs(y), [1.0, 0.0, 1.0, 0.0, 1.0])
    assert y[0] == 1.0 and y[2] == -1.0 and y[4] == 1.0
    # symmetry cos(2 pi (1 - u)) = cos(2 pi u) holds exactly on the grid
    np.testing.assert_array_equal(oracle.mathf("cos2pi", 1.0 - grid[:4096]), c[:4096])


def test_log1p_accuracy():
    rng = np.random.default_rng(4)
    x = _f32(np.concatenate([rng.uniform(-0.999, 2.0, 1_000_000),
                             np.exp(rng.uniform(-40, 30, 500_000)),
                             -np.exp(rng.uniform(-40, -0.001, 500_000))]))
    x = x[x > -1.0]
    assert _ulps(oracle.mathf("log1p", x), np.log1p(x)).max() <= 1.5
    y = oracle.mathf("log1p", [0.0, -1.0, -2.0, np.inf, 1e-30])
    assert y[0] == 0.0 and y[1] == -np.inf and np.isnan(y[2]) and y[3] == np.inf
    assert y[4] == _f32(1e-30)


def test_expm1_accuracy():
    rng = np.random.default_rng(5)
    x = _f32(np.concatenate([rng.uniform(-5, 5, 1_000_000), rng.uniform(-1e-3, 1e-3, 100_000),
                             rng.uniform(0, 88, 1_000_000), rng.uniform(-100, -5, 100_000)]))
    assert _ulps(oracle.mathf("expm1", x), np.expm1(x)).max() <= 1.5
    y = oracle.mathf("expm1", [0.0, np.inf, -np.inf, 1e-30, 100.0])
    assert y[0] == 0.0 and y[1] == np.inf and y[2] == -1.0 and y[3] == _f32(1e-30)
    assert y[4] == np.inf


def test_log_factorial():
    k = np.arange(0, 200_000, dtype=np.float64)
    lf = oracle.mathf("lfact", k)
    ref = gammaln(k + 1.0)
    # below 32: the float rounding of the FP64 sum of logs (within one ulp of exact)
    assert _ulps(lf[:32], ref[:32]).max() <= 1.0
    assert lf[0] == 0.0 and lf[1] == 0.0
    assert _ulps(lf[32:], ref[32:]).max() <= 3.0
