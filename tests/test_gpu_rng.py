"""GPU random numbers vs the oracle's independent implementation (GPU)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_philox_bit_exact_1e6_counters():
    import torch
    from paper_2112_00364_gb300 import smc

    n = 1_000_000
    rng = np.random.Generator(np.random.PCG64(3))
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    out = smc.philox(torch.from_numpy(ctr.view(np.int32)).cuda(),
                     torch.from_numpy(key.view(np.int32)).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.philox(ctr, key))


@pytest.mark.parametrize("dist,p1,p2", [("uniform", 0, 0), ("uniform_ab", -1.0, 3.0),
                                        ("bernoulli", 0.3, 0), ("exponential", 2.5, 0),
                                        ("gamma1", 0.5, 0), ("normal", 1.5, 2.0),
                                        ("lognormal", 0.3, 0), ("poisson", 0.7, 0),
                                        ("poisson", 9.99, 0), ("poisson", 10.0, 0),
                                        ("poisson", 50.0, 0)])
def test_variates_fp64(dist, p1, p2):
    from paper_2112_00364_gb300 import smc

    n = 200_000
    g, gb = smc.sample(dist, n, p1, p2, seed=21, precision="fp64")
    g, gb = g.cpu().numpy(), gb.cpu().numpy()
    o, ob = oracle.sample(dist, n, p1, p2, seed=21, precision=oracle.FP64, return_blocks=True)
    if dist in ("uniform", "uniform_ab", "bernoulli"):
        np.testing.assert_array_equal(g, o)  # integer grid, one fma: exact
    elif dist == "poisson":
        # integer result; a decision can only flip where CUDA's and glibc's
        # exp/log/lgamma differ in the last place at a comparison boundary
        assert np.mean(g != o) < 1e-4
    else:
        # a few ulp of the variate's scale (fma(sd, z, mean) can cancel near 0)
        scale = max(abs(p1), abs(p2), 1.0)
        np.testing.assert_allclose(g, o, rtol=4e-15, atol=2e-15 * scale)
    assert np.mean(gb != ob) < 1e-4


@pytest.mark.parametrize("dist,p1,p2", [("uniform", 0, 0), ("uniform_ab", -1.0, 3.0),
                                        ("bernoulli", 0.3, 0), ("exponential", 2.5, 0),
                                        ("gamma1", 0.5, 0), ("normal", 1.5, 2.0),
                                        ("lognormal", 0.3, 0), ("poisson", 3.0, 0),
                                        ("poisson", 9.99, 0), ("poisson", 10.0, 0),
                                        ("poisson", 50.0, 0), ("poisson", 3000.0, 0),
                                        ("binomial", 40, 0.1), ("binomial", 7370, 0.3),
                                        ("binomial", 200, 0.9), ("beta", 1.45, 2.55),
                                        ("gamma", 3.5, 0), ("neg_binomial", 2.0, 1.5),
                                        ("neg_binomial", 30.0, 2.0), ("lomax", 3.0, 1.5)])
def test_variates_fp32_bit_exact(dist, p1, p2):
    """In FP32 mode the GPU's samplers and the oracle's perform the same
    single-precision operations (the mode's own log / exp / cos(2 pi u) / log1p
    / expm1 / log k! included), so every variate and every count of Philox
    blocks consumed is identical, bit for bit."""
    from paper_2112_00364_gb300 import smc

    n = 200_000
    g, gb = smc.sample(dist, n, p1, p2, seed=22, precision="fp32")
    o, ob = oracle.sample(dist, n, p1, p2, seed=22, precision=oracle.FP32, return_blocks=True)
    np.testing.assert_array_equal(g.cpu().numpy(), o)
    np.testing.assert_array_equal(gb.cpu().numpy(), ob)


def _f32_grid():
    return (np.arange(1 << 23, dtype=np.float64) * 2.0 + 1.0) * 2.0 ** -24


@pytest.mark.parametrize("fn", ["log", "exp", "cos2pi", "log1p", "expm1", "lfact"])
def test_fp32_functions_bit_exact_and_near_cuda(fn):
    """The FP32 mode's own functions on the GPU equal the oracle's bit for bit
    (exhaustively over the FP32 uniform grid for log and cos(2 pi u), on wide
    random samples otherwise) and stay within 2 ulp of CUDA's logf / expf /
    cospif / log1pf / expm1f."""
    from paper_2112_00364_gb300 import smc

    rng = np.random.default_rng(31)
    if fn in ("log", "cos2pi"):
        x = np.concatenate([_f32_grid(), np.exp(rng.uniform(-100, 88, 1_000_000)), [1.0, 2.0]])
        if fn == "cos2pi":
            x = np.concatenate([_f32_grid(), rng.random(100_000), [0.0, 0.25, 0.5, 0.75, 1.0]])
    elif fn == "exp":
        x = np.concatenate([rng.uniform(-104, 89, 2_000_000), rng.uniform(-1e-3, 1e-3, 10_000),
                            [0.0, 88.7, -87.3, -103.9]])
    elif fn == "log1p":
        x = np.concatenate([rng.uniform(-0.999, 2.0, 1_000_000), np.exp(rng.uniform(-40, 30, 500_000))])
    elif fn == "expm1":
        x = np.concatenate([rng.uniform(-5, 5, 1_000_000), rng.uniform(0, 88, 500_000),
                            rng.uniform(-1e-3, 1e-3, 10_000)])
    else:
        x = np.arange(0, 300_000, dtype=np.float64)
    x = x.astype(np.float32).astype(np.float64)
    g = smc.math_eval("f32_" + fn, x)
    np.testing.assert_array_equal(g, oracle.mathf(fn, x))
    if fn != "lfact":
        c = smc.math_eval("cuda_" + {"cos2pi": "cos2pif"}.get(fn, fn + "f"), x)
        ok = np.isfinite(c) & (np.abs(c) > 1e-30)
        ia = g[ok].astype(np.float32).view(np.int32).astype(np.int64)
        ib = c[ok].astype(np.float32).view(np.int32).astype(np.int64)
        if fn == "cos2pi":  # near the zeros of cos compare in absolute terms
            assert np.abs(g - c).max() <= 2 * 2.0 ** -24
        else:
            assert np.abs(ia - ib).max() <= 2


def _ulp_diff(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


@pytest.mark.parametrize("fn", ["log", "exp"])
def test_table_math_within_two_ulp(fn):
    """The table-driven FP64 log / exp used by the samplers (Tang's method) stay
    within 2 ulp of CUDA's library functions and of numpy's (glibc) results."""
    from paper_2112_00364_gb300 import smc

    rng = np.random.default_rng(5)
    if fn == "log":
        x = np.concatenate([rng.random(400_000), np.exp(rng.uniform(-700, 700, 400_000)),
                            1.0 + rng.uniform(-1e-3, 1e-3, 100_000), [1.0, 2.0, 0.5, 1e-300]])
        ref = np.log(x)
    else:
        x = np.concatenate([rng.uniform(-700, 700, 400_000), rng.uniform(-40, 0, 400_000),
                            rng.uniform(-1e-3, 1e-3, 100_000), [0.0, -1.0, 1.0]])
        ref = np.exp(x)
    tab = smc.math_eval("table_" + fn, x)
    lib = smc.math_eval("lib_" + fn, x)
    assert _ulp_diff(tab, lib).max() <= 2
    ok = np.isfinite(ref) & (ref != 0)
    assert _ulp_diff(tab[ok], ref[ok]).max() <= 2


def test_uniform_log_from_bits_matches_table_log():
    """The samplers take log u of an FP64 uniform straight from its 64 random
    bits (reduction and the log1p polynomial on the integer pipes, the final
    combination in FP64): within 1 ulp of the correctly rounded log u (decimal
    arithmetic at 50 digits, on a subsample and near u = 1, where log u is
    tiny), within 2 ulp of numpy's log and of the table log of the uniform
    built as a double."""
    from decimal import Decimal, getcontext

    from paper_2112_00364_gb300 import smc

    getcontext().prec = 50
    rng = np.random.default_rng(11)
    near_one = np.array([((1 << 53) - k) << 11 for k in range(1, 2000)], dtype=np.uint64)
    bits = np.concatenate([rng.integers(0, 2**63, 500_000, dtype=np.uint64) * 2
                           + rng.integers(0, 2, 500_000, dtype=np.uint64), near_one,
                           np.array([0, 1, 2**11, 2**64 - 1, 0x6A09E667F3BCD << 12,
                                     (0x6A09E667F3BCD << 12) - 1, 1 << 63], dtype=np.uint64)])
    a = smc.math_eval("unif_log_bits", bits)
    b = smc.math_eval("unif_log_table", bits)
    assert _ulp_diff(a, b).max() <= 2
    n = (bits >> np.uint64(11)) | np.uint64(1)
    u = n.astype(np.float64) * 2.0**-53
    assert _ulp_diff(a, np.log(u)).max() <= 2
    pick = np.concatenate([np.arange(0, len(bits), 97), np.arange(500_000, len(bits))])
    ln2 = Decimal(2).ln()
    ref = np.array([float(Decimal(int(n[i])).ln() - 53 * ln2) for i in pick])
    assert _ulp_diff(a[pick], ref).max() <= 1


def test_fixed_point_weight_exponential():
    """The segment kernel forms each particle's weight as the integer
    round(e^d 2^54), d <= 0, on the integer pipes: within one unit of the exact
    rounding (decimal arithmetic at 60 digits) and within two of the table
    exponential rounded to the same grid; 0 below e^-38.5."""
    from decimal import Decimal, getcontext

    from paper_2112_00364_gb300 import smc

    getcontext().prec = 60
    rng = np.random.default_rng(21)
    d = np.concatenate([-rng.uniform(0, 38.6, 20_000), -rng.uniform(0, 1e-3, 2_000),
                        -rng.uniform(0, 0.7, 8_000),
                        [0.0, -1e-300, -38.1, -38.13, -38.2, -38.49, -38.6, -1000.0,
                         -0.6931471805599453]])
    got = smc.math_eval("exp_fix54", d)
    tab = smc.math_eval("table_exp_fix54", d)
    scale = Decimal(2) ** 54
    ref = np.array([int((Decimal(float(x)).exp() * scale).to_integral_value()) for x in d])
    assert np.abs(got - ref).max() <= 1
    assert np.abs(got - tab).max() <= 2
    assert got[d <= -38.5].max() == 0


@pytest.mark.parametrize("bits", [54, 50])
def test_two_table_fixed_point_exponential(bits):
    """The standalone resampler's weights come from a cheaper integer
    exponential (two 64-entry tables of 2^(-j/64) and 2^(-j/4096) and a degree-4
    polynomial): round(e^d 2^B) within one unit of the exact rounding (decimal
    arithmetic at 60 digits) for B = 54 and 50, 1.0 exactly at d = 0, 0 below
    e^-38.5, and non-increasing in d over a fine sorted grid."""
    from decimal import Decimal, getcontext

    from paper_2112_00364_gb300 import smc

    getcontext().prec = 60
    rng = np.random.default_rng(22 + bits)
    d = np.concatenate([-rng.uniform(0, 38.6, 20_000), -rng.uniform(0, 1e-3, 2_000),
                        -rng.uniform(0, 0.7, 8_000), -np.arange(64) * np.log(2.0) / 64,
                        -np.arange(64) * np.log(2.0) / 4096,
                        [0.0, -1e-300, -38.1, -38.13, -38.2, -38.49, -38.6, -1000.0,
                         -0.6931471805599453]])
    got = smc.math_eval(f"exp2t_fix{bits}", d)
    scale = Decimal(2) ** bits
    ref = np.array([int((Decimal(float(x)).exp() * scale).to_integral_value()) for x in d])
    assert np.abs(got - ref).max() <= 1
    assert got[np.flatnonzero(d == 0.0)[0]] == 1 << bits
    assert got[d <= -38.5].max() == 0
    grid = -np.sort(rng.uniform(0, 3.0, 50_000))[::-1]  # increasing toward 0
    g = smc.math_eval(f"exp2t_fix{bits}", grid)
    assert np.all(np.diff(g) >= 0)


def test_resampler_table_exponential():
    """smc_resample's weights: round(e^d 2^50) from the argument in 2^-52 units,
    one 9216-entry table of e^(-j/256) in units of 2^-56 and a degree-5
    polynomial in the remainder: within one unit of the exact rounding (decimal
    arithmetic at 60 digits) over the whole range and at every table point, 2^50
    exactly at d = 0, 0 from e^-36 on, and non-increasing in d over a fine
    sorted grid."""
    from decimal import Decimal, getcontext

    from paper_2112_00364_gb300 import smc

    getcontext().prec = 60
    rng = np.random.default_rng(31)
    d = np.concatenate([-rng.uniform(0, 36.5, 20_000), -rng.uniform(0, 1e-3, 2_000),
                        -rng.uniform(0, 0.7, 8_000), -np.arange(9300) / 256.0,
                        -np.arange(9300) / 256.0 - 2.0**-9, -np.arange(1, 9300) / 256.0 + 2.0**-40,
                        [0.0, -1e-300, -35.3, -35.36, -35.9, -36.0, -36.01, -1000.0,
                         -0.6931471805599453]])
    got = smc.math_eval("rs_fix50", d)
    scale = Decimal(2) ** 50
    ref = np.array([int((Decimal(float(x)).exp() * scale).to_integral_value()) for x in d])
    assert np.abs(got - ref).max() <= 1
    assert got[np.flatnonzero(d == 0.0)[0]] == 1 << 50
    assert got[d <= -36.0].max() == 0
    grid = -np.sort(rng.uniform(0, 3.0, 50_000))[::-1]
    g = smc.math_eval("rs_fix50", grid)
    assert np.all(np.diff(g) >= 0)


def test_integer_pipe_exponential_double():
    """The FP64 Poisson sampler forms e^-mean on the integer pipes (two-table
    exponential, then one rounding of a 61-bit significand to 53 bits and an
    exact exponent shift): within 1 ulp of the correctly rounded e^-m (decimal
    arithmetic at 60 digits) over [0, 64), exactly 1 at 0, and the table
    exponential outside the range."""
    from decimal import Decimal, getcontext

    from paper_2112_00364_gb300 import smc

    getcontext().prec = 60
    rng = np.random.default_rng(41)
    m = np.concatenate([rng.uniform(0, 10, 40_000), rng.uniform(0, 64, 10_000),
                        10.0 ** rng.uniform(-17, 0, 10_000), np.arange(64) * np.log(2.0) / 64,
                        [0.0, 5e-324, 1e-300, 9.999999999999998, 63.99999999, 64.0, 100.0]])
    got = smc.math_eval("exp_neg_int", m)
    ref = np.array([float((-Decimal(float(x))).exp()) for x in m])
    assert got[np.flatnonzero(m == 0.0)[0]] == 1.0
    assert _ulp_diff(got, ref).max() <= 1


def test_q_ratio_exact():
    """The search's offset scale S / N in 64.64 fixed point: floor(S 2^64 / N)
    exactly (Python's integers), over the whole argument range (S < 2^63,
    N < 2^31), at quotient digits that are exact integers, one below and one
    above (the correction steps), and at the extremes."""
    from paper_2112_00364_gb300 import smc

    rng = np.random.default_rng(17)
    pairs = []
    for _ in range(20000):
        N = int(rng.integers(1, 1 << 31))
        S = int(rng.integers(0, 1 << 63))
        pairs.append((S, N))
    for N in (1, 2, 3, 7, 1024, 65536, (1 << 20) + 1, (1 << 31) - 257, (1 << 31) - 1):
        for S in (0, 1, N - 1, N, N + 1, (1 << 61), (1 << 62) + 12345, (1 << 63) - 1):
            pairs.append((S, N))
        for m in (1, 2, 12345, (1 << 31) - 1):  # S a multiple of N, and one either side
            for dS in (-1, 0, 1):
                S = m * N + dS
                if 0 <= S < (1 << 63):
                    pairs.append((S, N))
    x = np.array(pairs, dtype=np.uint64)
    got = smc.math_eval("q_ratio", x)
    for (S, N), (hi, lo) in zip(pairs, got):
        q = (S << 64) // N
        assert (int(hi), int(lo)) == (q >> 64, q & ((1 << 64) - 1)), (S, N)
