"""Standalone resampling primitives vs the oracle (GPU): FP64 normaliser,
scan and systematic search, and the stack-bounded particle gather."""
import math

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _gpu_resample(lw, u):
    import torch
    from paper_2112_00364_gb300 import smc

    x = torch.from_numpy(lw).cuda()
    anc, o3, nn = smc.resample(x, u)
    torch.cuda.synchronize()
    return anc.cpu().numpy(), o3.cpu().numpy(), int(nn.cpu()[0])


@pytest.mark.parametrize("N", [1, 2, 3, 33, 4095, 4096, 4097, 100_003, 1 << 20, (1 << 24) + 4097])
@pytest.mark.parametrize("dead", [0.0, 0.3])
def test_resample_matches_oracle(N, dead):
    lw = inputs.random_logw(N, seed=N, scale=2.0, dead_frac=dead if N > 3 else 0.0)
    if not np.isfinite(lw).any():
        lw[0] = 0.0
    u = 0.3141592653589793
    a_g, o3, n_near = _gpu_resample(lw, u)
    a_o, flag, incr, m, S, rc = oracle.resample(lw, u)
    assert rc == 0
    diff = a_g != a_o
    assert np.all(flag[diff] == 1), np.where(diff & (flag == 0))[0][:10]
    # the GPU normalises by a power-of-two reference 2^k >= max weight: same total
    k = o3[0] / np.log(2.0)
    assert abs(k - round(k)) < 1e-9 and o3[0] >= m - 1e-12
    assert abs((o3[0] + np.log(o3[1])) - (m + np.log(S))) <= 1e-12 * max(1.0, abs(m))
    assert abs(o3[2] - incr) <= 1e-12 * max(1.0, abs(incr))
    assert np.all(np.diff(a_g) >= 0) and a_g.min() >= 0 and a_g.max() < N


def _adversarial_logw(kind, N, seed):
    rng = np.random.default_rng(seed)
    if kind == "dominant":  # one particle holds nearly all the weight: one tile spans ~N offsets
        lw = rng.normal(0.0, 1.0, N)
        lw[N // 3] = 40.0
    elif kind == "two_level":  # half the weights ~e^-30 of the rest: flat running sums up to the cap
        lw = np.where(rng.random(N) < 0.5, 0.0, -30.0) + rng.normal(0.0, 1e-3, N)
    elif kind == "wide":  # log-weights spread over +-100: a few particles per tile matter
        lw = rng.normal(0.0, 30.0, N)
    elif kind == "steps":  # every tile a different reference, far apart
        lw = -0.75 * (np.arange(N) // 4096) + rng.normal(0.0, 0.5, N)
    else:  # "ties": many exactly equal log-weights, boundaries on exact multiples
        lw = rng.integers(-3, 1, N).astype(np.float64)
    return lw


def _exact_tied_ancestors(lw, u, offsets):
    """a_i = min{ j : P_j N / S > i + u } in exact arithmetic for log-weights
    taking a few integer values: each class weight e^k to 2^-120 (decimal
    arithmetic at 60 digits), running sums from the classes' running counts,
    compared with (i + u) S as exact rationals."""
    from decimal import Decimal, getcontext
    from fractions import Fraction

    getcontext().prec = 60
    ks = sorted({int(v) for v in np.unique(lw)})
    W = {k: int(Decimal(k).exp() * (Decimal(2) ** 120)) for k in ks}
    cnt = {k: np.cumsum(lw == k) for k in ks}
    N = lw.size

    def P(j):
        return sum(int(cnt[k][j]) * W[k] for k in ks)

    S, uf = P(N - 1), Fraction(u)
    out = []
    for i in offsets:
        target = (int(i) + uf) * S
        lo, hi = 0, N - 1
        while lo < hi:
            mid = (lo + hi) // 2
            if P(mid) * N > target:
                hi = mid
            else:
                lo = mid + 1
        out.append(lo)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("kind", ["dominant", "two_level", "wide", "steps", "ties"])
@pytest.mark.parametrize("u", [1e-9, 0.5, 1.0 - 1e-9])
def test_resample_adversarial_weights(kind, u):
    """The 32-bit offset counts of smc_resample's third pass and their exact
    fallback on weight shapes that push elements to it (tiles spanning most of
    the offsets, flat running sums near a tile's end, widely spread and tied
    weights, offsets at the ends of (0, 1)): every ancestor against the oracle
    (differences only at flagged offsets), the allocation-free form equal to
    the workspace form."""
    import torch
    from paper_2112_00364_gb300 import smc

    N = (1 << 20) + 12345
    lw = _adversarial_logw(kind, N, seed=sum(map(ord, kind)))
    x = torch.from_numpy(lw).cuda()
    anc, o3, nn = smc.resample(x, u)
    a_g = anc.cpu().numpy()
    a_o, flag, incr, m, S, rc = oracle.resample(lw, u)
    assert rc == 0
    diff = a_g != a_o
    unflagged = np.flatnonzero(diff & (flag == 0))
    if kind == "ties":
        # a million tied terms make the oracle's left-to-right FP64 running sum
        # drift past the 1e-12 N band: where it differs unflagged, the GPU must
        # give the exact ancestor
        exact = _exact_tied_ancestors(lw, u, unflagged)
        np.testing.assert_array_equal(a_g[unflagged], exact)
    else:
        assert unflagged.size == 0, unflagged[:10]
    assert np.all(np.diff(a_g) >= 0) and a_g[0] >= 0 and a_g[-1] < N
    # the increment against log-sum-exp with a correctly rounded sum (math.fsum):
    # on a million tied terms the oracle's left-to-right FP64 sum drifts by ~1e-11
    mx = lw.max()
    ref = mx + math.log(math.fsum(np.exp(lw - mx))) - math.log(N)
    assert abs(o3[2].item() - ref) <= 1e-12 * max(1.0, abs(ref))
    assert abs(incr - ref) <= 1e-9 * max(1.0, abs(ref))
    a_s, o3_s, nn_s = smc.resample_static(x, u)
    assert torch.equal(a_s, anc) and torch.equal(o3_s, o3) and torch.equal(nn_s, nn)


@pytest.mark.parametrize("N", [1, 5, 4096, 4097, 1 << 16])
def test_resample_equal_weights_identity(N):
    a_g, o3, _ = _gpu_resample(np.full(N, 0.75), 0.999)
    np.testing.assert_array_equal(a_g, np.arange(N))
    assert abs(o3[2] - 0.75) <= 2e-14  # a few ulp of k ln 2, log S and log N


def test_resample_degenerate():
    a_g, o3, _ = _gpu_resample(np.full(1000, -np.inf), 0.5)
    np.testing.assert_array_equal(a_g, np.arange(1000))
    assert o3[0] == -np.inf and o3[2] == -np.inf


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N", [7, 4096, 10_001])
def test_gather_with_stack_bound(dtype, N):
    import torch
    from paper_2112_00364_gb300 import smc

    rng = np.random.default_rng(N)
    F = 5
    src = rng.standard_normal((F, N)).astype(dtype)
    dst0 = rng.standard_normal((F, N)).astype(dtype)
    anc = np.sort(rng.integers(0, N, N)).astype(np.int32)
    sp = rng.integers(0, F + 1, N).astype(np.int32)
    d = torch.from_numpy(dst0.copy()).cuda()
    smc.gather(torch.from_numpy(src).cuda(), d, torch.from_numpy(anc).cuda(),
               torch.from_numpy(sp).cuda())
    got = d.cpu().numpy()
    exp = dst0.copy()
    for f in range(F):
        m = f < sp[anc]
        exp[f, m] = src[f, anc[m]]
    np.testing.assert_array_equal(got, exp)
    # without a stack pointer every row is copied
    d2 = torch.from_numpy(dst0.copy()).cuda()
    smc.gather(torch.from_numpy(src).cuda(), d2, torch.from_numpy(anc).cuda())
    np.testing.assert_array_equal(d2.cpu().numpy(), src[:, anc])


def test_resample_and_gather_bench_size():
    """The benchmark's standalone step at its full size (2^24 log-weights
    normal(0, 2), seed 24; a 2-field f64 state): every ancestor against the
    oracle (differences only where the oracle flags the offset), the
    normaliser and log-Z increment, and the gather element by element; with the
    workspace and static entry points giving the same ancestors."""
    import torch
    from paper_2112_00364_gb300 import smc

    N = 1 << 24
    lw = inputs.random_logw(N, seed=24, scale=2.0)
    for u in (0.5, 0.0123456789):
        x = torch.from_numpy(lw).cuda()
        anc, o3, nn = smc.resample(x, u)
        a_g = anc.cpu().numpy()
        a_o, flag, incr, m, S, rc = oracle.resample(lw, u)
        assert rc == 0
        diff = a_g != a_o
        assert np.all(flag[diff] == 1), np.where(diff & (flag == 0))[0][:10]
        assert np.all(np.diff(a_g) >= 0) and a_g[0] >= 0 and a_g[-1] < N
        assert abs(o3[2].item() - incr) <= 1e-12 * max(1.0, abs(incr))
        anc_s, _, _ = smc.resample_static(x, u)
        assert torch.equal(anc_s, anc)
    rng = np.random.default_rng(5)
    src_h = rng.standard_normal((2, N))
    src = torch.from_numpy(src_h).cuda()
    dst = torch.empty_like(src)
    smc.gather(src, dst, anc)
    np.testing.assert_array_equal(dst.cpu().numpy(), src_h[:, a_g])
