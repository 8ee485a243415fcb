"""Standalone resampling primitives vs the oracle (GPU): FP64 normaliser,
scan and systematic search, and the stack-bounded particle gather."""
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


@pytest.mark.parametrize("N", [1, 2, 3, 33, 4095, 4096, 4097, 100_003, 1 << 20])
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
