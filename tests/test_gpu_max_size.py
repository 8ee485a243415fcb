"""A run at the largest particle count the library accepts (GPU).

N = SMC_MAX_PARTICLES = 2^31 - 257 particles of the linear-Gaussian model
(T = 3), outputs kept on the device (about 190 GB in all): 8.4 million tiles of
256, so the run's last CTA of each segment combines the others' tile records
for the next wave, ancestor indices reach the int32 limit, and every particle
array is indexed past 2^31 bytes.  The oracle cannot run this size, so the
checks are properties that hold at any N: the status and counts, every
particle at b_stop, the last ancestor row non-decreasing inside [0, N), and
log Z and the weighted mean and variance of x_T against the Kalman filter
(their Monte Carlo error at this N is far below the tolerances).
"""
import math

import pytest

import closed_forms as cf
import inputs

pytestmark = pytest.mark.gpu

CHUNK = 1 << 28


def test_lg_at_max_particles():
    import torch

    from paper_2112_00364_gb300 import smc

    torch.cuda.empty_cache()  # blocks cached by earlier tests
    free, total = torch.cuda.mem_get_info()
    if total < 200 * 2 ** 30:
        pytest.skip("needs about 200 GiB of device memory")
    assert free >= 190 * 2 ** 30, f"only {free / 2 ** 30:.0f} GiB free of {total / 2 ** 30:.0f}"
    N = smc.MAX_PARTICLES
    y = inputs.lg_observations(3, seed=5)
    m = smc.Model("lg", obs=y)
    r = None
    try:
        r = smc.run(m, N, seed=2, where="device")
        torch.cuda.synchronize()
        assert r["status"] == smc.OK
        assert r["n_segments"] == 3 and r["n_resamples"] == 2
        assert r["n_overflow"] == 0 and r["n_limit"] == 0
        pc = r["int_fields"][0]
        anc = r["ancestors"][0]
        lw = r["final_logw"]
        x = r["real_fields"][0]
        assert pc.numel() == N and anc.numel() == N
        mx = float(lw.max())
        s0 = s1 = s2 = 0.0
        for lo in range(0, N, CHUNK):
            hi = min(N, lo + CHUNK)
            assert bool((pc[lo:hi] == -1).all())
            a = anc[lo:min(N, hi + 1)]
            assert bool((a[1:] >= a[:-1]).all())
            w = torch.exp(lw[lo:hi] - mx)
            xs = x[lo:hi]
            s0 += float(w.sum())
            s1 += float((w * xs).sum())
            s2 += float((w * xs * xs).sum())
        assert int(anc[0]) >= 0 and int(anc[N - 1]) < N
        ll, mean, var = cf.kalman_filter(y)
        log_z = float(r["log_z"].cpu()[0])
        assert abs(log_z - ll) < 1e-3, (log_z, ll)
        est_mean = s1 / s0
        est_var = s2 / s0 - est_mean * est_mean
        assert abs(est_mean - mean) < 1e-3 * math.sqrt(var), (est_mean, mean)
        assert abs(est_var - var) < 2e-3 * var, (est_var, var)
    finally:
        del r
        m.close()
        torch.cuda.empty_cache()
