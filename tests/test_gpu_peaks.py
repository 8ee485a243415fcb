"""The compute-peak probe behind the bench line's measured FP64 denominator
(GPU): every rate positive and within what the SM's units can issue, FP64
far below FP32 on GB300's CUDA cores, and the rate independent of the number of
steps timed (the probe's operation count is right)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_peak_probe_rates_are_physical():
    import torch
    from paper_2112_00364_gb300 import smc

    iters = {0: 500, 1: 20000, 2: 5000, 3: 10000, 4: 1000}
    r = {smc.PEAK_KINDS[k][0]: smc.peak_probe(k, n) for k, n in iters.items()}
    assert all(np.isfinite(v) and v > 0 for v in r.values()), r
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.2e9  # above GB300's 2070 MHz maximum SM clock
    assert r["fp32_fma"] <= sms * clk * 128, r   # 128 FP32 lanes per SM
    assert r["fp64_fma"] <= sms * clk * 64, r    # no more than one FP64 lane per two FP32
    assert r["fp32_fma"] > 8 * r["fp64_fma"], r
    assert r["int32_imad"] <= sms * clk * 128, r
    assert r["fp32_ex2_sfu"] <= sms * clk * 128, r


def test_peak_probe_rate_does_not_depend_on_steps():
    from paper_2112_00364_gb300 import smc

    a = smc.peak_probe(0, 400)
    b = smc.peak_probe(0, 1600)
    assert 0.8 < a / b < 1.25, (a, b)
