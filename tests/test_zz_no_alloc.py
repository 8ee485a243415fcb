"""The allocation-free resampling entry point (GPU).

smc_resample_static serves callers that cannot allocate device memory
themselves (their device memory is owned by another framework's pool, or an
allocation's implicit device-wide synchronisation is not allowed on their path).
Its scratch is a fixed array inside the library.  It must give exactly what
smc_resample gives, call after call (the array keeps the previous call's
contents), and refuse populations larger than its fixed limit.
"""
import ctypes as C

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def _both(lw_np, u):
    import torch
    from paper_2112_00364_gb300 import smc

    x = torch.from_numpy(lw_np).cuda()
    a_ref, o_ref, n_ref = smc.resample(x, u)
    a_st, o_st, n_st = smc.resample_static(x, u)
    torch.cuda.synchronize()
    return (a_ref.cpu().numpy(), o_ref.cpu().numpy(), int(n_ref.cpu()[0]),
            a_st.cpu().numpy(), o_st.cpu().numpy(), int(n_st.cpu()[0]))


@pytest.mark.parametrize("N", [1, 4097, 300_001])
def test_static_matches_workspace_version_two_calls(N):
    # two calls in a row with different populations: the second must not see
    # anything the first left in the shared scratch
    for call, (seed, u) in enumerate([(N, 0.25), (N + 7, 0.8125)]):
        lw = inputs.random_logw(N, seed=seed, scale=2.5, dead_frac=0.2 if N > 1 else 0.0)
        if not np.isfinite(lw).any():
            lw[0] = 0.0
        a_ref, o_ref, n_ref, a_st, o_st, n_st = _both(lw, u)
        np.testing.assert_array_equal(a_st, a_ref)
        np.testing.assert_array_equal(o_st, o_ref)
        assert n_st == n_ref


def test_static_rejects_populations_above_its_limit():
    import torch
    from paper_2112_00364_gb300 import smc

    L = smc.lib()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    anc = torch.empty(8, dtype=torch.int32, device="cuda")
    o3 = torch.empty(3, dtype=torch.float64, device="cuda")
    nn = torch.empty(1, dtype=torch.int64, device="cuda")
    st = L.smc_resample_static(x.data_ptr(), smc.RESAMPLE_STATIC_MAX_N + 1, 0.5, anc.data_ptr(),
                               o3.data_ptr(), nn.data_ptr(), None)
    assert st == smc.EINVAL
    assert b"static scratch limit" in L.smc_last_error()


def test_static_calls_leave_device_free_memory_unchanged():
    """With caller-owned outputs, repeated calls allocate no device memory: the
    device's free memory (cudaMemGetInfo) is the same before and after twenty
    calls, once a first call has set up the device."""
    import torch
    from paper_2112_00364_gb300 import smc

    N = 1_000_003
    x = torch.from_numpy(inputs.random_logw(N, seed=11, scale=2.0)).cuda()
    anc = torch.empty(N, dtype=torch.int32, device="cuda")
    o3 = torch.empty(3, dtype=torch.float64, device="cuda")
    nn = torch.empty(1, dtype=torch.int64, device="cuda")
    smc.resample_static(x, 0.5, anc, o3, nn)  # first call on the device: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(20):
        smc.resample_static(x, (k + 0.5) / 21, anc, o3, nn)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
