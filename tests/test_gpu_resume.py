"""Checkpoint / resume on the GPU (smc_run_cfg.resume_*).

Between checkpoints a run is its particles' states and log-weights, the log Z
closed so far and its segment index, and every draw comes from a counter keyed
by (seed, run, particle, segment, draw).  A run stopped by max_segments after k
segments (a snapshot: SMC_ESTEPLIMIT and its outputs) and resumed from those
outputs must therefore end exactly as the uninterrupted run: log Z, final
states and log-weights bit for bit, and the same ancestors and resampling
decisions from checkpoint k - 1 on.  Checked for every model, FP64 and FP32,
resampling at every checkpoint and ESS-triggered, snapshots in host and in
device memory, a chain of two snapshots, and against the oracle resumed from
the same snapshot.
"""
import numpy as np
import pytest

import inputs
import oracle
from parity import assert_parity_exact

pytestmark = pytest.mark.gpu


def _params(kind):
    if kind == "lg":
        return dict(obs=inputs.lg_observations(30, seed=2))
    if kind == "seir":
        return dict(obs=inputs.seir_observations(28, seed=7))
    if kind == "geometric":
        return {}
    tree = inputs.yule_tree(12, seed=3)
    if kind == "rateshift":
        return dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
    return dict(tree=tree)


def _same(a, b, from_row):
    assert a["run_status"] == b["run_status"]
    assert a["log_z_value"] == b["log_z_value"]
    assert a["n_segments"] == b["n_segments"]
    for k in ("final_logw", "real_fields", "int_fields", "stack"):
        if k in b:
            np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(a["ancestors"][from_row:], b["ancestors"][from_row:])
    np.testing.assert_array_equal(a["resampled"][from_row:], b["resampled"][from_row:])


@pytest.mark.parametrize("kind", ["lg", "crbd", "rateshift", "geometric", "seir", "crbd_ds"])
@pytest.mark.parametrize("ess", [0.0, 0.5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gpu_resume_equals_uninterrupted_run(kind, ess, prec):
    from paper_2112_00364_gb300 import smc

    m = smc.Model(kind, **_params(kind))
    kw = dict(precision=prec, ess_threshold=ess, record_all_ancestors=True)
    N, seed = 700, 5
    full = smc.run(m, N, seed, **kw)
    assert full["run_status"] == 0 and full["n_segments"] >= 4
    for k in (1, 2, full["n_segments"] // 2, full["n_segments"] - 1):
        snap = smc.run(m, N, seed, max_segments=k, **kw)
        assert snap["status"] == smc.ESTEPLIMIT and snap["n_segments"] == k
        res = smc.run(m, N, seed, resume_from=snap, **kw)
        _same(res, full, k - 1)
    m.close()


def test_gpu_resume_from_device_snapshot_and_chain():
    """A snapshot held in device memory, and a resumed run that is itself
    stopped and resumed again (ESS-triggered, so a snapshot may carry weights
    not yet closed into log Z)."""
    import torch
    from paper_2112_00364_gb300 import smc

    m = smc.Model("lg", **_params("lg"))
    kw = dict(ess_threshold=0.3, record_all_ancestors=True)
    full = smc.run(m, 600, 9, **kw)
    s1 = smc.run(m, 600, 9, max_segments=6, where="device", **kw)
    torch.cuda.synchronize()
    s2 = smc.run(m, 600, 9, max_segments=17, resume_from=s1, **kw)
    assert s2["status"] == smc.ESTEPLIMIT and s2["n_segments"] == 17
    res = smc.run(m, 600, 9, resume_from=s2, **kw)
    _same(res, full, 16)
    opened = [smc.run(m, 600, 9, max_segments=k, **kw) for k in range(2, 12)]
    assert any(s["log_z_closed"] != s["log_z_value"] for s in opened)
    m.close()


@pytest.mark.parametrize("kind", ["crbd", "rateshift", "seir"])
def test_gpu_resume_equals_oracle_resume(kind):
    """FP32: the GPU's resumed run and the oracle resumed from the same GPU
    snapshot, in follow mode, element by element (bit for bit)."""
    from paper_2112_00364_gb300 import smc

    p = _params(kind)
    m = smc.Model(kind, **p)
    N, seed, k = 900, 3, 5
    snap = smc.run(m, N, seed, precision="fp32", max_segments=k, record_all_ancestors=True)
    res = smc.run(m, N, seed, precision="fp32", record_all_ancestors=True, resume_from=snap)
    o = oracle.smc_run(kind, N, seed, precision=oracle.FP32, resume_from=snap,
                       follow=res["ancestors"], record_ancestors=True, **p)
    assert_parity_exact(res, o)
    m.close()


def test_gpu_resume_argument_checks():
    from paper_2112_00364_gb300 import smc

    m = smc.Model("crbd", **_params("crbd"))
    snap = smc.run(m, 100, 1, max_segments=3)
    with pytest.raises(smc.SmcError) as e:  # a limit below the snapshot's segment
        smc.run(m, 100, 1, max_segments=2, resume_from=snap)
    assert e.value.status == smc.EINVAL
    bad = dict(snap, final_logw=None)
    with pytest.raises(Exception):
        smc.run(m, 100, 1, resume_from=bad)
    m.close()
