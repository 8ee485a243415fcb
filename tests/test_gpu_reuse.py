"""Model handles built and destroyed per request (GPU).

A destroyed handle's device blocks (model data, run workspace) are kept by the
library for the next handle instead of being freed and allocated again.  A
handle that inherits a block must give the bits of a run on fresh memory, for
every model kind and size in any order, and the kept blocks must stay within
the library's bound (1 GB) however many handles come and go."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def _models():
    tree = inputs.yule_tree(24, seed=4)
    return [("lg", dict(obs=inputs.lg_observations(30, seed=2)), 1000),
            ("crbd", dict(tree=tree), 4096),
            ("rateshift", dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1), 3000),
            ("seir", dict(obs=inputs.seir_observations(14, seed=7)), 2048),
            ("crbd_ds", dict(tree=tree), 700),
            ("geometric", {}, 5000)]


def _same(a, b):
    assert a["log_z_value"] == b["log_z_value"] and a["n_segments"] == b["n_segments"]
    for k in ("final_logw", "real_fields", "int_fields", "stack", "ancestors"):
        if k in a:
            np.testing.assert_array_equal(a[k], b[k])


def test_reused_blocks_give_the_same_bits():
    from paper_2112_00364_gb300 import smc

    cases = _models()
    ref = []
    for kind, p, N in cases:  # each on a handle of its own, kept alive meanwhile
        m = smc.Model(kind, **p)
        ref.append((m, smc.run(m, N, 11)))
    for m, _ in ref:
        m.close()
    # new handles, in the reverse order and twice: they inherit the kept blocks
    for rep in range(2):
        for q in reversed(range(len(cases))):
            kind, p, N = cases[q]
            m = smc.Model(kind, **p)
            _same(smc.run(m, N, 11), ref[q][1])
            m.close()


def test_kept_blocks_stay_bounded():
    import torch
    from paper_2112_00364_gb300 import smc

    obs = inputs.lg_observations(20, seed=5)
    m = smc.Model("lg", obs=obs)
    smc.run(m, 1 << 16, 1)
    m.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for q in range(60):  # 60 handles of growing sizes, one at a time
        m = smc.Model("lg", obs=obs)
        smc.run(m, (1 << 14) + 977 * q, 2 + q)
        m.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 <= (1 << 30) + (64 << 20)
