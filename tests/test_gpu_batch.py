"""Batched execution (smc_run_batch) on the GPU.

Every run of a mixed batch must give exactly what it gives alone through
smc_run (its tiling depends only on its own N), and agree with the oracle.
"""
import numpy as np
import pytest

import inputs
import oracle
from parity import assert_parity_exact, assert_parity_fp64

pytestmark = pytest.mark.gpu


def _mixed(precision="fp64"):
    from paper_2112_00364_gb300 import smc

    rng = np.random.default_rng(11)
    models, specs, params = [], [], []
    for q in range(12):
        kind = ["lg", "crbd", "rateshift", "geometric"][q % 4]
        N = int(rng.integers(1, 6000)) if q % 3 else int(rng.integers(20000, 40000))
        if kind == "lg":
            p = dict(obs=inputs.lg_observations(int(rng.integers(5, 80)), seed=100 + q))
        elif kind in ("crbd", "rateshift"):
            tree = inputs.yule_tree(int(rng.integers(3, 40)), seed=200 + q)
            p = dict(tree=tree)
            if kind == "rateshift":
                p.update(sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1)
        else:
            p = {}
        models.append(smc.Model(kind, **p))
        specs.append(dict(N=N, seed=1000 + q, run_id=q))
        params.append((kind, p))
    return models, specs, params


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_individual_runs(precision):
    from paper_2112_00364_gb300 import smc

    models, specs, _ = _mixed(precision)
    batch = smc.run_batch(models, specs, precision=precision, record_all_ancestors=True)
    for m, sp, b in zip(models, specs, batch):
        a = smc.run(m, sp["N"], sp["seed"], run_id=sp["run_id"], precision=precision,
                    record_all_ancestors=True)
        assert b["run_status"] == a["run_status"]
        assert b["log_z_value"] == a["log_z_value"]
        assert b["n_segments"] == a["n_segments"]
        np.testing.assert_array_equal(b["ancestors"], a["ancestors"])
        np.testing.assert_array_equal(b["final_logw"], a["final_logw"])
        np.testing.assert_array_equal(b["int_fields"], a["int_fields"])
        if "real_fields" in a:
            np.testing.assert_array_equal(b["real_fields"], a["real_fields"])


def test_batch_runs_match_oracle():
    from paper_2112_00364_gb300 import smc

    models, specs, params = _mixed()
    batch = smc.run_batch(models, specs, record_all_ancestors=True)
    for (kind, p), sp, b in zip(params, specs, batch):
        o = oracle.smc_run(kind, sp["N"], sp["seed"], run_id=sp["run_id"], follow=b["ancestors"],
                           record_ancestors=True, **p)
        b = dict(b, status=b["run_status"])
        assert_parity_fp64(b, o)


def test_batch_of_one_and_device_outputs():
    import torch
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(16, seed=2)
    m = smc.Model("crbd", tree=tree)
    b = smc.run_batch([m], [dict(N=5000, seed=3)], where="device")
    a = smc.run(m, 5000, 3)
    torch.cuda.synchronize()
    assert float(b[0]["log_z"].cpu()[0]) == a["log_z_value"]


def test_batch512_bench_workload():
    """The batched benchmark workload in full: the 512 runs of the seeded mix
    (half linear-Gaussian, half CRBD, N log-uniform 256..65,536), FP32 particles,
    seeds as the benchmark's first rank draws them.  Every run finishes with a
    finite log Z; a sample of 32 runs (the 8 smallest, 8 largest and 16 drawn at
    random) give exactly what they give alone through smc_run; the 2 smallest
    CRBD and the 2 smallest linear-Gaussian runs also equal the FP32 oracle in
    follow mode, element by element."""
    from paper_2112_00364_gb300 import smc

    specs = inputs.batch_specs(512, seed=4)
    models, runspecs, params = [], [], []
    for q, sp in enumerate(specs):
        if sp.kind == "lg":
            p = dict(obs=inputs.lg_observations(sp.T, seed=sp.obs_seed))
        else:
            p = dict(tree=inputs.yule_tree(sp.tips, seed=sp.tree_seed))
        models.append(smc.Model(sp.kind, **p))
        runspecs.append(dict(N=sp.n_particles, seed=1 + sp.seed, run_id=q))
        params.append((sp.kind, p))
    batch = smc.run_batch(models, runspecs, precision="fp32")
    assert all(b["run_status"] == 0 and np.isfinite(b["log_z_value"]) for b in batch)
    sizes = np.array([sp.n_particles * sp.n_segments() for sp in specs])
    order = np.argsort(sizes)
    rng = np.random.default_rng(3)
    pick = set(order[:8]) | set(order[-8:]) | set(rng.choice(512, 16, replace=False).tolist())
    for q in sorted(pick):
        sp = runspecs[q]
        a = smc.run(models[q], sp["N"], sp["seed"], run_id=sp["run_id"], precision="fp32")
        b = batch[q]
        assert b["log_z_value"] == a["log_z_value"], q
        assert b["n_segments"] == a["n_segments"]
        np.testing.assert_array_equal(b["ancestors"], a["ancestors"])
        np.testing.assert_array_equal(b["final_logw"], a["final_logw"])
        np.testing.assert_array_equal(b["int_fields"], a["int_fields"])
    small = [q for q in order if params[q][0] == "crbd"][:2] + \
        [q for q in order if params[q][0] == "lg"][:2]
    for q in small:
        kind, p = params[q]
        sp = runspecs[q]
        g = smc.run(models[q], sp["N"], sp["seed"], run_id=sp["run_id"], precision="fp32",
                    record_all_ancestors=True)
        o = oracle.smc_run(kind, sp["N"], sp["seed"], run_id=sp["run_id"],
                           precision=oracle.FP32, follow=g["ancestors"], record_ancestors=True,
                           **p)
        assert_parity_exact(g, o)
    for m in models:
        m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_every_model_kind_and_ess(precision):
    """A batch holding every model kind (SEIR and the delayed-sampling CRBD
    among them), some runs with ESS-triggered resampling at their own
    thresholds: each run equals its standalone smc_run bit for bit, resampling
    decisions included."""
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(20, seed=9)
    models = [smc.Model("seir", obs=inputs.seir_observations(28, seed=7)),
              smc.Model("crbd_ds", tree=tree),
              smc.Model("crbd", tree=tree),
              smc.Model("lg", obs=inputs.lg_observations(30, seed=4)),
              smc.Model("geometric"),
              smc.Model("rateshift", tree=tree, sigma=0.3,
                        lam_stack_cap=tree.max_pending_right() + 1)]
    specs = [dict(N=1200, seed=11, run_id=0), dict(N=3000, seed=12, run_id=1, ess_threshold=0.5),
             dict(N=2500, seed=13, run_id=2, ess_threshold=0.3), dict(N=700, seed=14, run_id=3),
             dict(N=900, seed=15, run_id=4, ess_threshold=0.6), dict(N=1800, seed=16, run_id=5)]
    batch = smc.run_batch(models, specs, precision=precision, record_all_ancestors=True)
    for m, sp, b in zip(models, specs, batch):
        a = smc.run(m, sp["N"], sp["seed"], run_id=sp["run_id"], precision=precision,
                    record_all_ancestors=True, ess_threshold=sp.get("ess_threshold", 0.0))
        assert b["run_status"] == a["run_status"] and b["n_segments"] == a["n_segments"]
        assert b["log_z_value"] == a["log_z_value"]
        np.testing.assert_array_equal(b["ancestors"], a["ancestors"])
        np.testing.assert_array_equal(b["final_logw"], a["final_logw"])
        np.testing.assert_array_equal(b["int_fields"], a["int_fields"])
        if "real_fields" in a:
            np.testing.assert_array_equal(b["real_fields"], a["real_fields"])
        if "resampled" in a:
            np.testing.assert_array_equal(b["resampled"], a["resampled"])
    for m in models:
        m.close()


def test_graph_launch_gives_the_same_bits():
    """Waves launched as one captured CUDA graph give exactly the results of the
    same waves launched one by one: smc_run (the graph kept in the model handle
    and launched again for new seeds, captured again when N changes) and
    smc_run_batch (captured per call), FP64 and FP32."""
    import torch
    from paper_2112_00364_gb300 import smc

    s = torch.cuda.Stream()
    tree = inputs.yule_tree(24, seed=5)
    m = smc.Model("crbd", tree=tree)
    for N, seed, prec in [(3000, 1, "fp64"), (3000, 2, "fp64"), (3000, 3, "fp32"),
                          (777, 4, "fp64"), (3000, 5, "fp64")]:
        a = smc.run(m, N, seed, precision=prec, stream=s, record_all_ancestors=True)
        g = smc.run(m, N, seed, precision=prec, stream=s, record_all_ancestors=True,
                    launch_graph=True)
        assert g["log_z_value"] == a["log_z_value"] and g["n_segments"] == a["n_segments"]
        np.testing.assert_array_equal(g["ancestors"], a["ancestors"])
        np.testing.assert_array_equal(g["final_logw"], a["final_logw"])
        np.testing.assert_array_equal(g["real_fields"], a["real_fields"])
    specs = inputs.batch_specs(24, seed=8)
    models = [smc.Model(sp.kind, **(dict(obs=inputs.lg_observations(sp.T, seed=sp.obs_seed))
                                    if sp.kind == "lg" else
                                    dict(tree=inputs.yule_tree(sp.tips, seed=sp.tree_seed))))
              for sp in specs]
    rs = [dict(N=sp.n_particles, seed=sp.seed, run_id=q) for q, sp in enumerate(specs)]
    for prec in ("fp32", "fp64"):
        a = smc.run_batch(models, rs, precision=prec, stream=s)
        g = smc.run_batch(models, rs, precision=prec, stream=s, launch_graph=True)
        for x, y in zip(a, g):
            assert x["log_z_value"] == y["log_z_value"]
            np.testing.assert_array_equal(x["final_logw"], y["final_logw"])
            np.testing.assert_array_equal(x["ancestors"], y["ancestors"])
    for mm in models + [m]:
        mm.close()


@pytest.mark.parametrize("launch", ["one_cta", "cluster"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_launch_forms_give_the_same_bits(precision, launch):
    """A small run (32-particle tiles, few enough for one CTA or one cluster)
    launched as one CTA, or one thread-block cluster, that runs every segment
    gives exactly what its waves give, for every model kind, ESS-triggered
    resampling and record_all included; one case against the oracle too."""
    import oracle
    from parity import assert_parity_exact, assert_parity_fp64

    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(20, seed=9)
    cases = [("lg", dict(obs=inputs.lg_observations(40, seed=3)), 1024, 0.0),
             ("lg", dict(obs=inputs.lg_observations(25, seed=4)), 700, 0.5),
             ("geometric", {}, 999, 0.0),
             ("crbd", dict(tree=tree), 512, 0.0),
             ("rateshift", dict(tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1),
              480, 0.5),
             ("crbd_ds", dict(tree=tree), 300, 0.5),
             ("seir", dict(obs=inputs.seir_observations(21, seed=7)), 512, 0.0)]
    if launch == "cluster":  # up to 32 tiles for every model, the last CTA half full
        cases += [("crbd", dict(tree=tree), 1024, 0.5),
                  ("seir", dict(obs=inputs.seir_observations(21, seed=7)), 1000, 0.0),
                  ("crbd_ds", dict(tree=tree), 33, 0.0)]
    for q, (kind, p, N, tau) in enumerate(cases):
        m = smc.Model(kind, **p)
        kw = dict(precision=precision, record_all_ancestors=True, ess_threshold=tau)
        a = smc.run(m, N, 60 + q, launch="waves", **kw)
        b = smc.run(m, N, 60 + q, launch=launch, **kw)
        assert b["kernel_launches"] == 1, kind
        assert a["log_z_value"] == b["log_z_value"] and a["n_segments"] == b["n_segments"], kind
        for key in ("final_logw", "int_fields", "ancestors", "resampled", "real_fields", "stack"):
            if key in a:
                np.testing.assert_array_equal(a[key], b[key])
        assert (a["n_near_boundary"], a["n_draws"], a["n_blocks"]) == \
            (b["n_near_boundary"], b["n_draws"], b["n_blocks"])
        if q == 3:
            o = oracle.smc_run(kind, N, 60 + q, follow=b["ancestors"], record_ancestors=True,
                               precision=oracle.FP64 if precision == "fp64" else oracle.FP32, **p)
            (assert_parity_fp64 if precision == "fp64" else assert_parity_exact)(b, o)
        m.close()
