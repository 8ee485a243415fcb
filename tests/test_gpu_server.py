"""Continuous batching (smc_server_*) on the GPU.

Requests submitted while others run are admitted into the running waves; every
result must be identical to what the same request gives alone through smc_run.
Failure paths are exercised on the host: cancellation, a bounded wait that runs
out, a request larger than the memory budget.
"""
import time

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def _requests(n=16, seed=5):
    from paper_2112_00364_gb300 import smc

    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n):
        kind = ["lg", "crbd"][q % 2]
        if kind == "lg":
            p = dict(obs=inputs.lg_observations(int(rng.integers(10, 200)), seed=300 + q))
        else:
            p = dict(tree=inputs.yule_tree(int(rng.integers(4, 64)), seed=400 + q))
        reqs.append((smc.Model(kind, **p), int(rng.integers(100, 20000)), 700 + q, q))
    return reqs


def _same(a, b):
    assert a["run_status"] == b["run_status"]
    assert a["log_z_value"] == b["log_z_value"]
    np.testing.assert_array_equal(a["final_logw"], b["final_logw"])
    np.testing.assert_array_equal(a["int_fields"], b["int_fields"])
    np.testing.assert_array_equal(a["real_fields"], b["real_fields"])
    np.testing.assert_array_equal(a["ancestors"], b["ancestors"])


@pytest.mark.parametrize("budget_mb,precision", [(4096, "fp64"), (24, "fp64"), (4096, "fp32")])
def test_server_results_equal_standalone_runs(budget_mb, precision):
    from paper_2112_00364_gb300 import smc

    reqs = _requests()
    srv = smc.Server(budget_mb << 20, precision=precision)
    tickets = []
    for m, N, seed, rid in reqs:
        tickets.append(srv.submit(m, N, seed, run_id=rid))
        time.sleep(0.002)  # arrivals overlap with resident runs
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["worker_status"] == 0
    for (m, N, seed, rid), g in zip(reqs, got):
        a = smc.run(m, N, seed, run_id=rid, precision=precision)
        _same(g, a)
        assert g["latency_s"] > 0


def test_server_device_outputs_and_record_all():
    import torch
    from paper_2112_00364_gb300 import smc

    reqs = _requests(4, seed=9)
    srv = smc.Server(1 << 30)
    ts = [srv.submit(m, N, seed, run_id=rid, record_all_ancestors=True, where="device")
          for m, N, seed, rid in reqs]
    got = [srv.wait(t) for t in ts]
    srv.close()
    torch.cuda.synchronize()
    for (m, N, seed, rid), g in zip(reqs, got):
        a = smc.run(m, N, seed, run_id=rid, record_all_ancestors=True)
        assert float(g["log_z"].cpu()[0]) == a["log_z_value"]
        np.testing.assert_array_equal(g["ancestors"].cpu().numpy(), a["ancestors"])


def test_server_cancel_timeout_and_oversize():
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(64, seed=2)
    m = smc.Model("crbd", tree=tree)
    srv = smc.Server(64 << 20, max_resident_runs=1)
    t1 = srv.submit(m, 1 << 16, 1)
    t2 = srv.submit(m, 1 << 16, 2)  # waits behind t1 (one resident run at most)
    srv.cancel(t2)
    with pytest.raises(smc.SmcError) as e:
        srv.wait(t1, timeout=0.0)
    assert e.value.status == smc.ETIMEOUT
    r1 = srv.wait(t1)
    assert r1["status"] == 0
    r2 = srv.wait(t2)
    assert r2["status"] == smc.ECANCELLED
    with pytest.raises(smc.SmcError) as e:
        srv.submit(m, 1 << 24, 3)  # workspace larger than the whole budget
    assert e.value.status == smc.ENOMEM
    srv.close()


def test_server_bench_mix_stream():
    """The serving benchmark's request mix at its arrival rate: 400 requests
    drawn as the benchmark draws them (sizes from the batch512 mix, Poisson
    arrivals at 2000 requests/s), FP32, submitted on their arrival times so that
    new runs join waves already in flight.  Every request completes, and each of
    a sample of 40 equals its standalone smc_run bit for bit."""
    from paper_2112_00364_gb300 import smc

    specs = inputs.batch_specs(512, seed=4)
    models = {}
    arr = inputs.poisson_arrivals(2000.0, 0.2, seed=5)[:400]
    rng = np.random.default_rng(5)
    picks = rng.integers(0, len(specs), len(arr))
    srv = smc.Server(96 << 30, precision="fp32")
    tickets, reqs = [], []
    t0 = time.perf_counter()
    for a, q in zip(arr, picks):
        sp = specs[q]
        if q not in models:
            p = (dict(obs=inputs.lg_observations(sp.T, seed=sp.obs_seed)) if sp.kind == "lg"
                 else dict(tree=inputs.yule_tree(sp.tips, seed=sp.tree_seed)))
            models[q] = smc.Model(sp.kind, **p)
        while time.perf_counter() - t0 < a:
            time.sleep(1e-4)
        reqs.append((models[q], sp.n_particles, 1 + sp.seed, int(q)))
        tickets.append(srv.submit(models[q], sp.n_particles, 1 + sp.seed, run_id=int(q)))
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["worker_status"] == 0
    for i in np.random.default_rng(6).choice(len(reqs), 40, replace=False):
        m, N, seed, rid = reqs[i]
        _same(got[i], smc.run(m, N, seed, run_id=rid, precision="fp32"))
    for m in models.values():
        m.close()


def test_server_every_model_kind_and_ess():
    """Requests of every model kind (rate-shift with its PSTATE stack, the
    geometric program with its host-polled length, SEIR, the delayed-sampling
    CRBD), some with ESS-triggered resampling, served together: each equals its
    standalone smc_run bit for bit, ancestors and resampling decisions included."""
    from paper_2112_00364_gb300 import smc

    tree = inputs.yule_tree(24, seed=7)
    cases = [
        (smc.Model("rateshift", tree=tree, sigma=0.3, lam_stack_cap=tree.max_pending_right() + 1),
         3000, 0.0),
        (smc.Model("geometric"), 2000, 0.0),
        (smc.Model("seir", obs=inputs.seir_observations(35, seed=7)), 1500, 0.0),
        (smc.Model("crbd_ds", tree=tree), 4000, 0.5),
        (smc.Model("crbd", tree=tree), 5000, 0.3),
        (smc.Model("lg", obs=inputs.lg_observations(40, seed=2)), 2500, 0.5),
    ]
    srv = smc.Server(4096 << 20, precision="fp64")
    tickets = []
    for q, (m, N, tau) in enumerate(cases * 2):
        tickets.append(srv.submit(m, N, 40 + q, run_id=q, record_all_ancestors=True,
                                  ess_threshold=tau))
        time.sleep(0.001)
    got = [srv.wait(t) for t in tickets]
    srv.close()
    for q, ((m, N, tau), g) in enumerate(zip(cases * 2, got)):
        a = smc.run(m, N, 40 + q, run_id=q, record_all_ancestors=True, ess_threshold=tau)
        assert g["run_status"] == a["run_status"] and g["n_segments"] == a["n_segments"]
        assert g["log_z_value"] == a["log_z_value"]
        np.testing.assert_array_equal(g["final_logw"], a["final_logw"])
        np.testing.assert_array_equal(g["int_fields"], a["int_fields"])
        np.testing.assert_array_equal(g["ancestors"], a["ancestors"])
        if "real_fields" in a:
            np.testing.assert_array_equal(g["real_fields"], a["real_fields"])
        if "resampled" in a:
            np.testing.assert_array_equal(g["resampled"], a["resampled"])
        if "stack" in a:
            np.testing.assert_array_equal(g["stack"], a["stack"])
    for m, _, _ in cases:
        m.close()


def test_server_failed_retirement_fails_only_that_request(monkeypatch):
    """A request whose retirement fails after its result copies were queued
    (injected on the host through SMC_SERVER_FAIL_TICKET) completes at once with
    the error; every other request completes with its standalone result, the
    worker keeps running and no run stays resident."""
    from paper_2112_00364_gb300 import smc

    reqs = _requests(6, seed=13)
    monkeypatch.setenv("SMC_SERVER_FAIL_TICKET", "3")
    srv = smc.Server(4096 << 20)
    monkeypatch.delenv("SMC_SERVER_FAIL_TICKET")
    tickets = [srv.submit(m, N, seed, run_id=rid) for m, N, seed, rid in reqs]
    assert tickets[2] == 3
    t0 = time.perf_counter()
    got = [srv.wait(t, timeout=120.0) for t in tickets]
    assert time.perf_counter() - t0 < 60.0
    st = srv.stats()
    srv.close()
    assert got[2]["status"] == smc.ECUDA
    assert st["worker_status"] == 0 and st["resident"] == 0 and st["completed"] == len(reqs)
    for q, ((m, N, seed, rid), g) in enumerate(zip(reqs, got)):
        if q != 2:
            _same(g, smc.run(m, N, seed, run_id=rid))
        m.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_served_results_equal_the_oracle(precision):
    """Served results checked against the oracle itself (not only against
    smc_run): twelve requests of the serving benchmark's mix (the smallest of
    its linear-Gaussian and CRBD sizes, so that the oracle finishes quickly),
    submitted together so that they share waves, each with every resampling's
    ancestors recorded; each result equals the oracle in follow mode element by
    element (bit for bit in FP32, to FP64 rounding in FP64)."""
    import oracle
    from parity import assert_parity_exact, assert_parity_fp64

    from paper_2112_00364_gb300 import smc

    specs = inputs.batch_specs(512, seed=4)
    sizes = np.array([sp.n_particles * sp.n_segments() for sp in specs])
    order = [int(q) for q in np.argsort(sizes)]
    pick = [q for q in order if specs[q].kind == "lg"][:6] + \
        [q for q in order if specs[q].kind == "crbd"][:6]
    srv = smc.Server(4096 << 20, precision=precision)
    reqs = []
    for q in pick:
        sp = specs[q]
        p = (dict(obs=inputs.lg_observations(sp.T, seed=sp.obs_seed)) if sp.kind == "lg"
             else dict(tree=inputs.yule_tree(sp.tips, seed=sp.tree_seed)))
        m = smc.Model(sp.kind, **p)
        t = srv.submit(m, sp.n_particles, 1 + sp.seed, run_id=q, record_all_ancestors=True)
        reqs.append((sp, p, m, t, q))
    got = [srv.wait(t) for _, _, _, t, _ in reqs]
    srv.close()
    for (sp, p, m, _, q), g in zip(reqs, got):
        g["status"] = g["run_status"]
        o = oracle.smc_run(sp.kind, sp.n_particles, 1 + sp.seed, run_id=q,
                           precision=oracle.FP32 if precision == "fp32" else oracle.FP64,
                           follow=g["ancestors"], record_ancestors=True, **p)
        if precision == "fp32":
            assert_parity_exact(g, o)
        else:
            assert_parity_fp64(g, o)
        m.close()
