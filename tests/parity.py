"""Helpers for GPU-vs-oracle parity checks (test infrastructure).

A run is compared with the oracle in follow mode: the oracle computes its
own systematic-resampling ancestors at every checkpoint and compares them
with the GPU's element by element.  A differing ancestor is allowed only if
the oracle flags that offset as lying within 1e-12 N of a cumulative-weight
boundary (the two sides sum the weights in different orders); the oracle
then adopts the GPU's choice so the rest of the run stays comparable.

In FP32-particle mode both sides perform the same single-precision operations
(the mode's own log / exp / cos(2 pi u) / log1p / expm1 / log k! included), so
a run's log-weights and states are identical bit for bit and its ancestors
differ only at flagged offsets; log Z, summed in FP64 on both sides, agrees to
the FP64 tolerance.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2112_00364_gb300 import smc

LOGZ_RTOL_FP64 = 1e-9  # log-Z tolerance at FP64 (relative)
STATE_RTOL_FP64 = 1e-12  # final FP64 states / log-weights (relative)


def run_pair(kind: str, N: int, seed: int, precision: str = "fp64", run_id: int = 0,
             ess_threshold: float = 0.0, **params):
    model = smc.Model(kind, **params)
    g = smc.run(model, N, seed, run_id=run_id, precision=precision, record_all_ancestors=True,
                ess_threshold=ess_threshold)
    o = oracle.smc_run(kind, N, seed, run_id=run_id,
                       precision=oracle.FP64 if precision == "fp64" else oracle.FP32,
                       follow=g["ancestors"], record_ancestors=True, ess_threshold=ess_threshold,
                       follow_resampled=g["resampled"] if ess_threshold > 0 else None, **params)
    model.close()
    return g, o


def assert_parity_fp64(g, o, logz_rtol=LOGZ_RTOL_FP64, state_rtol=STATE_RTOL_FP64):
    # the library reports particles killed by the depth cap / call limit as a
    # warning status; the oracle reports the same events only as counts
    g_status = 0 if g["status"] == smc.WKILLED else g["status"]
    assert g_status == o["status"], (g["status"], o["status"])
    if g["status"] == smc.WKILLED:
        assert o["n_overflow"] + o["n_limit"] > 0
    assert g["n_segments"] == o["n_segments"]
    assert g["n_resamples"] == o["n_resamples"]
    assert o["n_hard_mismatch"] == 0, o["n_hard_mismatch"]
    assert o["n_dec_hard_mismatch"] == 0, o["n_dec_hard_mismatch"]
    lz_g, lz_o = g["log_z_value"], o["log_z"]
    if np.isfinite(lz_o):
        assert abs(lz_g - lz_o) <= logz_rtol * max(1.0, abs(lz_o)), (lz_g, lz_o)
    else:
        assert lz_g == lz_o
    np.testing.assert_allclose(g["final_logw"], o["final_logw"], rtol=state_rtol, atol=state_rtol)
    if "real_fields" in g:
        np.testing.assert_allclose(g["real_fields"], o["real_fields"], rtol=state_rtol,
                                   atol=state_rtol)
    np.testing.assert_array_equal(g["int_fields"], o["int_fields"])
    assert g["n_overflow"] == o["n_overflow"] and g["n_limit"] == o["n_limit"]


def assert_parity_exact(g, o, logz_rtol=LOGZ_RTOL_FP64):
    """Element-wise identity of an FP32-mode run with the FP32 oracle in follow
    mode: no unflagged ancestor or resampling-decision difference, log Z within
    the FP64 tolerance, and every final log-weight and state field equal bit for
    bit (FP32 values widened to f64 on both sides)."""
    g_status = 0 if g["status"] == smc.WKILLED else g["status"]
    assert g_status == o["status"], (g["status"], o["status"])
    assert g["n_segments"] == o["n_segments"]
    assert g["n_resamples"] == o["n_resamples"]
    assert o["n_hard_mismatch"] == 0, (o["n_hard_mismatch"], o["n_flag_mismatch"])
    assert o["n_dec_hard_mismatch"] == 0, o["n_dec_hard_mismatch"]
    lz_g, lz_o = g["log_z_value"], o["log_z"]
    if np.isfinite(lz_o):
        assert abs(lz_g - lz_o) <= logz_rtol * max(1.0, abs(lz_o)), (lz_g, lz_o)
    else:
        assert lz_g == lz_o
    np.testing.assert_array_equal(g["final_logw"], o["final_logw"])
    if "real_fields" in g:
        np.testing.assert_array_equal(g["real_fields"], o["real_fields"])
    np.testing.assert_array_equal(g["int_fields"], o["int_fields"])
    if g.get("stack") is not None and o.get("stack") is not None:
        np.testing.assert_array_equal(g["stack"], o["stack"])
    assert g["n_overflow"] == o["n_overflow"] and g["n_limit"] == o["n_limit"]
