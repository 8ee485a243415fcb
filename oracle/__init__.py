"""CPU oracle for the particle-SMC sweep over a PPL control-flow graph.

TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded C restatement of
Algorithm 1 (SMC over PCFGs) and the models it runs, compiled with gcc and
loaded through ctypes.  It shares no code with the CUDA library and imports
nothing from it.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it.

See smc_oracle.c for the passages of the paper each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_DIR = Path(__file__).resolve().parent
_SRC = [_DIR / "smc_oracle.c"]
_DEPS = _SRC + [_DIR / "smc_oracle.h", _DIR / "smc_oracle_prec.inc"]
_LIB_PATH = _DIR / "liboracle.so"

LG, CRBD, RATESHIFT, GEOMETRIC, SEIR, CRBD_DS = 1, 2, 3, 4, 5, 6
FP64, FP32 = 0, 1
OK, EINVAL, ENOMEM, EDEGENERATE, ESTEPLIMIT = 0, -1, -2, -4, -5

DIST = {"uniform": 0, "normal": 1, "exponential": 2, "gamma1": 3, "uniform_ab": 4,
        "bernoulli": 5, "poisson": 6, "lognormal": 7, "binomial": 8, "beta": 9, "gamma": 10,
        "neg_binomial": 11, "lomax": 12,
        "neg_binomial_rate": 13}

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)


class OrcModel(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("precision", C.c_int32), ("T", C.c_int32), ("n_nodes", C.c_int32),
        ("obs", _f64p),
        ("x0_mean", C.c_double), ("x0_sd", C.c_double), ("a", C.c_double), ("b", C.c_double),
        ("q_sd", C.c_double), ("r_sd", C.c_double),
        ("parent", _i32p), ("left", _i32p), ("right", _i32p), ("preorder", _i32p),
        ("age", _f64p),
        ("rho", C.c_double), ("lambda_fixed", C.c_double), ("mu_fixed", C.c_double),
        ("lambda_scale", C.c_double), ("mu_scale", C.c_double), ("sigma", C.c_double),
        ("fixed_mult", _f64p),
        ("fixed_rates", C.c_int32), ("depth_cap", C.c_int32), ("call_limit", C.c_int32),
        ("lam_stack_cap", C.c_int32),
        ("geo_p", C.c_double), ("geo_logw", C.c_double),
    ]


class OrcCfg(C.Structure):
    _fields_ = [("N", C.c_int64), ("seed", C.c_uint64), ("run_id", C.c_uint32),
                ("max_segments", C.c_int32), ("follow_anc", _i32p), ("n_follow", C.c_int32),
                ("pad_", C.c_int32), ("ess_threshold", C.c_double), ("follow_resampled", _i32p),
                ("n_follow_resampled", C.c_int32), ("pad2_", C.c_int32),
                ("resume_k", C.c_int32), ("pad3_", C.c_int32), ("resume_logw", _f64p),
                ("resume_real", _f64p), ("resume_int", _i32p), ("resume_stack", _f64p),
                ("resume_log_z", C.c_double)]


class OrcOut(C.Structure):
    _fields_ = [
        ("log_z", C.c_double), ("n_flagged", C.c_int64), ("n_flag_mismatch", C.c_int64),
        ("n_hard_mismatch", C.c_int64), ("n_overflow", C.c_int64), ("n_limit", C.c_int64),
        ("n_ess_flagged", C.c_int64), ("n_dec_flag_mismatch", C.c_int64),
        ("n_dec_hard_mismatch", C.c_int64),
        ("n_segments", C.c_int32), ("n_resamples", C.c_int32),
        ("final_logw", _f64p), ("real_fields", _f64p), ("int_fields", _i32p), ("stack", _f64p),
        ("ancestors", _i32p), ("resampled", _i32p), ("incr", _f64p), ("anc_capacity", C.c_int32),
        ("incr_capacity", C.c_int32), ("log_z_closed", C.c_double),
    ]


def build(force: bool = False) -> Path:
    """Compile liboracle.so with gcc (plain C11, no FP contraction)."""
    if not force and _LIB_PATH.exists():
        newest = max(p.stat().st_mtime for p in _DEPS)
        if _LIB_PATH.stat().st_mtime >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH.with_suffix(f".so.tmp{os.getpid()}")
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-Wno-unused-function",
           "-Wno-unused-parameter", "-o", str(tmp)] + [str(s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_LIB_PATH))
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_philox_many.argtypes = [C.c_int64, _u32p, _u32p, _u32p]
        L.orc_sample.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                 C.c_uint32, C.c_int64, _f64p, _i32p]
        L.orc_sample.restype = C.c_int
        L.orc_resample.argtypes = [_f64p, C.c_int64, C.c_double, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.orc_resample.restype = C.c_int
        L.orc_smc_run.argtypes = [C.POINTER(OrcModel), C.POINTER(OrcCfg), C.POINTER(OrcOut)]
        L.orc_smc_run.restype = C.c_int
        L.orc_n_fields.argtypes = [C.POINTER(OrcModel), _i32p, _i32p, _i32p]
        L.orc_n_fields.restype = C.c_int
        L.orc_mathf.argtypes = [C.c_int32, _f64p, _f64p, C.c_int64]
        L.orc_mathf.restype = C.c_int
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Raw Philox4x32-10 blocks.  ctr: uint32 [n,4], key: uint32 [n,2] -> uint32 [n,4]."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().orc_philox_many(ctr.shape[0], _p(ctr, C.c_uint32), _p(key, C.c_uint32),
                          _p(out, C.c_uint32))
    return out


def sample(dist: str, n: int, p1: float = 0.0, p2: float = 0.0, seed: int = 1, run_id: int = 0,
           precision: int = FP64, return_blocks: bool = False):
    """n independent variates; variate i uses counter (i, 0, d, 0)."""
    out = np.empty(n, dtype=np.float64)
    blocks = np.empty(n, dtype=np.int32)
    rc = lib().orc_sample(DIST[dist], precision, p1, p2, seed, run_id, n, _p(out, C.c_double),
                          _p(blocks, C.c_int32))
    if rc != OK:
        raise ValueError(f"orc_sample rc={rc}")
    return (out, blocks) if return_blocks else out


MATHF = {"log": 0, "exp": 1, "cos2pi": 2, "log1p": 3, "expm1": 4, "lfact": 5}


def mathf(fn: str, x) -> np.ndarray:
    """The FP32 mode's single-precision function `fn` of float32(x) (log k! of
    int(x) for "lfact"), widened to float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    rc = lib().orc_mathf(MATHF[fn], _p(x, C.c_double), _p(y, C.c_double), x.shape[0])
    if rc != OK:
        raise ValueError(f"orc_mathf rc={rc}")
    return y


def resample(logw: np.ndarray, u: float):
    """FP64 normaliser + systematic resampling of one population.
    Returns (ancestors, flags, increment, m, S)."""
    logw = np.ascontiguousarray(logw, dtype=np.float64)
    N = logw.shape[0]
    anc = np.empty(N, dtype=np.int32)
    flag = np.empty(N, dtype=np.int32)
    incr, m, S = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_resample(_p(logw, C.c_double), N, u, _p(anc, C.c_int32), _p(flag, C.c_int32),
                            C.byref(incr), C.byref(m), C.byref(S))
    return anc, flag, incr.value, m.value, S.value, rc


def _model_struct(kind: int, precision: int, keep: list, *, obs=None, tree=None,
                  x0_mean=0.0, x0_sd=1.0, a=0.9, b=0.0, q_sd=1.0, r_sd=0.5, rho=1.0,
                  rates=None, lambda_scale=1.0, mu_scale=0.5, sigma=0.3, fixed_mult=None,
                  depth_cap=64, call_limit=1 << 16, lam_stack_cap=0, geo_p=0.5,
                  geo_logw=float(np.log(1.5))):
    m = OrcModel()
    m.kind, m.precision = kind, precision
    m.x0_mean, m.x0_sd, m.a, m.b, m.q_sd, m.r_sd = x0_mean, x0_sd, a, b, q_sd, r_sd
    if obs is not None:
        obs = np.ascontiguousarray(obs, dtype=np.float64)
        keep.append(obs)
        m.obs, m.T = _p(obs, C.c_double), obs.shape[0]
    if tree is not None:
        arrs = {k: np.ascontiguousarray(getattr(tree, k), dtype=np.int32)
                for k in ("parent", "left", "right", "preorder")}
        age = np.ascontiguousarray(tree.age, dtype=np.float64)
        keep.extend(list(arrs.values()) + [age])
        m.parent, m.left, m.right, m.preorder = (_p(arrs[k], C.c_int32)
                                                 for k in ("parent", "left", "right", "preorder"))
        m.age, m.n_nodes = _p(age, C.c_double), tree.n_nodes
    m.rho = rho
    if rates is not None:
        m.fixed_rates, m.lambda_fixed, m.mu_fixed = 1, rates[0], rates[1]
    m.lambda_scale, m.mu_scale, m.sigma = lambda_scale, mu_scale, sigma
    if fixed_mult is not None:
        fm = np.ascontiguousarray(fixed_mult, dtype=np.float64)
        keep.append(fm)
        m.fixed_mult = _p(fm, C.c_double)
    m.depth_cap, m.call_limit, m.lam_stack_cap = depth_cap, call_limit, lam_stack_cap
    m.geo_p, m.geo_logw = geo_p, geo_logw
    return m


KINDS = {"lg": LG, "crbd": CRBD, "rateshift": RATESHIFT, "geometric": GEOMETRIC, "seir": SEIR,
         "crbd_ds": CRBD_DS}


def smc_run(model: str, N: int, seed: int, run_id: int = 0, precision: int = FP64,
            max_segments: int = 1 << 20, follow=None, record_ancestors: bool = False,
            record_incr: bool = False, ess_threshold: float = 0.0, follow_resampled=None,
            resume_from: dict | None = None, **params) -> dict:
    """Run the oracle SMC once.  `model` is one of lg / crbd / rateshift / geometric;
    params: obs, tree, rates=(lambda, mu), rho, sigma, fixed_mult, depth_cap,
    call_limit, lam_stack_cap, x0_mean, x0_sd, a, b, q_sd, r_sd, geo_p, geo_logw.
    follow: int32 [transitions, N] ancestors from another implementation (row k:
    after checkpoint k); ess_threshold tau > 0: resample only when ESS < tau N;
    follow_resampled: int32 [transitions] another implementation's decisions.
    resume_from: the result of a run of the same model, N, seed and run_id that
    max_segments stopped (a snapshot); this run continues it from there."""
    keep: list = []
    m = _model_struct(KINDS[model], precision, keep, **params)
    nr, ni, sc = C.c_int32(), C.c_int32(), C.c_int32()
    lib().orc_n_fields(C.byref(m), C.byref(nr), C.byref(ni), C.byref(sc))
    nr, ni, sc = nr.value, ni.value, sc.value
    cfg = OrcCfg()
    cfg.N, cfg.seed, cfg.run_id, cfg.max_segments = N, seed, run_id, max_segments
    if follow is not None:
        follow = np.ascontiguousarray(follow, dtype=np.int32)
        keep.append(follow)
        cfg.follow_anc, cfg.n_follow = _p(follow, C.c_int32), follow.shape[0]
    cfg.ess_threshold = ess_threshold
    if follow_resampled is not None:
        follow_resampled = np.ascontiguousarray(follow_resampled, dtype=np.int32)
        keep.append(follow_resampled)
        cfg.follow_resampled = _p(follow_resampled, C.c_int32)
        cfg.n_follow_resampled = follow_resampled.shape[0]
    if resume_from is not None:
        snap = {k: np.ascontiguousarray(resume_from[k2], dtype=dt) for k, k2, dt in
                (("logw", "final_logw", np.float64), ("ints", "int_fields", np.int32))}
        keep.extend(snap.values())
        cfg.resume_k = int(resume_from["n_segments"])
        cfg.resume_log_z = float(resume_from["log_z_closed"])
        cfg.resume_logw, cfg.resume_int = _p(snap["logw"], C.c_double), _p(snap["ints"], C.c_int32)
        if nr > 0:
            rf = np.ascontiguousarray(resume_from["real_fields"], dtype=np.float64)
            keep.append(rf)
            cfg.resume_real = _p(rf, C.c_double)
        if sc > 0:
            st = np.ascontiguousarray(resume_from["stack"], dtype=np.float64)
            keep.append(st)
            cfg.resume_stack = _p(st, C.c_double)
    o = OrcOut()
    logw = np.empty(N)
    real = np.empty((max(nr, 1), N))
    ints = np.empty((ni, N), dtype=np.int32)
    stack = np.empty((max(sc, 1), N))
    o.final_logw, o.real_fields, o.int_fields = _p(logw, C.c_double), _p(real, C.c_double), _p(ints, C.c_int32)
    o.stack = _p(stack, C.c_double)
    cap_seg = min(max_segments, _segments_hint(model, params))
    anc = incr = None
    resampled = np.zeros(cap_seg, dtype=np.int32)
    o.resampled = _p(resampled, C.c_int32)
    o.anc_capacity = cap_seg
    if record_ancestors:
        anc = np.empty((cap_seg, N), dtype=np.int32)
        o.ancestors = _p(anc, C.c_int32)
    if record_incr:
        incr = np.empty(cap_seg)
        o.incr, o.incr_capacity = _p(incr, C.c_double), cap_seg
    rc = lib().orc_smc_run(C.byref(m), C.byref(cfg), C.byref(o))
    res = dict(status=rc, log_z=o.log_z, log_z_closed=o.log_z_closed, n_segments=o.n_segments,
               n_resamples=o.n_resamples,
               n_flagged=o.n_flagged, n_flag_mismatch=o.n_flag_mismatch,
               n_hard_mismatch=o.n_hard_mismatch, n_overflow=o.n_overflow, n_limit=o.n_limit,
               n_ess_flagged=o.n_ess_flagged, n_dec_flag_mismatch=o.n_dec_flag_mismatch,
               n_dec_hard_mismatch=o.n_dec_hard_mismatch,
               resampled=resampled[: max(0, min(o.n_segments - 1, cap_seg))],
               final_logw=logw, real_fields=real[:nr], int_fields=ints,
               stack=stack[:sc] if sc else None)
    if anc is not None:
        res["ancestors"] = anc[: max(0, min(o.n_segments - 1, cap_seg))]
    if incr is not None:
        res["incr"] = incr[: min(o.n_segments, cap_seg)]
    return res


def _segments_hint(model: str, params: dict) -> int:
    if model in ("lg", "seir"):
        return len(params["obs"])
    if model in ("crbd", "rateshift", "crbd_ds"):
        return params["tree"].n_nodes
    return 4096
