"""Python binding of the C ABI in include/smc.h (ctypes, argument marshalling only).

Every step of the SMC path runs in the CUDA library ``libsmc.so``; this module
only builds the C structs, hands over host (numpy) or device (torch CUDA)
pointers and raises on a negative status.  There is no fallback: if the
library cannot be loaded the import of ``lib()`` fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libsmc.so"

OK, EINVAL, ENOMEM, ECUDA, EDEGENERATE, ESTEPLIMIT, ETIMEOUT, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
ECANCELLED = -8
WKILLED = 1
MODEL_LG, MODEL_CRBD, MODEL_RATESHIFT, MODEL_GEOMETRIC, MODEL_SEIR, MODEL_CRBD_DS = 1, 2, 3, 4, 5, 6
KINDS = {"lg": MODEL_LG, "crbd": MODEL_CRBD, "rateshift": MODEL_RATESHIFT,
         "geometric": MODEL_GEOMETRIC, "seir": MODEL_SEIR, "crbd_ds": MODEL_CRBD_DS}
PREC_FP64, PREC_FP32 = 0, 1
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32}
MEM_HOST, MEM_DEVICE = 0, 1
MAX_DEPTH = 64
MAX_PARTICLES = (1 << 31) - 257  # SMC_MAX_PARTICLES
DIST = {"uniform": 0, "normal": 1, "exponential": 2, "gamma1": 3, "uniform_ab": 4,
        "bernoulli": 5, "poisson": 6, "lognormal": 7, "binomial": 8, "beta": 9, "gamma": 10,
        "neg_binomial": 11, "lomax": 12}

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_vp = C.c_void_p


class SmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"smc status {status}: {msg}")
        self.status = status


class ModelDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("T", C.c_int32), ("n_nodes", C.c_int32), ("fixed_rates", C.c_int32),
        ("obs", _f64p),
        ("x0_mean", C.c_double), ("x0_sd", C.c_double), ("a", C.c_double), ("b", C.c_double),
        ("q_sd", C.c_double), ("r_sd", C.c_double),
        ("parent", _i32p), ("left", _i32p), ("right", _i32p), ("preorder", _i32p),
        ("age", _f64p),
        ("rho", C.c_double), ("lambda_fixed", C.c_double), ("mu_fixed", C.c_double),
        ("lambda_scale", C.c_double), ("mu_scale", C.c_double), ("sigma", C.c_double),
        ("fixed_mult", _f64p),
        ("depth_cap", C.c_int32), ("call_limit", C.c_int32), ("lam_stack_cap", C.c_int32),
        ("pad_", C.c_int32),
        ("geo_p", C.c_double), ("geo_logw", C.c_double),
    ]


class RunCfg(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("seed", C.c_uint64), ("run_id", C.c_uint32),
                ("precision", C.c_int32), ("max_segments", C.c_int32),
                ("record_all_ancestors", C.c_int32), ("time_kernels", C.c_int32),
                ("launch_mode", C.c_int32), ("workspace", _vp),
                ("workspace_bytes", C.c_size_t), ("ess_threshold", C.c_double),
                ("resume_k", C.c_int32), ("resume_where", C.c_int32), ("resume_logw", _vp),
                ("resume_real", _vp), ("resume_int", _vp), ("resume_stack", _vp),
                ("resume_log_z", C.c_double)]


class Counters(C.Structure):
    _fields_ = [("n_segments", C.c_int32), ("n_resamples", C.c_int32),
                ("n_near_boundary", C.c_int64), ("n_overflow", C.c_int64),
                ("n_limit", C.c_int64), ("device_ms", C.c_double), ("kernel_ms", C.c_double),
                ("kernel_launches", C.c_int32), ("n_ess_near", C.c_int32), ("status", C.c_int32),
                ("pad2_", C.c_int32), ("n_draws", C.c_int64), ("n_blocks", C.c_int64),
                ("log_z_closed", C.c_double), ("debug_code", C.c_int32), ("pad3_", C.c_int32),
                ("debug_index", C.c_int64), ("debug_count", C.c_int64)]


class Result(C.Structure):
    _fields_ = [("where", C.c_int32), ("ancestors_rows", C.c_int32), ("log_z", _vp),
                ("final_logw", _vp), ("ancestors", _vp), ("real_fields", _vp),
                ("int_fields", _vp), ("stack", _vp), ("resampled", _vp), ("counters", Counters)]


class TileBand(C.Structure):
    _fields_ = [("n_max", C.c_int64), ("slots", C.c_int32), ("tile_min", C.c_int32),
                ("tile_max", C.c_int32), ("pad_", C.c_int32)]


class ServerCfg(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_resident_runs", C.c_int32),
                ("poll_waves", C.c_int32), ("pad_", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("waves", C.c_int64), ("completed", C.c_int64), ("particle_steps", C.c_int64),
                ("resident", C.c_int32), ("queued", C.c_int32), ("worker_status", C.c_int32),
                ("pad_", C.c_int32)]


_lib = None


def lib():
    """Load libsmc.so (building it first if the sources are newer); with the
    environment variable SMC_LIB_VARIANT=debug, the checking build
    libsmc_debug.so instead (one variant per process)."""
    global _lib
    if _lib is None:
        from . import build as _build

        debug = os.environ.get("SMC_LIB_VARIANT", "") == "debug"
        path = _build.LIB_DEBUG if debug else LIB_PATH
        if not _build.up_to_date(path):
            _build.build(debug=debug)
        if not path.exists():
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(str(path))
        L.smc_model_register.argtypes = [C.POINTER(ModelDesc), C.POINTER(_vp)]
        L.smc_model_register.restype = C.c_int32
        L.smc_model_destroy.argtypes = [_vp]
        L.smc_model_destroy.restype = None
        L.smc_model_info.argtypes = [_vp, _i32p, _i32p, _i32p, _i32p]
        L.smc_model_info.restype = C.c_int32
        L.smc_workspace_bytes.argtypes = [_vp, C.POINTER(RunCfg), C.POINTER(C.c_size_t)]
        L.smc_workspace_bytes.restype = C.c_int32
        L.smc_run.argtypes = [_vp, C.POINTER(RunCfg), C.POINTER(Result), _vp]
        L.smc_run.restype = C.c_int32
        L.smc_run_batch.argtypes = [_vp, _vp, _vp, C.c_int32, _vp]
        L.smc_run_batch.restype = C.c_int32
        L.smc_server_create.argtypes = [C.c_size_t, C.POINTER(ServerCfg), C.POINTER(_vp)]
        L.smc_server_create.restype = C.c_int32
        L.smc_server_submit.argtypes = [_vp, _vp, C.POINTER(RunCfg), C.POINTER(Result),
                                        C.POINTER(C.c_uint64)]
        L.smc_server_submit.restype = C.c_int32
        L.smc_server_poll.argtypes = [_vp, C.c_uint64, C.POINTER(C.c_int32)]
        L.smc_server_poll.restype = C.c_int32
        L.smc_server_wait.argtypes = [_vp, C.c_uint64, C.c_double, C.POINTER(C.c_double)]
        L.smc_server_wait.restype = C.c_int32
        L.smc_server_cancel.argtypes = [_vp, C.c_uint64]
        L.smc_server_cancel.restype = C.c_int32
        L.smc_server_stats.argtypes = [_vp, C.POINTER(ServerStats)]
        L.smc_server_stats.restype = C.c_int32
        L.smc_server_destroy.argtypes = [_vp]
        L.smc_server_destroy.restype = None
        L.smc_resample_workspace_bytes.argtypes = [C.c_int64]
        L.smc_resample_workspace_bytes.restype = C.c_size_t
        L.smc_resample.argtypes = [_vp, C.c_int64, C.c_double, _vp, _vp, _vp, _vp, C.c_size_t, _vp]
        L.smc_resample.restype = C.c_int32
        L.smc_resample_static.argtypes = [_vp, C.c_int64, C.c_double, _vp, _vp, _vp, _vp]
        L.smc_resample_static.restype = C.c_int32
        L.smc_gather.argtypes = [_vp, _vp, _vp, _vp, C.c_int64, C.c_int32, C.c_int32, _vp]
        L.smc_gather.restype = C.c_int32
        L.smc_philox.argtypes = [_vp, _vp, _vp, C.c_int64, _vp]
        L.smc_philox.restype = C.c_int32
        L.smc_sample.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                 C.c_uint32, C.c_int64, _vp, _vp, _vp]
        L.smc_sample.restype = C.c_int32
        L.smc_math_eval.argtypes = [C.c_int32, _vp, _vp, C.c_int64, _vp]
        L.smc_math_eval.restype = C.c_int32
        L.smc_peak_probe_threads.argtypes = []
        L.smc_peak_probe_threads.restype = C.c_int64
        L.smc_peak_probe.argtypes = [C.c_int32, C.c_int64, _vp, _vp]
        L.smc_peak_probe.restype = C.c_int32
        L.smc_shard_records_bytes.argtypes = [C.c_int64]
        L.smc_shard_records_bytes.restype = C.c_size_t
        L.smc_shard_reduce.argtypes = [_vp, C.c_int64, _vp, _vp]
        L.smc_shard_reduce.restype = C.c_int32
        L.smc_shard_workspace_bytes.argtypes = [C.c_int64]
        L.smc_shard_workspace_bytes.restype = C.c_size_t
        L.smc_shard_ancestors.argtypes = [_vp, C.c_int64, C.c_int64, _vp, C.c_int64, C.c_double,
                                          _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]
        L.smc_shard_ancestors.restype = C.c_int32
        L.smc_set_tile_bands.argtypes = [_vp, C.c_int32]
        L.smc_set_tile_bands.restype = C.c_int32
        L.smc_get_tile_bands.argtypes = [_vp, C.c_int32, C.POINTER(C.c_int32)]
        L.smc_get_tile_bands.restype = C.c_int32
        L.smc_tile_size.argtypes = [C.c_int64]
        L.smc_tile_size.restype = C.c_int32
        L.smc_last_error.argtypes = []
        L.smc_last_error.restype = C.c_char_p
        L.smc_version.argtypes = []
        L.smc_version.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st: int) -> int:
    if st < 0:
        raise SmcError(st, lib().smc_last_error().decode())
    return st


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Model:
    """A registered model (owns device copies of its observations / tree)."""

    def __init__(self, kind: str, *, obs=None, tree=None, x0_mean=0.0, x0_sd=1.0, a=0.9, b=0.0,
                 q_sd=1.0, r_sd=0.5, rho=1.0, rates=None, lambda_scale=1.0, mu_scale=0.5,
                 sigma=0.3, fixed_mult=None, depth_cap=MAX_DEPTH, call_limit=1 << 16,
                 lam_stack_cap=0, geo_p=0.5, geo_logw=float(np.log(1.5))):
        d = ModelDesc()
        keep = []
        d.kind = KINDS[kind]
        d.x0_mean, d.x0_sd, d.a, d.b, d.q_sd, d.r_sd = x0_mean, x0_sd, a, b, q_sd, r_sd
        if obs is not None:
            o = np.ascontiguousarray(obs, dtype=np.float64)
            keep.append(o)
            d.obs, d.T = o.ctypes.data_as(_f64p), o.shape[0]
        if tree is not None:
            arr = {k: np.ascontiguousarray(getattr(tree, k), dtype=np.int32)
                   for k in ("parent", "left", "right", "preorder")}
            age = np.ascontiguousarray(tree.age, dtype=np.float64)
            keep += list(arr.values()) + [age]
            d.parent, d.left, d.right, d.preorder = (arr[k].ctypes.data_as(_i32p)
                                                     for k in ("parent", "left", "right", "preorder"))
            d.age, d.n_nodes = age.ctypes.data_as(_f64p), tree.n_nodes
        d.rho = rho
        if rates is not None:
            d.fixed_rates, d.lambda_fixed, d.mu_fixed = 1, rates[0], rates[1]
        d.lambda_scale, d.mu_scale, d.sigma = lambda_scale, mu_scale, sigma
        if fixed_mult is not None:
            fm = np.ascontiguousarray(fixed_mult, dtype=np.float64)
            keep.append(fm)
            d.fixed_mult = fm.ctypes.data_as(_f64p)
        d.depth_cap, d.call_limit, d.lam_stack_cap = depth_cap, call_limit, lam_stack_cap
        d.geo_p, d.geo_logw = geo_p, geo_logw
        h = _vp()
        _check(lib().smc_model_register(C.byref(d), C.byref(h)))
        self.handle = h
        self.kind = kind
        nr, ni, sc, ns = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().smc_model_info(h, C.byref(nr), C.byref(ni), C.byref(sc), C.byref(ns)))
        self.n_real, self.n_int, self.stack_cap, self.n_segments = nr.value, ni.value, sc.value, ns.value

    def close(self):
        if getattr(self, "handle", None):
            lib().smc_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, N: int, precision: str = "fp64", max_segments: int = 0,
                        record_all_ancestors: bool = False) -> int:
        cfg = _cfg(N, 0, 0, precision, max_segments, record_all_ancestors, None)
        out = C.c_size_t()
        _check(lib().smc_workspace_bytes(self.handle, C.byref(cfg), C.byref(out)))
        return out.value


LAUNCH = {"auto": 0, "graph": 1, "one_cta": 2, "cluster": 3, "waves": 4}


def _cfg(N, seed, run_id, precision, max_segments, record_all, workspace, time_kernels=False,
         ess_threshold=0.0, launch="auto"):
    c = RunCfg()
    c.time_kernels = int(time_kernels)
    c.launch_mode = LAUNCH[launch]
    c.ess_threshold = float(ess_threshold)
    c.n_particles, c.seed, c.run_id = N, seed, run_id
    c.precision = PRECISIONS[precision]
    c.max_segments, c.record_all_ancestors = max_segments, int(record_all)
    if workspace is not None:
        c.workspace, c.workspace_bytes = _ptr(workspace), workspace.numel() * workspace.element_size()
    return c


def _alloc_outputs(model: Model, N: int, rows: int, where: str, outputs: dict | None) -> dict:
    shapes = _output_shapes(model, N, rows)
    out = dict(outputs or {})
    if where == "host":
        for k, (shp, dt) in shapes.items():
            if k not in out and _wanted(model, k):
                out[k] = np.zeros(shp, dtype=dt)
    else:
        import torch

        tmap = {"f8": torch.float64, "i4": torch.int32}
        for k, (shp, dt) in shapes.items():
            if k not in out and _wanted(model, k):
                out[k] = torch.zeros(shp, dtype=tmap[dt], device="cuda")
    return out


def _output_shapes(model: Model, N: int, rows: int) -> dict:
    return dict(log_z=((1,), "f8"), final_logw=((N,), "f8"), ancestors=((rows, N), "i4"),
                real_fields=((model.n_real, N), "f8"), int_fields=((model.n_int, N), "i4"),
                stack=((model.stack_cap, N), "f8"), resampled=((rows,), "i4"))


def _wanted(model: Model, key: str) -> bool:
    return (key != "stack" or model.stack_cap) and (key != "real_fields" or model.n_real)


def _rows(model: Model, max_segments: int, record_all: bool) -> int:
    return max(1, (max_segments or model.n_segments or 4096) - 1) if record_all else 1


def _result_struct(out: dict, where: str, rows: int) -> Result:
    r = Result()
    r.where = MEM_HOST if where == "host" else MEM_DEVICE
    r.ancestors_rows = rows
    for k in ("log_z", "final_logw", "ancestors", "real_fields", "int_fields", "stack",
              "resampled"):
        setattr(r, k, _ptr(out.get(k)))
    return r


def _result_dict(st: int, r: Result, out: dict, where: str, record_all: bool) -> dict:
    c = r.counters
    res = dict(status=st, run_status=c.status, n_segments=c.n_segments,
               n_resamples=c.n_resamples, n_near_boundary=c.n_near_boundary,
               n_overflow=c.n_overflow, n_limit=c.n_limit, device_ms=c.device_ms,
               kernel_ms=c.kernel_ms, kernel_launches=c.kernel_launches, n_ess_near=c.n_ess_near,
               n_draws=c.n_draws, n_blocks=c.n_blocks, log_z_closed=c.log_z_closed,
               debug_code=c.debug_code, debug_index=c.debug_index, debug_count=c.debug_count,
               **out)
    res["log_z_value"] = float(out["log_z"][0]) if where == "host" else None
    if record_all:
        n_tr = max(0, c.n_segments - 1)  # checkpoints after which the run went on
        for k in ("ancestors", "resampled"):
            if k in out:
                res[k] = out[k][:n_tr]
    return res


def run(model: Model, N: int, seed: int, run_id: int = 0, precision: str = "fp64",
        max_segments: int = 0, record_all_ancestors: bool = False, where: str = "host",
        stream=None, workspace=None, outputs: dict | None = None,
        time_kernels: bool = False, ess_threshold: float = 0.0,
        launch: str = "auto", launch_graph: bool = False,
        resume_from: dict | None = None) -> dict:
    """smc_run.  where="host": outputs are numpy arrays; where="device": outputs are
    torch CUDA tensors (allocated here unless passed in `outputs`).  ess_threshold
    tau > 0: resample only when ESS < tau N.  launch: "auto" (the library's choice:
    "cluster" where it applies, else "waves"), "waves", "graph" (the waves as one
    captured CUDA graph; needs a stream other than the legacy default stream;
    launch_graph=True says the same), "one_cta" (a small run in one CTA) or
    "cluster" (a small run in one thread-block cluster).
    resume_from: the result of a run of the same model, N, seed, run_id, precision
    and ess_threshold that max_segments stopped (a snapshot); this run continues it."""
    cfg = _cfg(N, seed, run_id, precision, max_segments, record_all_ancestors, workspace,
               time_kernels, ess_threshold, "graph" if launch_graph else launch)
    keep = []
    if resume_from is not None:
        snap = resume_from
        dev = hasattr(snap["final_logw"], "data_ptr")
        if not dev:
            snap = {k: np.ascontiguousarray(snap[k]) if snap.get(k) is not None else None
                    for k in ("final_logw", "real_fields", "int_fields", "stack")}
            keep.append(snap)
        cfg.resume_k = int(resume_from["n_segments"])
        cfg.resume_where = MEM_DEVICE if dev else MEM_HOST
        cfg.resume_logw = _ptr(snap["final_logw"])
        cfg.resume_int = _ptr(snap["int_fields"])
        if model.n_real:
            cfg.resume_real = _ptr(snap["real_fields"])
        if model.stack_cap:
            cfg.resume_stack = _ptr(snap["stack"])
        cfg.resume_log_z = float(resume_from["log_z_closed"])
    rows = _rows(model, max_segments, record_all_ancestors)
    out = _alloc_outputs(model, N, rows, where, outputs)
    r = _result_struct(out, where, rows)
    st = lib().smc_run(model.handle, C.byref(cfg), C.byref(r), _stream(stream))
    if st < 0 and st not in (EDEGENERATE, ESTEPLIMIT):
        _check(st)
    return _result_dict(st, r, out, where, record_all_ancestors)


def run_batch(models: list, specs: list, precision: str = "fp64", where: str = "host",
              record_all_ancestors: bool = False, stream=None, launch_graph: bool = False) -> list:
    """smc_run_batch.  specs[q] = dict(N=..., seed=..., run_id=0, max_segments=0);
    returns one result dict per run (same keys as run())."""
    n = len(models)
    cfgs = (RunCfg * n)()
    ress = (Result * n)()
    outs, rows_l = [], []
    for q, (m, sp) in enumerate(zip(models, specs)):
        c = _cfg(sp["N"], sp["seed"], sp.get("run_id", 0), precision, sp.get("max_segments", 0),
                 record_all_ancestors, None, False, sp.get("ess_threshold", 0.0),
                 "graph" if launch_graph else "waves")
        cfgs[q] = c
        rows = _rows(m, sp.get("max_segments", 0), record_all_ancestors)
        out = _alloc_outputs(m, sp["N"], rows, where, sp.get("outputs"))
        ress[q] = _result_struct(out, where, rows)
        outs.append(out)
        rows_l.append(rows)
    handles = (_vp * n)(*[m.handle for m in models])
    st = lib().smc_run_batch(handles, cfgs, ress, n, _stream(stream))
    _check(st)
    return [_result_dict(ress[q].counters.status, ress[q], outs[q], where, record_all_ancestors)
            for q in range(n)]


class Server:
    """Continuous-batching server (smc_server_*): submit requests from any thread;
    the library's worker admits them into the running waves as memory frees up."""

    def __init__(self, budget_bytes: int, precision: str = "fp64", max_resident_runs: int = 0,
                 poll_waves: int = 0):
        cfg = ServerCfg()
        cfg.precision, cfg.max_resident_runs, cfg.poll_waves = (PRECISIONS[precision],
                                                                max_resident_runs, poll_waves)
        h = _vp()
        _check(lib().smc_server_create(budget_bytes, C.byref(cfg), C.byref(h)))
        self.handle, self.precision = h, precision
        self._live = {}

    def submit(self, model: Model, N: int, seed: int, run_id: int = 0, max_segments: int = 0,
               record_all_ancestors: bool = False, where: str = "host",
               outputs: dict | None = None, ess_threshold: float = 0.0) -> int:
        cfg = _cfg(N, seed, run_id, self.precision, max_segments, record_all_ancestors, None,
                   False, ess_threshold)
        rows = _rows(model, max_segments, record_all_ancestors)
        out = _alloc_outputs(model, N, rows, where, outputs)
        r = _result_struct(out, where, rows)
        t = C.c_uint64()
        _check(lib().smc_server_submit(self.handle, model.handle, C.byref(cfg), C.byref(r),
                                       C.byref(t)))
        self._live[t.value] = (cfg, r, out, where, record_all_ancestors, model)
        return t.value

    def poll(self, ticket: int):
        done = C.c_int32()
        st = lib().smc_server_poll(self.handle, ticket, C.byref(done))
        return bool(done.value), st

    def wait(self, ticket: int, timeout: float = 120.0) -> dict:
        lat = C.c_double()
        st = lib().smc_server_wait(self.handle, ticket, timeout, C.byref(lat))
        if st == ETIMEOUT:
            raise SmcError(st, lib().smc_last_error().decode())
        cfg, r, out, where, rec, _ = self._live.pop(ticket)
        res = _result_dict(st, r, out, where, rec)
        res["latency_s"] = lat.value
        return res

    def cancel(self, ticket: int):
        _check(lib().smc_server_cancel(self.handle, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().smc_server_stats(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_ if k != "pad_"}

    def close(self):
        if getattr(self, "handle", None):
            lib().smc_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def resample_workspace_bytes(N: int) -> int:
    return int(lib().smc_resample_workspace_bytes(N))


def resample(logw, u: float, ancestors=None, out3=None, n_near=None, workspace=None, stream=None):
    """Standalone FP64 systematic resampling of a device population (torch f64 CUDA)."""
    import torch

    N = logw.numel()
    dev = logw.device
    anc = ancestors if ancestors is not None else torch.empty(N, dtype=torch.int32, device=dev)
    o3 = out3 if out3 is not None else torch.empty(3, dtype=torch.float64, device=dev)
    nn = n_near if n_near is not None else torch.empty(1, dtype=torch.int64, device=dev)
    ws = workspace if workspace is not None else torch.empty(
        resample_workspace_bytes(N), dtype=torch.uint8, device=dev)
    _check(lib().smc_resample(_ptr(logw), N, u, _ptr(anc), _ptr(o3), _ptr(nn), _ptr(ws),
                              ws.numel() * ws.element_size(), _stream(stream)))
    return anc, o3, nn


RESAMPLE_STATIC_MAX_N = 1 << 24


def resample_static(logw, u: float, ancestors=None, out3=None, n_near=None, stream=None):
    """smc_resample without a workspace: for callers that cannot allocate device
    memory; scratch is a fixed array inside the library (N <= 2^24, calls on the
    GPU must not overlap)."""
    import torch

    N = logw.numel()
    dev = logw.device
    anc = ancestors if ancestors is not None else torch.empty(N, dtype=torch.int32, device=dev)
    o3 = out3 if out3 is not None else torch.empty(3, dtype=torch.float64, device=dev)
    nn = n_near if n_near is not None else torch.empty(1, dtype=torch.int64, device=dev)
    _check(lib().smc_resample_static(_ptr(logw), N, u, _ptr(anc), _ptr(o3), _ptr(nn),
                                     _stream(stream)))
    return anc, o3, nn


RESAMPLE_TILE = 4096


def shard_reduce(logw, stream=None):
    """smc_shard_reduce: the tiles' records of this rank's slice (a uint8 CUDA
    tensor, 16 bytes a tile)."""
    import torch

    n = logw.numel()
    rec = torch.empty(int(lib().smc_shard_records_bytes(n)), dtype=torch.uint8, device=logw.device)
    _check(lib().smc_shard_reduce(_ptr(logw), n, _ptr(rec), _stream(stream)))
    return rec


def shard_ancestors(logw, first: int, records_all, n_total: int, u: float, ancestors=None,
                    stream=None):
    """smc_shard_ancestors: returns (ancestors [n_total] int32 with [lo, hi) written,
    range int64 [2] = (lo, hi), out3 [3], n_near [1]), CUDA tensors."""
    import torch

    dev = logw.device
    anc = ancestors if ancestors is not None else torch.empty(n_total, dtype=torch.int32, device=dev)
    rng = torch.empty(2, dtype=torch.int64, device=dev)
    o3 = torch.empty(3, dtype=torch.float64, device=dev)
    nn = torch.empty(1, dtype=torch.int64, device=dev)
    ws = torch.empty(int(lib().smc_shard_workspace_bytes(n_total)), dtype=torch.uint8, device=dev)
    _check(lib().smc_shard_ancestors(_ptr(logw), logw.numel(), first, _ptr(records_all), n_total,
                                     u, _ptr(anc), _ptr(rng), _ptr(o3), _ptr(nn), _ptr(ws),
                                     ws.numel(), _stream(stream)))
    return anc, rng, o3, nn


def gather(src, dst, anc, sp=None, stream=None):
    """dst[f][i] = src[f][anc[i]] for 2-D [n_fields, N] device tensors of 4- or 8-byte elements."""
    n_fields, N = src.shape
    _check(lib().smc_gather(_ptr(src), _ptr(dst), _ptr(anc), _ptr(sp), N, n_fields,
                            src.element_size(), _stream(stream)))
    return dst


def gather_row(src, dst, anc, first: int = 0, stream=None):
    """dst[i] = src[anc[i] - first] for 1-D device tensors of 4- or 8-byte
    elements (anc int32 [dst.numel()]; src holds the particles first.. of a
    population indexed from 0)."""
    src_at = _ptr(src) - first * src.element_size()  # the population's element 0
    _check(lib().smc_gather(src_at, _ptr(dst), _ptr(anc), None, dst.numel(), 1,
                            src.element_size(), _stream(stream)))
    return dst


def philox(ctr, key, stream=None):
    """Raw Philox4x32-10 blocks for int32-typed device tensors ctr [n,4], key [n,2]."""
    import torch

    out = torch.empty_like(ctr)
    _check(lib().smc_philox(_ptr(ctr), _ptr(key), _ptr(out), ctr.shape[0], _stream(stream)))
    return out


def sample(dist: str, n: int, p1: float = 0.0, p2: float = 0.0, seed: int = 1, run_id: int = 0,
           precision: str = "fp64", stream=None):
    import torch

    out = torch.empty(n, dtype=torch.float64, device="cuda")
    blocks = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(lib().smc_sample(DIST[dist], PRECISIONS[precision], p1, p2, seed, run_id, n,
                            _ptr(out), _ptr(blocks), _stream(stream)))
    return out, blocks


def math_eval(fn: str, x):
    """Device math parity hook: fn in table_log / table_exp / lib_log / lib_exp, or
    unif_log_bits / unif_log_table with x uint64 random bits (log of the FP64 uniform
    they make, reduced on the integer pipes / through the table log of the double), or
    exp_fix54 / table_exp_fix54: round(e^x 2^54) as int64 for x <= 0 (integer pipes /
    table exponential rounded to that grid), or exp2t_fix54 / exp2t_fix50: round(e^x
    2^54) / round(e^x 2^50) from the two-table integer exponential, or rs_fix50:
    round(e^x 2^50) as smc_resample forms its weights (one table of e^(-j/256) and a
    degree-5 polynomial), or exp_neg_int:
    e^-x (double, 0 <= x < 64) from the same integer exponential, or q_ratio: x an
    [n, 2] array of (S, N) integers, returns [n, 2] uint64 (integer part, fraction
    bits) of floor(S 2^64 / N)."""
    import torch

    code = {"table_log": 0, "table_exp": 1, "lib_log": 2, "lib_exp": 3, "unif_log_bits": 4,
            "unif_log_table": 5, "exp_fix54": 6, "table_exp_fix54": 7, "exp2t_fix54": 8,
            "exp2t_fix50": 9, "exp_neg_int": 10,
            # the FP32 mode's own single-precision functions, and CUDA's for comparison
            "f32_log": 11, "f32_exp": 12, "f32_cos2pi": 13, "f32_log1p": 14, "f32_expm1": 15,
            "f32_lfact": 16, "cuda_logf": 17, "cuda_expf": 18, "cuda_cos2pif": 19,
            "cuda_log1pf": 20, "cuda_expm1f": 21, "q_ratio": 22, "rs_fix50": 23}[fn]
    if code == 22:
        x = np.ascontiguousarray(x, dtype=np.uint64).reshape(-1).view(np.float64)
    if code in (4, 5):
        x = np.ascontiguousarray(x, dtype=np.uint64).view(np.float64)
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    y = torch.empty_like(xd)
    _check(lib().smc_math_eval(code, _ptr(xd), _ptr(y), xd.numel(), None))
    out = y.cpu().numpy()
    if code == 22:
        return out.view(np.uint64).reshape(-1, 2)
    return out.view(np.int64) if 6 <= code <= 9 or code == 23 else out


# the probe's operations: (name, unit, flop per operation or None)
PEAK_KINDS = {0: ("fp64_fma", "TFLOP/s", 2), 1: ("fp32_fma", "TFLOP/s", 2),
              2: ("fp32_ex2_sfu", "T ops/s", None), 3: ("int32_imad", "T ops/s", None),
              4: ("u64_mulhi", "T ops/s", None)}


def peak_probe(kind: int, iters: int, repeats: int = 3) -> float:
    """Operations per second of one arithmetic operation at full occupancy on
    every SM (smc_peak_probe; best of `repeats` launches timed with CUDA
    events after one warm-up launch)."""
    import torch

    L = lib()
    n = int(L.smc_peak_probe_threads())
    if n <= 0:
        raise RuntimeError("no CUDA device for the peak probe")
    sink = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    _check(L.smc_peak_probe(kind, 16, _ptr(sink), _vp(stream.cuda_stream)))
    best = None
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _check(L.smc_peak_probe(kind, iters, _ptr(sink), _vp(stream.cuda_stream)))
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        best = t if best is None else min(best, t)
    return n * 8.0 * iters / best


def set_tile_bands(bands) -> None:
    """Replace the process's tile table: a list of (n_max, slots, tile_min,
    tile_max) with increasing n_max; None restores the built-in table."""
    if bands is None:
        _check(lib().smc_set_tile_bands(None, 0))
        return
    arr = (TileBand * len(bands))()
    for i, (n_max, slots, tmin, tmax) in enumerate(bands):
        arr[i].n_max, arr[i].slots, arr[i].tile_min, arr[i].tile_max = n_max, slots, tmin, tmax
    _check(lib().smc_set_tile_bands(arr, len(bands)))


def get_tile_bands() -> list:
    n = C.c_int32()
    _check(lib().smc_get_tile_bands(None, 0, C.byref(n)))
    arr = (TileBand * max(1, n.value))()
    _check(lib().smc_get_tile_bands(arr, n.value, C.byref(n)))
    return [(b.n_max, b.slots, b.tile_min, b.tile_max) for b in arr[: n.value]]


def tile_size(N: int) -> int:
    """The tile size a run of N particles gets under the current table."""
    return int(lib().smc_tile_size(N))


def version() -> str:
    return lib().smc_version().decode()
