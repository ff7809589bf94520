"""Thin Python binding of the ttc C ABI (include/ttc.h).

Argument marshalling only: every step of the computation runs in the CUDA
library libttc.so.  Importing this module never falls back to a CPU path: if
the library is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttc.so")

PREC_FP64, PREC_MIXED, PREC_FP32 = 0, 1, 2
STOP_RELERR, STOP_STEP, STOP_NONE, STOP_RESID = 0, 1, 2, 3
STEP_CONSTANT, STEP_STEEPEST = 0, 1
METRIC_PRECOND, METRIC_UNIFORM = 0, 1
RETRACT_PLAIN, RETRACT_WEIGHTED = 0, 1
DENSE_AUTO, DENSE_FP64, DENSE_FF = 0, 1, 2

STATUS = {
    0: "TTC_OK", -1: "TTC_EINVAL", -2: "TTC_ENOMEM", -3: "TTC_ERANGE", -4: "TTC_EDUP",
    -5: "TTC_ENONFINITE", -6: "TTC_ENOTCONV", -7: "TTC_ETIMEOUT", -8: "TTC_ECUDA", -9: "TTC_EBUSY",
    -10: "TTC_EUNSUPPORTED",
}


class TTCError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("eps_rel", C.c_double), ("alpha_scale", C.c_double),
        ("eps_frozen", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("stop_rule", C.c_int),
        ("check_every", C.c_int), ("polish_below", C.c_double), ("use_graph", C.c_int),
        ("step_rule", C.c_int), ("metric", C.c_int), ("retraction", C.c_int), ("polish_factor", C.c_double),
        ("step_fallback", C.c_int), ("dense_mode", C.c_int),
    ]


class StepInfo(C.Structure):
    _fields_ = [("eps", C.c_double), ("alpha", C.c_double), ("res_norm", C.c_double), ("precision_used", C.c_int),
                ("subspace_iters", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("last_metric", C.c_double),
                ("res_norm", C.c_double), ("polish_iter", C.c_int), ("fallback_iter", C.c_int)]


class Request(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("n", C.POINTER(C.c_int64)), ("r", C.POINTER(C.c_int32)), ("N", C.c_int64),
        ("idx", C.POINTER(C.c_int32)), ("y", C.POINTER(C.c_double)),
        ("init", C.POINTER(C.POINTER(C.c_double))), ("truth_r", C.POINTER(C.c_int32)),
        ("truth", C.POINTER(C.POINTER(C.c_double))), ("opt", C.POINTER(Options)),
    ]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("converged", C.c_int), ("last_metric", C.c_double),
                ("res_norm", C.c_double), ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("detail", C.c_char * 128)]


class ServingStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int64),
                ("iterations", C.c_int64), ("launches", C.c_int64), ("entry_iterations", C.c_double),
                ("busy_ms", C.c_double), ("wall_ms", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("rebuilds", C.c_int64),
                ("rebuild_ms", C.c_double), ("admit_ms", C.c_double)]


_lib = None

EXPORTS = [
    "ttc_default_options", "ttc_create", "ttc_set_observations", "ttc_set_cores", "ttc_get_cores",
    "ttc_set_truth", "ttc_step", "ttc_solve", "ttc_relerr", "ttc_eval", "ttc_get_residual",
    "ttc_get_slice_energy", "ttc_get_scatter", "ttc_get_layout", "ttc_profile_enable", "ttc_profile_read",
    "ttc_device_bytes", "ttc_destroy", "ttc_strerror", "ttc_last_cuda_error", "ttc_launch_count",
    "ttc_tt_dist2_static", "ttc_batch_create", "ttc_batch_step", "ttc_batch_sync", "ttc_batch_set_lanes",
    "ttc_batch_join", "ttc_batch_profile_enable",
    "ttc_batch_profile_read", "ttc_batch_profile_read_dense", "ttc_batch_launch_count", "ttc_batch_destroy",
    "ttc_server_create", "ttc_submit", "ttc_poll", "ttc_server_stats", "ttc_server_destroy",
]


def lib():
    """Load libttc.so (built by paper_2501_13385_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: call __graft_entry__.build() or "
                           "paper_2501_13385_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    vp, i32p, i64p, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    dpp = C.POINTER(dp)
    sig = {
        "ttc_default_options": (None, [C.POINTER(Options)]),
        "ttc_create": (C.c_int, [C.POINTER(vp), C.c_int, i64p, i32p, C.POINTER(Options), vp]),
        "ttc_set_observations": (C.c_int, [vp, C.c_int64, i32p, dp]),
        "ttc_set_cores": (C.c_int, [vp, dpp]),
        "ttc_get_cores": (C.c_int, [vp, dpp]),
        "ttc_set_truth": (C.c_int, [vp, i32p, dpp]),
        "ttc_step": (C.c_int, [vp, C.c_double, C.POINTER(StepInfo)]),
        "ttc_solve": (C.c_int, [vp, C.POINTER(SolveInfo)]),
        "ttc_relerr": (C.c_int, [vp, dp]),
        "ttc_eval": (C.c_int, [vp, C.c_int64, i32p, C.c_int, dp]),
        "ttc_get_residual": (C.c_int, [vp, dp]),
        "ttc_get_slice_energy": (C.c_int, [vp, C.c_int, dp]),
        "ttc_get_scatter": (C.c_int, [vp, C.c_int, dp]),
        "ttc_get_layout": (C.c_int, [vp, C.c_int, i32p, i64p]),
        "ttc_profile_enable": (C.c_int, [vp, C.c_int]),
        "ttc_profile_read": (C.c_int, [vp, dp, i64p, C.c_int]),
        "ttc_device_bytes": (C.c_int, [vp, i64p]),
        "ttc_launch_count": (C.c_int, [vp, i64p]),
        "ttc_tt_dist2_static": (C.c_int, [C.c_int, i64p, i32p, C.POINTER(vp), i32p, C.POINTER(vp), vp, vp]),
        "ttc_destroy": (None, [vp]),
        "ttc_batch_create": (C.c_int, [C.POINTER(vp), C.POINTER(vp), C.c_int, vp]),
        "ttc_batch_step": (C.c_int, [vp]),
        "ttc_batch_set_lanes": (C.c_int, [vp, C.c_int]),
        "ttc_batch_join": (C.c_int, [vp]),
        "ttc_batch_sync": (C.c_int, [vp]),
        "ttc_batch_profile_enable": (C.c_int, [vp, C.c_int]),
        "ttc_batch_profile_read": (C.c_int, [vp, dp, i64p, C.c_int]),
        "ttc_batch_profile_read_dense": (C.c_int, [vp, dp, i64p, C.c_int]),
        "ttc_batch_launch_count": (C.c_int, [vp, i64p]),
        "ttc_batch_destroy": (None, [vp]),
        "ttc_server_create": (C.c_int, [C.POINTER(vp), C.c_size_t, C.c_int, vp]),
        "ttc_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "ttc_poll": (C.c_int, [vp, C.c_uint64, C.c_int64, C.POINTER(Result), dpp]),
        "ttc_server_stats": (C.c_int, [vp, C.POINTER(ServingStats)]),
        "ttc_server_destroy": (None, [vp]),
        "ttc_strerror": (C.c_char_p, [C.c_int]),
        "ttc_last_cuda_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != 0:
        detail = ""
        if status == -8:
            detail = lib().ttc_last_cuda_error().decode()
        raise TTCError(status, where, detail)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def default_options(**kw) -> Options:
    o = Options()
    lib().ttc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """One completion problem on the GPU (ttc_ctx)."""

    def __init__(self, n: Sequence[int], r: Sequence[int], options: Optional[Options] = None,
                 stream: Optional[int] = None, **kw):
        L = lib()
        self.n = [int(x) for x in n]
        self.r = [int(x) for x in r]
        self.m = len(self.n)
        opt = options if options is not None else default_options(**kw)
        self._h = C.c_void_p()
        na = np.asarray(self.n, dtype=np.int64)
        ra = np.asarray(self.r, dtype=np.int32)
        _check(L.ttc_create(C.byref(self._h), self.m, na.ctypes.data_as(C.POINTER(C.c_int64)),
                            ra.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(opt),
                            C.c_void_p(stream) if stream else None), "ttc_create")
        self.N = 0

    # -- lifetime
    def close(self):
        if self._h:
            lib().ttc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- data in / out
    def set_observations(self, idx, y):
        idx, ip = _i32(idx)
        y, yp = _f64(y)
        if idx.ndim != 2 or idx.shape[1] != self.m or y.shape[0] != idx.shape[0]:
            raise ValueError("idx must be (N, d) and y (N,)")
        _check(lib().ttc_set_observations(self._h, idx.shape[0], ip, yp), "ttc_set_observations")
        self.N = idx.shape[0]

    def _core_ptrs(self, cores, ranks):
        arrs = []
        for k in range(self.m):
            c = np.ascontiguousarray(cores[k], dtype=np.float64)
            if c.shape != (ranks[k], self.n[k], ranks[k + 1]):
                raise ValueError(f"core {k} has shape {c.shape}, expected {(ranks[k], self.n[k], ranks[k + 1])}")
            arrs.append(c)
        ptrs = (C.POINTER(C.c_double) * self.m)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
        return arrs, ptrs

    def set_cores(self, cores):
        arrs, ptrs = self._core_ptrs(cores, self.r)
        _check(lib().ttc_set_cores(self._h, ptrs), "ttc_set_cores")

    def get_cores(self) -> List[np.ndarray]:
        arrs = [np.empty((self.r[k], self.n[k], self.r[k + 1])) for k in range(self.m)]
        ptrs = (C.POINTER(C.c_double) * self.m)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
        _check(lib().ttc_get_cores(self._h, ptrs), "ttc_get_cores")
        return arrs

    def set_truth(self, cores):
        rt = [1] + [int(c.shape[2]) for c in cores[:-1]] + [1]
        arrs, ptrs = self._core_ptrs(cores, rt)
        ra = np.asarray(rt, dtype=np.int32)
        _check(lib().ttc_set_truth(self._h, ra.ctypes.data_as(C.POINTER(C.c_int32)), ptrs), "ttc_set_truth")

    # -- iteration
    def step_async(self, alpha: float = 0.0):
        """Enqueue one iteration on the context's stream without waiting."""
        _check(lib().ttc_step(self._h, float(alpha), None), "ttc_step")

    def step(self, alpha: float = 0.0) -> dict:
        info = StepInfo()
        _check(lib().ttc_step(self._h, float(alpha), C.byref(info)), "ttc_step")
        return {"eps": info.eps, "alpha": info.alpha, "res_norm": info.res_norm,
                "precision_used": info.precision_used, "subspace_iters": info.subspace_iters}

    def solve(self, raise_on_notconv: bool = False) -> dict:
        info = SolveInfo()
        st = lib().ttc_solve(self._h, C.byref(info))
        if st not in (0, -6) or (raise_on_notconv and st == -6):
            _check(st, "ttc_solve")
        return {"status": STATUS.get(st, st), "iters": info.iters, "converged": bool(info.converged),
                "last_metric": info.last_metric, "res_norm": info.res_norm, "polish_iter": info.polish_iter,
                "fallback_iter": info.fallback_iter}

    def relerr(self) -> float:
        v = C.c_double()
        _check(lib().ttc_relerr(self._h, C.byref(v)), "ttc_relerr")
        return v.value

    def eval(self, idx, precision: int = PREC_FP64) -> np.ndarray:
        idx, ip = _i32(idx)
        out = np.empty(idx.shape[0])
        _check(lib().ttc_eval(self._h, idx.shape[0], ip, precision, out.ctypes.data_as(C.POINTER(C.c_double))),
               "ttc_eval")
        return out

    # -- intermediate results of the last step
    def residual(self) -> np.ndarray:
        out = np.empty(self.N)
        _check(lib().ttc_get_residual(self._h, out.ctypes.data_as(C.POINTER(C.c_double))), "ttc_get_residual")
        return out

    def slice_energy(self, k: int) -> np.ndarray:
        out = np.empty(self.n[k])
        _check(lib().ttc_get_slice_energy(self._h, k, out.ctypes.data_as(C.POINTER(C.c_double))),
               "ttc_get_slice_energy")
        return out

    def scatter(self, k: int) -> np.ndarray:
        """E_k as (n_k, r_{k-1}, r_k)."""
        out = np.empty((self.n[k], self.r[k], self.r[k + 1]))
        _check(lib().ttc_get_scatter(self._h, k, out.ctypes.data_as(C.POINTER(C.c_double))), "ttc_get_scatter")
        return out

    def layout(self, k: int):
        perm = np.empty(self.N, dtype=np.int32)
        seg = np.empty(self.n[k] + 1, dtype=np.int64)
        _check(lib().ttc_get_layout(self._h, k, perm.ctypes.data_as(C.POINTER(C.c_int32)),
                                    seg.ctypes.data_as(C.POINTER(C.c_int64))), "ttc_get_layout")
        return perm, seg

    # -- profiling
    def profile_enable(self, on: bool = True):
        _check(lib().ttc_profile_enable(self._h, 1 if on else 0), "ttc_profile_enable")

    def profile_read(self, reset: bool = False):
        ms = C.c_double()
        cnt = C.c_int64()
        _check(lib().ttc_profile_read(self._h, C.byref(ms), C.byref(cnt), 1 if reset else 0), "ttc_profile_read")
        return ms.value, cnt.value

    def launch_count(self) -> int:
        v = C.c_int64()
        _check(lib().ttc_launch_count(self._h, C.byref(v)), "ttc_launch_count")
        return v.value

    def device_bytes(self) -> int:
        v = C.c_int64()
        _check(lib().ttc_device_bytes(self._h, C.byref(v)), "ttc_device_bytes")
        return v.value


class Batch:
    """Several contexts stepped together by one CUDA graph launch per iteration
    (ttc_batch_*).  Holds references to its members; close it before them."""

    def __init__(self, members: Sequence[Context], stream: Optional[int] = None, lanes: int = 1):
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        self._h = C.c_void_p()
        _check(lib().ttc_batch_create(C.byref(self._h), arr, len(self.members),
                                      C.c_void_p(stream) if stream else None), "ttc_batch_create")
        if lanes != 1:
            _check(lib().ttc_batch_set_lanes(self._h, int(lanes)), "ttc_batch_set_lanes")

    def step(self):
        _check(lib().ttc_batch_step(self._h), "ttc_batch_step")

    def sync(self):
        _check(lib().ttc_batch_sync(self._h), "ttc_batch_sync")

    def join(self):
        """Make the batch's stream wait for the lanes' work (no host wait)."""
        _check(lib().ttc_batch_join(self._h), "ttc_batch_join")

    def profile_enable(self, on: bool = True):
        _check(lib().ttc_batch_profile_enable(self._h, 1 if on else 0), "ttc_batch_profile_enable")

    def profile_read(self, reset: bool = False):
        ms = C.c_double()
        cnt = C.c_int64()
        _check(lib().ttc_batch_profile_read(self._h, C.byref(ms), C.byref(cnt), 1 if reset else 0),
               "ttc_batch_profile_read")
        return ms.value, cnt.value

    def profile_read_dense(self, reset: bool = False):
        """(ms, steps) of the dense part of the profiled steps (end of the pass to the join of all members)."""
        ms = C.c_double()
        cnt = C.c_int64()
        _check(lib().ttc_batch_profile_read_dense(self._h, C.byref(ms), C.byref(cnt), 1 if reset else 0),
               "ttc_batch_profile_read_dense")
        return ms.value, cnt.value

    def launch_count(self) -> int:
        v = C.c_int64()
        _check(lib().ttc_batch_launch_count(self._h, C.byref(v)), "ttc_batch_launch_count")
        return v.value

    def close(self):
        if self._h:
            lib().ttc_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching solver service (ttc_server_*): submit requests,
    poll for their results.  The engine thread runs inside the library."""

    def __init__(self, budget_bytes: int = 0, max_slots: int = 64, stream: Optional[int] = None):
        self._h = C.c_void_p()
        self._shapes = {}
        _check(lib().ttc_server_create(C.byref(self._h), int(budget_bytes), int(max_slots),
                                       C.c_void_p(stream) if stream else None), "ttc_server_create")

    def submit(self, n, r, idx, y, init, truth=None, options: Optional[Options] = None) -> int:
        m = len(n)
        na = np.ascontiguousarray(n, dtype=np.int64)
        ra = np.ascontiguousarray(r, dtype=np.int32)
        idx, ip = _i32(idx)
        y, yp = _f64(y)
        if idx.ndim != 2 or idx.shape[1] != m or y.shape[0] != idx.shape[0]:
            raise ValueError("idx must be (N, d) and y (N,)")
        keep = [na, ra, idx, y]
        dptr = C.POINTER(C.c_double)
        cores = [np.ascontiguousarray(c, dtype=np.float64) for c in init]
        for k, c in enumerate(cores):
            if c.shape != (r[k], n[k], r[k + 1]):
                raise ValueError(f"core {k} has shape {c.shape}")
        init_p = (dptr * m)(*[c.ctypes.data_as(dptr) for c in cores])
        keep += cores
        req = Request(d=m, n=na.ctypes.data_as(C.POINTER(C.c_int64)), r=ra.ctypes.data_as(C.POINTER(C.c_int32)),
                      N=idx.shape[0], idx=ip, y=yp, init=init_p)
        if truth is not None:
            rt = np.asarray([1] + [int(c.shape[2]) for c in truth[:-1]] + [1], dtype=np.int32)
            tc = [np.ascontiguousarray(c, dtype=np.float64) for c in truth]
            keep += [rt] + tc
            req.truth_r = rt.ctypes.data_as(C.POINTER(C.c_int32))
            req.truth = (dptr * m)(*[c.ctypes.data_as(dptr) for c in tc])
        if options is not None:
            req.opt = C.pointer(options)
        t = C.c_uint64()
        _check(lib().ttc_submit(self._h, C.byref(req), C.byref(t)), "ttc_submit")
        self._shapes[t.value] = (list(n), list(r))
        del keep
        return t.value

    def poll(self, ticket: int, timeout_s: Optional[float] = None, cores: bool = True):
        """Result dict (with the final cores), or None if not finished within
        timeout_s (None: wait without limit)."""
        n, r = self._shapes.get(ticket, (None, None))
        cores = cores and n is not None
        res = Result()
        arrs = [np.empty((r[k], n[k], r[k + 1])) for k in range(len(n))] if cores else None
        dptr = C.POINTER(C.c_double)
        ptrs = (dptr * len(n))(*[a.ctypes.data_as(dptr) for a in arrs]) if cores else None
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        st = lib().ttc_poll(self._h, ticket, us, C.byref(res), ptrs)
        if st == -7:
            return None
        _check(st, "ttc_poll")
        self._shapes.pop(ticket, None)
        out = {"status": STATUS.get(res.status, res.status), "iters": res.iters, "converged": bool(res.converged),
               "last_metric": res.last_metric, "res_norm": res.res_norm, "latency_ms": res.latency_ms,
               "queue_ms": res.queue_ms, "detail": res.detail.decode(errors="replace")}
        if cores and res.status in (0, -6):
            out["cores"] = arrs
        return out

    def stats(self) -> dict:
        v = ServingStats()
        _check(lib().ttc_server_stats(self._h, C.byref(v)), "ttc_server_stats")
        return {f: getattr(v, f) for f, _ in ServingStats._fields_}

    def close(self):
        if self._h:
            lib().ttc_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
