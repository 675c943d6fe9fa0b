"""ctypes binding of libhydro (``include/hydro.h``): argument marshalling only.

Every computation runs in the CUDA kernels of ``csrc/``; this module turns
Python objects (torch tensors, ints, streams) into the plain pointers and
sizes of the C ABI and turns status codes into exceptions.  If the shared
library is missing the import of the functions fails loudly: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

from . import _build

HYDRO_OK = 0
HYDRO_EINVAL = -1
HYDRO_ENOMEM = -2
HYDRO_ECUDA = -3
HYDRO_ENONPHYS = -4
HYDRO_EBUDGET = -5
HYDRO_ETIMEDOUT = -6
HYDRO_EBUSY = -7
HYDRO_ETOOBIG = -8
NOALLOC_MAX_SUBGRIDS = 8192
HYDRO_MAX_FIELDS = 11
HYDRO_MAX_N = 256

FP64 = 0
FP32_FLUX_FP64_ACC = 1
PLAN_AUTOTUNE = 1
PLAN_NO_GRAPH = 2
PLAN_KNP = 4
PLAN_PIPELINED = 8
PLAN_REGISTER_LOADS = 16
PLAN_QUAD26 = 32
F_NO_STATUS = 1
F_KNP = 2
F_REGISTER_LOADS = 4
F_QUAD26 = 8
FOREST_MAX_LEVEL = 15



class HydroError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = "%s: %s (%d)" % (where, strerror(code), code)
        if code == HYDRO_ECUDA:
            msg += " [%s]" % last_cuda_error()
        super().__init__(msg)


class Subgrid(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("dx", ctypes.c_double), ("N", ctypes.c_int32),
                ("n_fields", ctypes.c_int32)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("ghost", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("prec", ctypes.c_int), ("per_task", ctypes.c_int32),
                ("dry_run_ns", ctypes.c_int64), ("flags", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "submitted", "completed", "rejected", "launches", "subgrids_launched",
        "max_subgrids_per_launch", "bytes_in_flight", "peak_bytes_in_flight", "queued")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Leaf(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("bx", ctypes.c_int32), ("by", ctypes.c_int32),
                ("bz", ctypes.c_int32)]


class ForestInfo(ctypes.Structure):
    _fields_ = [("n_leaves", ctypes.c_int32), ("N", ctypes.c_int32), ("n_fields", ctypes.c_int32),
                ("nb0", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("n_level_faces", ctypes.c_int32), ("n_reflux_leaves", ctypes.c_int32),
                ("quad26", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_subgrids", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("interior_cells", ctypes.c_int64), ("out_doubles", ctypes.c_int64),
                ("alg_bytes", ctypes.c_int64), ("threads_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("tuned_ms", ctypes.c_float),
                ("n_candidates", ctypes.c_int32), ("lines_per_chunk", ctypes.c_int32),
                ("prefetch", ctypes.c_int32), ("regs_cap", ctypes.c_int32),
                ("load_batch", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libhydro.  Raises if it is not built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError("libhydro is not built (%s); run __graft_entry__.build()"
                               % _build.LIB)
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    i32, i64, dbl, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
    SG = ctypes.POINTER(Subgrid)
    sig = {
        "hydro_rhs": (ctypes.c_int, [SG, i64, i32, i32, i32, dbl, P, P]),
        "hydro_rhs_ex": (ctypes.c_int, [SG, i64, i32, i32, i32, dbl, P, P, ctypes.c_int, P, u32]),
        "hydro_rhs_per_subgrid": (ctypes.c_int, [SG, i64, i32, dbl, P, P, ctypes.c_int,
                                                 ctypes.POINTER(P), i32]),
        "hydro_rhs_per_subgrid_ex": (ctypes.c_int, [SG, i64, i32, dbl, P, P, ctypes.c_int,
                                                 ctypes.POINTER(P), i32, u32]),
        "hydro_plan_create": (ctypes.c_int, [SG, i64, i32, dbl, ctypes.c_int, u32, P,
                                             ctypes.POINTER(P)]),
        "hydro_plan_execute": (ctypes.c_int, [P, P, P, P]),
        "hydro_plan_info": (ctypes.c_int, [P, ctypes.POINTER(PlanInfo)]),
        "hydro_plan_destroy": (ctypes.c_int, [P]),
        "hydro_status": (ctypes.c_int, [P, ctypes.POINTER(i64)]),
        "hydro_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "hydro_last_cuda_error": (ctypes.c_char_p, []),
        "hydro_output_doubles": (i64, [SG, i64]),
        "hydro_version": (ctypes.c_int, []),
        "hydro_server_create": (ctypes.c_int, [ctypes.POINTER(ServerCfg), ctypes.POINTER(P)]),
        "hydro_server_submit": (ctypes.c_int, [P, SG, i32, P, P, ctypes.POINTER(i64)]),
        "hydro_server_poll": (ctypes.c_int, [P, i64]),
        "hydro_server_wait": (ctypes.c_int, [P, i64, i64]),
        "hydro_server_times": (ctypes.c_int, [P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                              ctypes.POINTER(i64)]),
        "hydro_server_stats": (ctypes.c_int, [P, ctypes.POINTER(ServerStats)]),
        "hydro_server_destroy": (ctypes.c_int, [P]),
        "hydro_now_ns": (i64, []),
        "hydro_rhs_noalloc": (ctypes.c_int, [SG, i64, i32, i32, i32, dbl, P, P, ctypes.c_int, P]),
        "hydro_probe_fp64": (ctypes.c_int, [i32, i32, P, ctypes.POINTER(ctypes.c_double)]),
        "hydro_domain_rhs": (ctypes.c_int, [P, i32, i32, i32, dbl, dbl, P, P, ctypes.c_int, P, u32]),
        "hydro_domain_stage": (ctypes.c_int, [P, P, dbl, dbl, dbl, i32, i32, i32, dbl, dbl, P, P,
                                              ctypes.c_int, P, u32]),
        "hydro_forest_links": (ctypes.c_int, [ctypes.POINTER(Leaf), i32, i32, i32, P, P]),
        "hydro_forest_create": (ctypes.c_int, [ctypes.POINTER(Leaf), i32, i32, i32, i32,
                                               ctypes.POINTER(P)]),
        "hydro_forest_info": (ctypes.c_int, [P, ctypes.POINTER(ForestInfo)]),
        "hydro_forest_rhs": (ctypes.c_int, [P, P, dbl, dbl, P, P, ctypes.c_int, P, u32]),
        "hydro_forest_stage": (ctypes.c_int, [P, P, P, dbl, dbl, dbl, dbl, dbl, P, P, ctypes.c_int,
                                              P, u32]),
        "hydro_forest_destroy": (ctypes.c_int, [P]),
        "hydro_forest_stage_dt": (ctypes.c_int, [P, P, P, dbl, dbl, P, dbl, dbl, P, P, ctypes.c_int, P,
                                                 u32]),
        "hydro_domain_stage_dt": (ctypes.c_int, [P, P, dbl, dbl, P, i32, i32, i32, dbl, dbl, P, P,
                                                 ctypes.c_int, P, u32]),
        "hydro_courant": (ctypes.c_int, [P, i32, i64, i64, P, dbl, dbl, dbl, P, P, i64, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().hydro_strerror(int(code)).decode()


def last_cuda_error() -> str:
    return load().hydro_last_cuda_error().decode()


def _check(rc, where):
    if rc != HYDRO_OK:
        raise HydroError(rc, where)


def _ptr(x) -> int:
    """Address of a buffer: a torch tensor of binary64 values stored densely
    (the C ABI reads and writes plain arrays), or an int address."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if str(x.dtype) != "torch.float64":
        raise TypeError("libhydro buffers hold binary64 values, not %s" % x.dtype)
    if not x.is_contiguous():
        raise ValueError("libhydro reads and writes dense arrays: pass a contiguous tensor "
                         "(or the whole buffer, with its stride where the call takes one)")
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def descriptors(items: Sequence) -> ctypes.Array:
    """Descriptor array from (U, dx, N, n_fields) tuples; U a device tensor or address."""
    arr = (Subgrid * max(len(items), 1))()
    for i, (U, dx, N, F) in enumerate(items):
        arr[i].U = _ptr(U)
        arr[i].dx = float(dx)
        arr[i].N = int(N)
        arr[i].n_fields = int(F)
    return arr


def output_doubles(desc, n=None) -> int:
    n = len(desc) if n is None else n
    r = load().hydro_output_doubles(desc, n)
    if r < 0:
        raise HydroError(HYDRO_EINVAL, "hydro_output_doubles")
    return int(r)


def rhs(desc, out, amax, ghost=3, gamma=5.0 / 3.0, N=0, n_fields=0, prec=FP64, stream=None,
        flags=0, n=None):
    """One aggregated RHS (hydro_rhs_ex): ``desc`` from ``descriptors``."""
    n = len(desc) if n is None else n
    _check(load().hydro_rhs_ex(desc, n, N, ghost, n_fields, float(gamma), _ptr(out), _ptr(amax),
                               int(prec), _stream(stream), int(flags)), "hydro_rhs_ex")


def rhs_noalloc(desc, out, amax, N, n_fields, ghost=3, gamma=5.0 / 3.0, prec=FP64, stream=None,
                n=None):
    """hydro_rhs_noalloc: a uniform batch evaluated without any allocation (its
    descriptors go to a fixed device array of the library)."""
    n = len(desc) if n is None else n
    _check(load().hydro_rhs_noalloc(desc, n, int(N), ghost, int(n_fields), float(gamma), _ptr(out),
                                    _ptr(amax), int(prec), _stream(stream)), "hydro_rhs_noalloc")


def probe_fp64(blocks_per_sm=4, iters=10000, stream=None):
    """hydro_probe_fp64: enqueue the binary64 fused multiply-add probe on
    `stream`; returns the number of fused multiply-adds it runs."""
    n = ctypes.c_double(0.0)
    _check(load().hydro_probe_fp64(int(blocks_per_sm), int(iters), _stream(stream), ctypes.byref(n)),
           "hydro_probe_fp64")
    return n.value


def domain_rhs(U, nb, N, n_fields, dx, out, amax, gamma=5.0 / 3.0, prec=FP64, stream=None,
               flags=0):
    """hydro_domain_rhs: periodic domain stored without ghosts ([s][f][N^3])."""
    _check(load().hydro_domain_rhs(_ptr(U), int(nb), int(N), int(n_fields), float(dx),
                                   float(gamma), _ptr(out), _ptr(amax), int(prec),
                                   _stream(stream), int(flags)), "hydro_domain_rhs")


def domain_stage(U, U0, alpha, beta, dt, nb, N, n_fields, dx, U_out, amax, gamma=5.0 / 3.0,
                 prec=FP64, stream=None, flags=0):
    """hydro_domain_stage: U_out = alpha U0 + beta (U + dt dU/dt(U)) in one launch."""
    _check(load().hydro_domain_stage(_ptr(U), _ptr(U0), float(alpha), float(beta), float(dt),
                                     int(nb), int(N), int(n_fields), float(dx), float(gamma),
                                     _ptr(U_out), _ptr(amax), int(prec), _stream(stream),
                                     int(flags)), "hydro_domain_stage")


def _leaves(leaves):
    """(level, bx, by, bz) rows -> a ctypes array of hydro_leaf_t."""
    rows = [tuple(int(v) for v in r) for r in leaves]
    return (Leaf * max(len(rows), 1))(*[Leaf(*r) for r in rows]), len(rows)


def forest_links(leaves, nb0, N):
    """hydro_forest_links (host only): (kind, nbr) as lists of 6 per leaf;
    kind -1 coarser, 0 same level, +1 finer."""
    arr, n = _leaves(leaves)
    kind = (ctypes.c_int32 * (6 * max(n, 1)))()
    nbr = (ctypes.c_int32 * (6 * max(n, 1)))()
    _check(load().hydro_forest_links(arr, n, int(nb0), int(N), ctypes.addressof(kind),
                                     ctypes.addressof(nbr)), "hydro_forest_links")
    return ([list(kind[6 * s:6 * s + 6]) for s in range(n)],
            [list(nbr[6 * s:6 * s + 6]) for s in range(n)])


class Forest:
    """hydro_forest_*: a multi-level forest of N^3 leaves (ghost slabs across
    levels and the flux correction on the device)."""

    def __init__(self, leaves, nb0, N, n_fields):
        arr, n = _leaves(leaves)
        h = ctypes.c_void_p()
        _check(load().hydro_forest_create(arr, n, int(nb0), int(N), int(n_fields), ctypes.byref(h)),
               "hydro_forest_create")
        self._h = h

    def rhs(self, U, dx0, out, amax, gamma=5.0 / 3.0, prec=FP64, stream=None, flags=0):
        _check(load().hydro_forest_rhs(self._h, _ptr(U), float(dx0), float(gamma), _ptr(out),
                                       _ptr(amax), int(prec), _stream(stream), int(flags)),
               "hydro_forest_rhs")

    def stage(self, U, U0, alpha, beta, dt, dx0, U_out, amax, gamma=5.0 / 3.0, prec=FP64,
              stream=None, flags=0):
        _check(load().hydro_forest_stage(self._h, _ptr(U), _ptr(U0), float(alpha), float(beta),
                                         float(dt), float(dx0), float(gamma), _ptr(U_out),
                                         _ptr(amax), int(prec), _stream(stream), int(flags)),
               "hydro_forest_stage")

    def stage_dt(self, U, U0, alpha, beta, dt_dev, dx0, U_out, amax, gamma=5.0 / 3.0, prec=FP64,
                 stream=None, flags=0):
        _check(load().hydro_forest_stage_dt(self._h, _ptr(U), _ptr(U0), float(alpha), float(beta),
                                            _ptr(dt_dev), float(dx0), float(gamma), _ptr(U_out),
                                            _ptr(amax), int(prec), _stream(stream), int(flags)),
               "hydro_forest_stage_dt")

    def info(self) -> dict:
        fi = ForestInfo()
        _check(load().hydro_forest_info(self._h, ctypes.byref(fi)), "hydro_forest_info")
        return fi.as_dict()

    def close(self):
        if self._h is not None and self._h.value:
            load().hydro_forest_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def domain_stage_dt(U, U0, alpha, beta, dt_dev, nb, N, n_fields, dx, U_out, amax, gamma=5.0 / 3.0,
                    prec=FP64, stream=None, flags=0):
    """hydro_domain_stage_dt: the stage with dt read from device memory (dt_dev)."""
    _check(load().hydro_domain_stage_dt(_ptr(U), _ptr(U0), float(alpha), float(beta), _ptr(dt_dev),
                                        int(nb), int(N), int(n_fields), float(dx), float(gamma),
                                        _ptr(U_out), _ptr(amax), int(prec), _stream(stream),
                                        int(flags)), "hydro_domain_stage_dt")


def courant(amax, n_rows, row_stride, n, clock, cfl, t_end, dx=None, dx_uniform=0.0, dt_hist=None,
            hist_len=0, stream=None):
    """hydro_courant: dt from the largest signal speeds, on the device."""
    _check(load().hydro_courant(_ptr(amax), int(n_rows), int(row_stride), int(n),
                                _ptr(dx) if dx is not None else None, float(dx_uniform), float(cfl),
                                float(t_end), _ptr(clock), _ptr(dt_hist) if dt_hist is not None else None,
                                int(hist_len), _stream(stream)), "hydro_courant")


def rhs_per_subgrid(desc, out, amax, streams: Iterable, ghost=3, gamma=5.0 / 3.0, prec=FP64,
                    n=None, flags=0):
    """The per-sub-grid launch form (hydro_rhs_per_subgrid_ex) over a stream pool."""
    n = len(desc) if n is None else n
    st = [_stream(s) for s in streams]
    arr = (ctypes.c_void_p * len(st))(*st)
    _check(load().hydro_rhs_per_subgrid_ex(desc, n, ghost, float(gamma), _ptr(out), _ptr(amax),
                                           int(prec), arr, len(st), int(flags)), "hydro_rhs_per_subgrid_ex")


def status(stream=None):
    """(status code, first bad sub-grid or -1); synchronises the stream."""
    fb = ctypes.c_int64(-1)
    rc = load().hydro_status(_stream(stream), ctypes.byref(fb))
    if rc not in (HYDRO_OK, HYDRO_ENONPHYS):
        raise HydroError(rc, "hydro_status")
    return rc, int(fb.value)


class Plan:
    """hydro_plan_*: fixed batch, tuned launch shape, CUDA-graph replay."""

    def __init__(self, desc, ghost=3, gamma=5.0 / 3.0, prec=FP64, autotune=False, graph=True,
                 stream=None, n=None, knp=False, flags=0):
        n = len(desc) if n is None else n
        self._desc = desc  # keep the pointers' owner alive
        h = ctypes.c_void_p()
        flags = (int(flags) | (PLAN_AUTOTUNE if autotune else 0) | (0 if graph else PLAN_NO_GRAPH)
                 | (PLAN_KNP if knp else 0))
        _check(load().hydro_plan_create(desc, n, ghost, float(gamma), int(prec), flags,
                                        _stream(stream), ctypes.byref(h)), "hydro_plan_create")
        self._h = h

    def execute(self, out, amax, stream=None):
        _check(load().hydro_plan_execute(self._h, _ptr(out), _ptr(amax), _stream(stream)),
               "hydro_plan_execute")

    def info(self) -> dict:
        pi = PlanInfo()
        _check(load().hydro_plan_info(self._h, ctypes.byref(pi)), "hydro_plan_info")
        return pi.as_dict()

    def close(self):
        if self._h is not None and self._h.value:
            load().hydro_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """hydro_server_*: continuous batching of sub-grid tasks (see include/hydro.h)."""

    def __init__(self, budget_bytes=40 << 30, max_batch=4096, n_streams=4, ghost=3,
                 queue_capacity=1 << 20, gamma=5.0 / 3.0, prec=FP64, per_task=False,
                 dry_run_ns=0, knp=False, flags=0):
        cfg = ServerCfg(int(budget_bytes), int(max_batch), int(n_streams), int(ghost),
                        int(queue_capacity), float(gamma), int(prec), 1 if per_task else 0,
                        int(dry_run_ns), int(flags) | (F_KNP if knp else 0))
        h = ctypes.c_void_p()
        _check(load().hydro_server_create(ctypes.byref(cfg), ctypes.byref(h)), "hydro_server_create")
        self._h = h

    def submit(self, desc, out, amax, n=None):
        """Returns (status, ticket); status is HYDRO_OK, HYDRO_EBUDGET or HYDRO_EBUSY."""
        n = len(desc) if n is None else n
        t = ctypes.c_int64(0)
        rc = load().hydro_server_submit(self._h, desc, n, _ptr(out), _ptr(amax), ctypes.byref(t))
        if rc not in (HYDRO_OK, HYDRO_EBUDGET, HYDRO_EBUSY):
            raise HydroError(rc, "hydro_server_submit")
        return rc, int(t.value)

    def poll(self, ticket):
        return load().hydro_server_poll(self._h, int(ticket))

    def wait(self, ticket, timeout_ns=-1):
        return load().hydro_server_wait(self._h, int(ticket), int(timeout_ns))

    def times(self, ticket):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().hydro_server_times(self._h, int(ticket), ctypes.byref(a), ctypes.byref(b),
                                         ctypes.byref(c)), "hydro_server_times")
        return a.value, b.value, c.value

    def stats(self):
        st = ServerStats()
        _check(load().hydro_server_stats(self._h, ctypes.byref(st)), "hydro_server_stats")
        return st.as_dict()

    def close(self):
        if self._h is not None and self._h.value:
            load().hydro_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def now_ns() -> int:
    return int(load().hydro_now_ns())
