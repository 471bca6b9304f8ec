"""GB300 interval branch-and-bound global minimiser: thin Python binding.

The compute path is the CUDA library ``_build/libgb.so`` (C ABI declared in
include/gb.h).  This module only marshals arguments through ctypes; every
step of the method runs in the library's kernels.  There is no CPU fallback:
if the library is missing or cannot be loaded the import of the binding's
functions raises.

Device buffers for the per-box hook are PyTorch CUDA tensors (PyTorch is used
for device memory and streams only).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

GB_OK, GB_E_INVALID, GB_E_OOM, GB_E_CAPACITY, GB_E_LIMIT, GB_E_TIMEOUT, GB_E_CUDA, GB_E_BUSY = range(8)


class GbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{gb_status_str(status)}: {msg}")
        self.status = status


class gb_options(ctypes.Structure):
    _fields_ = [("tol_f", ctypes.c_double), ("tol_x", ctypes.c_double),
                ("block", ctypes.c_int32), ("split_m", ctypes.c_int32),
                ("split_d", ctypes.c_int32), ("fp32_prefilter", ctypes.c_int32),
                ("max_generations", ctypes.c_int64), ("max_children", ctypes.c_int64),
                ("max_boxes", ctypes.c_int64), ("pool_bytes", ctypes.c_size_t),
                ("device", ctypes.c_int32), ("eval_mode", ctypes.c_int32),
                ("gens_per_sync", ctypes.c_int32), ("pool_mode", ctypes.c_int32),
                ("samples", ctypes.c_int32), ("max_records", ctypes.c_int64),
                ("mono_all", ctypes.c_int32), ("pad", ctypes.c_int32)]


class gb_gen_stat(ctypes.Structure):
    _fields_ = [("parents", ctypes.c_int64), ("children", ctypes.c_int64),
                ("kept32", ctypes.c_int64), ("kept", ctypes.c_int64),
                ("pool", ctypes.c_int64), ("gub", ctypes.c_double)]


_PD = ctypes.POINTER(ctypes.c_double)


class gb_snapshot(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("block", ctypes.c_int32), ("count", ctypes.c_int64),
                ("lo", ctypes.POINTER(ctypes.c_double)), ("hi", ctypes.POINTER(ctypes.c_double)),
                ("flo", ctypes.POINTER(ctypes.c_double)), ("cyc", ctypes.POINTER(ctypes.c_int32)),
                ("gub", ctypes.c_double), ("generations", ctypes.c_int64)]


class gb_result(ctypes.Structure):
    _fields_ = [("fmin_lo", ctypes.c_double), ("fmin_hi", ctypes.c_double),
                ("n_boxes", ctypes.c_int64), ("n", ctypes.c_int32), ("status", ctypes.c_int32),
                ("box_lo", _PD), ("box_hi", _PD), ("box_flo", _PD),
                ("generations", ctypes.c_int64), ("box_evals_fp32", ctypes.c_int64),
                ("box_evals_fp64", ctypes.c_int64), ("mid_evals", ctypes.c_int64),
                ("solve_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("eval64_ms", ctypes.c_double), ("eval32_ms", ctypes.c_double),
                ("eval64_launches", ctypes.c_int64), ("eval32_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ops64", ctypes.c_int64),
                ("ops32", ctypes.c_int64), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("pool_mode", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("record_gcs", ctypes.c_int64), ("n_trace", ctypes.c_int64),
                ("trace", ctypes.POINTER(gb_gen_stat))]


EXPORTS = ["gb_default_options", "gb_create_problem", "gb_solve", "gb_solve_device",
           "gb_free_result", "gb_destroy_problem", "gb_status_str", "gb_last_error",
           "gb_eval_boxes", "gb_eval_boxes_noalloc", "gb_problem_info", "gb_measure_peak",
           "gb_server_create", "gb_submit", "gb_poll", "gb_server_destroy", "gb_autotune",
           "gb_snapshot_take", "gb_solve_resume", "gb_free_snapshot", "gb_server_set_fused"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgb.so (building it first if needed); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path}")
    L = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.gb_autotune.argtypes = [vp, i32, i32, ctypes.POINTER(_PD), ctypes.POINTER(i64), i32, i32, _PD, _PD,
                              ctypes.c_double, ctypes.POINTER(gb_options), ctypes.c_double,
                              ctypes.POINTER(gb_options), ctypes.POINTER(ctypes.c_double)]
    L.gb_autotune.restype = ctypes.c_int
    L.gb_default_options.argtypes = [ctypes.POINTER(gb_options)]
    L.gb_default_options.restype = None
    L.gb_create_problem.argtypes = [vp, i32, i32, ctypes.POINTER(_PD), ctypes.POINTER(i64), i32, i32,
                                    _PD, _PD, ctypes.c_double, ctypes.POINTER(gb_options),
                                    ctypes.POINTER(vp)]
    L.gb_create_problem.restype = ctypes.c_int
    for fn in ("gb_solve", "gb_solve_device"):
        getattr(L, fn).argtypes = [vp, ctypes.POINTER(gb_result)]
        getattr(L, fn).restype = ctypes.c_int
    L.gb_free_result.argtypes = [ctypes.POINTER(gb_result)]
    L.gb_free_result.restype = None
    L.gb_snapshot_take.argtypes = [vp, ctypes.POINTER(gb_snapshot)]
    L.gb_snapshot_take.restype = ctypes.c_int
    L.gb_solve_resume.argtypes = [vp, ctypes.POINTER(gb_snapshot), ctypes.POINTER(gb_result)]
    L.gb_solve_resume.restype = ctypes.c_int
    L.gb_free_snapshot.argtypes = [ctypes.POINTER(gb_snapshot)]
    L.gb_free_snapshot.restype = None
    L.gb_destroy_problem.argtypes = [vp]
    L.gb_destroy_problem.restype = None
    L.gb_status_str.argtypes = [ctypes.c_int]
    L.gb_status_str.restype = ctypes.c_char_p
    L.gb_last_error.argtypes = []
    L.gb_last_error.restype = ctypes.c_char_p
    for fn in ("gb_eval_boxes", "gb_eval_boxes_noalloc"):
        getattr(L, fn).argtypes = [vp, vp, vp, i64, i32, i32, vp, vp, vp, vp, vp]
        getattr(L, fn).restype = ctypes.c_int
    L.gb_problem_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64)]
    L.gb_problem_info.restype = ctypes.c_int
    L.gb_measure_peak.argtypes = [i32, i32, _PD, _PD]
    L.gb_measure_peak.restype = ctypes.c_int
    L.gb_server_create.argtypes = [ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)]
    L.gb_server_create.restype = ctypes.c_int
    L.gb_server_set_fused.argtypes = [vp, i32]
    L.gb_server_set_fused.restype = ctypes.c_int
    L.gb_submit.argtypes = [vp, vp, i32, i32, ctypes.POINTER(_PD), ctypes.POINTER(i64), i32, i32, _PD, _PD,
                            ctypes.c_double, ctypes.POINTER(gb_options), ctypes.POINTER(ctypes.c_uint64)]
    L.gb_submit.restype = ctypes.c_int
    L.gb_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(gb_result)]
    L.gb_poll.restype = ctypes.c_int
    L.gb_server_destroy.argtypes = [vp]
    L.gb_server_destroy.restype = ctypes.c_int
    _lib = L
    return L


def gb_status_str(status: int) -> str:
    return load().gb_status_str(int(status)).decode()


def gb_last_error() -> str:
    return load().gb_last_error().decode()


def gb_default_options(**overrides) -> gb_options:
    o = gb_options()
    load().gb_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class _Problem:
    """Owns a gb_problem handle and the host arrays passed at creation."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def close(self):
        if self.handle:
            load().gb_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gb_create_problem(nodes: np.ndarray, root: int, tables, n: int, l, u, tol: float,
                      options: gb_options | None = None) -> _Problem:
    L = load()
    nodes = np.ascontiguousarray(nodes)
    if nodes.dtype.itemsize != 32:
        raise ValueError("nodes must use the 32-byte gb_node layout")
    tabs = [np.ascontiguousarray(t, dtype=np.float64) for t in tables]
    ptrs = (_PD * max(1, len(tabs)))(*[t.ctypes.data_as(_PD) for t in tabs])
    lens = (ctypes.c_int64 * max(1, len(tabs)))(*[len(t) for t in tabs])
    l = np.ascontiguousarray(l, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    h = ctypes.c_void_p()
    rc = L.gb_create_problem(nodes.ctypes.data, len(nodes), int(root), ptrs, lens, len(tabs), int(n),
                             l.ctypes.data_as(_PD), u.ctypes.data_as(_PD), float(tol),
                             ctypes.byref(options) if options is not None else None, ctypes.byref(h))
    if rc != GB_OK:
        raise GbError(rc, gb_last_error())
    return _Problem(h, int(n))


def gb_autotune(problem, budget_ms: float = 2000.0, base: gb_options | None = None) -> tuple[gb_options, float]:
    """Fastest fan-out / parents-per-generation / child-kernel setting for a
    problem description (nodes, root, tables, n, l, u, tol_f), by timing
    complete solves; returns (options, solve ms)."""
    L = load()
    nodes = np.ascontiguousarray(problem.nodes)
    tabs = [np.ascontiguousarray(t, dtype=np.float64) for t in problem.tables]
    ptrs = (_PD * max(1, len(tabs)))(*[t.ctypes.data_as(_PD) for t in tabs])
    lens = (ctypes.c_int64 * max(1, len(tabs)))(*[len(t) for t in tabs])
    l = np.ascontiguousarray(problem.l, dtype=np.float64)
    u = np.ascontiguousarray(problem.u, dtype=np.float64)
    best, ms = gb_options(), ctypes.c_double()
    rc = L.gb_autotune(nodes.ctypes.data, len(nodes), int(problem.root), ptrs, lens, len(tabs), int(problem.n),
                       l.ctypes.data_as(_PD), u.ctypes.data_as(_PD), float(problem.tol_f),
                       ctypes.byref(base) if base is not None else None, float(budget_ms), ctypes.byref(best),
                       ctypes.byref(ms))
    if rc != GB_OK:
        raise GbError(rc, gb_last_error())
    return best, ms.value


@dataclass
class Result:
    fmin_lo: float
    fmin_hi: float
    status: int
    n_boxes: int
    box_lo: np.ndarray | None
    box_hi: np.ndarray | None
    box_flo: np.ndarray | None
    generations: int
    box_evals_fp32: int
    box_evals_fp64: int
    mid_evals: int
    solve_ms: float
    device_ms: float
    eval64_ms: float
    eval32_ms: float
    eval64_launches: int
    eval32_launches: int
    kernel_launches: int
    ops64: int
    ops32: int
    queue_ms: float
    latency_ms: float
    pool_mode: int
    record_gcs: int
    trace: dict


def _result(r: gb_result, n: int, rc: int | None = None) -> Result:
    """The host copy of a result; `rc` (the call's return code) is the
    status whenever it is given, so a failed call never reads as OK."""
    nb = r.n_boxes

    def arr(ptr, count):
        if not ptr or count == 0:
            return None
        return np.ctypeslib.as_array(ptr, shape=(count,)).copy()

    lo = arr(r.box_lo, nb * n)
    hi = arr(r.box_hi, nb * n)
    tr = {k: [] for k in ("parents", "children", "kept32", "kept", "pool", "gub")}
    for t in range(r.n_trace):
        g = r.trace[t]
        for k in tr:
            tr[k].append(getattr(g, k))
    tr = {k: np.array(v) for k, v in tr.items()}
    return Result(r.fmin_lo, r.fmin_hi, r.status if rc is None else int(rc), nb,
                  lo.reshape(nb, n) if lo is not None else None,
                  hi.reshape(nb, n) if hi is not None else None,
                  arr(r.box_flo, nb), r.generations, r.box_evals_fp32, r.box_evals_fp64,
                  r.mid_evals, r.solve_ms, r.device_ms, r.eval64_ms, r.eval32_ms,
                  r.eval64_launches, r.eval32_launches, r.kernel_launches, r.ops64, r.ops32,
                  r.queue_ms, r.latency_ms, r.pool_mode, r.record_gcs, tr)


def gb_solve(prob: _Problem, device_only: bool = False, raise_on_error: bool = True) -> Result:
    L = load()
    r = gb_result()
    rc = (L.gb_solve_device if device_only else L.gb_solve)(prob.handle, ctypes.byref(r))
    try:
        res = _result(r, prob.n, rc)
    finally:
        L.gb_free_result(ctypes.byref(r))
    if rc not in (GB_OK, GB_E_CAPACITY, GB_E_LIMIT) and raise_on_error:
        raise GbError(rc, gb_last_error())
    return res


def gb_problem_info(prob: _Problem) -> dict:
    b, nb = ctypes.c_int32(), ctypes.c_int32()
    oe, om = ctypes.c_int64(), ctypes.c_int64()
    rc = load().gb_problem_info(prob.handle, ctypes.byref(b), ctypes.byref(nb), ctypes.byref(oe), ctypes.byref(om))
    if rc != GB_OK:
        raise GbError(rc, gb_last_error())
    return dict(block=b.value, n_blocks=nb.value, ops_eval=oe.value, ops_mid=om.value)


def gb_eval_boxes(prob: _Problem, lo, hi, block_index: int = -1, fp32: bool = False,
                  noalloc: bool = False):
    """Per-box F, midpoint F, block partials and monotonicity verdict.

    lo, hi: torch CUDA float64 tensors (nbox x n).  Returns torch tensors
    (F [nbox, 2], Fmid [nbox, 2], G [nbox, B, 2], mono [nbox]).  With
    noalloc=True the call goes to gb_eval_boxes_noalloc, which uses the
    library's fixed scratch array instead of allocating (at most 2^20
    coordinates per call)."""
    import torch
    L = load()
    fn = L.gb_eval_boxes_noalloc if noalloc else L.gb_eval_boxes
    lo = lo.contiguous()
    hi = hi.contiguous()
    nbox = lo.shape[0]
    B = gb_problem_info(prob)["block"]
    dev = lo.device
    F = torch.empty((nbox, 2), dtype=torch.float64, device=dev)
    Fm = torch.empty((nbox, 2), dtype=torch.float64, device=dev)
    G = torch.full((nbox, B, 2), float("nan"), dtype=torch.float64, device=dev)
    mono = torch.zeros(nbox, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = fn(prob.handle, lo.data_ptr(), hi.data_ptr(), nbox, int(block_index), int(fp32),
                         F.data_ptr(), Fm.data_ptr(), G.data_ptr() if block_index >= 0 else None,
                         mono.data_ptr() if block_index >= 0 else None, stream)
    if rc != GB_OK:
        raise GbError(rc, gb_last_error())
    return F, Fm, G, mono


def gb_measure_peak(device: int = 0, which: int = 0) -> tuple[float, float]:
    """(directed ops per second, kernel ms) of the library's peak probe."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    rc = load().gb_measure_peak(int(device), int(which), ctypes.byref(ops), ctypes.byref(ms))
    if rc != GB_OK:
        raise GbError(rc, gb_last_error())
    return ops.value, ms.value


@dataclass
class Snapshot:
    """The region list a solve left (gb_snapshot): boxes in pool order, their
    lower bounds, cycling words (bit 31: final), the incumbent and the
    generations run so far."""
    n: int
    block: int
    lo: np.ndarray
    hi: np.ndarray
    flo: np.ndarray
    cyc: np.ndarray
    gub: float
    generations: int


def gb_snapshot_take(prob: "_Problem") -> Snapshot:
    L = load()
    s = gb_snapshot()
    rc = L.gb_snapshot_take(prob.handle, ctypes.byref(s))
    try:
        if rc != GB_OK:
            raise GbError(rc, gb_last_error())
        c, n = int(s.count), int(s.n)

        def arr(ptr, count, dt):
            if count == 0:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dt, copy=True)

        return Snapshot(n, int(s.block), arr(s.lo, c * n, np.float64).reshape(c, n),
                        arr(s.hi, c * n, np.float64).reshape(c, n), arr(s.flo, c, np.float64),
                        arr(s.cyc, c, np.int32), float(s.gub), int(s.generations))
    finally:
        L.gb_free_snapshot(ctypes.byref(s))


def gb_solve_resume(prob: "_Problem", snap: Snapshot, raise_on_error: bool = True) -> Result:
    L = load()
    lo = np.ascontiguousarray(snap.lo, dtype=np.float64).reshape(-1)
    hi = np.ascontiguousarray(snap.hi, dtype=np.float64).reshape(-1)
    flo = np.ascontiguousarray(snap.flo, dtype=np.float64)
    cyc = np.ascontiguousarray(snap.cyc, dtype=np.int32)
    s = gb_snapshot(int(snap.n), int(snap.block), len(flo), lo.ctypes.data_as(_PD), hi.ctypes.data_as(_PD),
                    flo.ctypes.data_as(_PD), cyc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    float(snap.gub), int(snap.generations))
    r = gb_result()
    rc = L.gb_solve_resume(prob.handle, ctypes.byref(s), ctypes.byref(r))
    try:
        res = _result(r, prob.n, rc)
    finally:
        L.gb_free_result(ctypes.byref(r))
    if rc not in (GB_OK, GB_E_CAPACITY, GB_E_LIMIT) and raise_on_error:
        raise GbError(rc, gb_last_error())
    return res


class Solver:
    """Convenience wrapper: a problem description (nodes, root, tables, n,
    l, u, tol_f) plus options -> a device-resident problem."""

    def __init__(self, problem, **options):
        opts = gb_default_options()
        opts.block = int(options.pop("block", getattr(problem, "block", 0) or 0))
        for k, v in options.items():
            setattr(opts, k, v)
        self.problem = problem
        self.options = opts
        self.h = gb_create_problem(problem.nodes, problem.root, problem.tables, problem.n,
                                   problem.l, problem.u, problem.tol_f, opts)

    def solve(self, device_only: bool = False, raise_on_error: bool = True) -> Result:
        return gb_solve(self.h, device_only=device_only, raise_on_error=raise_on_error)

    def eval_boxes(self, lo, hi, block_index: int = -1, fp32: bool = False):
        return gb_eval_boxes(self.h, lo, hi, block_index, fp32)

    def snapshot(self) -> "Snapshot":
        return gb_snapshot_take(self.h)

    def resume(self, snap: "Snapshot", raise_on_error: bool = True) -> Result:
        return gb_solve_resume(self.h, snap, raise_on_error=raise_on_error)

    def info(self) -> dict:
        return gb_problem_info(self.h)

    def close(self):
        self.h.close()


class Server:
    """Binding of the gb_server_* calls (continuous batching on one GPU)."""

    def __init__(self, pool_budget_bytes: int, device: int = 0, max_active: int = 16, fused: bool = False):
        h = ctypes.c_void_p()
        rc = load().gb_server_create(int(pool_budget_bytes), int(device), int(max_active), ctypes.byref(h))
        if rc != GB_OK:
            raise GbError(rc, gb_last_error())
        self.h = h
        self.set_fused(fused)

    def set_fused(self, fused: bool):
        rc = load().gb_server_set_fused(self.h, int(bool(fused)))
        if rc != GB_OK:
            raise GbError(rc, gb_last_error())
        self._n = {}

    def submit(self, problem, options: gb_options | None = None) -> int:
        """Queue a problem description (nodes, root, tables, n, l, u, tol_f)."""
        nodes = np.ascontiguousarray(problem.nodes)
        tabs = [np.ascontiguousarray(t, dtype=np.float64) for t in problem.tables]
        ptrs = (_PD * max(1, len(tabs)))(*[t.ctypes.data_as(_PD) for t in tabs])
        lens = (ctypes.c_int64 * max(1, len(tabs)))(*[len(t) for t in tabs])
        l = np.ascontiguousarray(problem.l, dtype=np.float64)
        u = np.ascontiguousarray(problem.u, dtype=np.float64)
        rid = ctypes.c_uint64()
        rc = load().gb_submit(self.h, nodes.ctypes.data, len(nodes), int(problem.root), ptrs, lens, len(tabs),
                              int(problem.n), l.ctypes.data_as(_PD), u.ctypes.data_as(_PD),
                              float(problem.tol_f), ctypes.byref(options) if options is not None else None,
                              ctypes.byref(rid))
        if rc != GB_OK:
            raise GbError(rc, gb_last_error())
        self._n[rid.value] = int(problem.n)
        return rid.value

    def poll(self, rid: int):
        """None while running; the Result once finished."""
        L = load()
        r = gb_result()
        rc = L.gb_poll(self.h, ctypes.c_uint64(rid), ctypes.byref(r))
        if rc == GB_E_BUSY:
            return None
        n = self._n.pop(rid, None)
        try:
            res = _result(r, n) if n is not None else None
        finally:
            L.gb_free_result(ctypes.byref(r))
        if rc not in (GB_OK, GB_E_CAPACITY, GB_E_LIMIT):
            raise GbError(rc, gb_last_error())
        return res

    def close(self):
        if self.h:
            load().gb_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
