"""CPU oracle for the interval branch-and-bound minimiser (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It builds ``oracle.c`` (plain C, fesetround
directed rounding, FP64 and FP32) with gcc and exposes it through ctypes.
It imports nothing from the CUDA library and the CUDA library imports nothing
from it; both read the same objective description from ``synthetic``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_CFLAGS = ["-O1", "-frounding-math", "-ffp-contract=off", "-fno-fast-math",
           "-fno-math-errno", "-pthread", "-shared", "-fPIC"]
_lock = threading.Lock()
_lib = None

# operator codes of the objective node format (see synthetic.dag)
OP = dict(CONST=0, PI=1, EULER=2, VAR=3, IDX_VAR=4, IDX_COEF=5, ADD=6, SUB=7,
          MUL=8, DIV=9, NEG=10, SQR=11, SQRT=12, EXP=13, SIN=14, COS=15,
          SCALE=16, ISUM=17, IPROD=18, STEP=19)

ST_OK, ST_INVALID, ST_CAPACITY, ST_LIMIT = 0, 1, 3, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_CFLAGS, _SRC, "-lm", "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Opts(ctypes.Structure):
    _fields_ = [("tol_f", ctypes.c_double), ("tol_x", ctypes.c_double),
                ("split_m", ctypes.c_int32), ("split_d", ctypes.c_int32),
                ("fp32", ctypes.c_int32), ("samples", ctypes.c_int32),
                ("max_gen", ctypes.c_int64), ("max_parents", ctypes.c_int64),
                ("cap", ctypes.c_int64), ("mono_all", ctypes.c_int32), ("threads", ctypes.c_int32)]


_P64 = ctypes.POINTER(ctypes.c_int64)
_PD = ctypes.POINTER(ctypes.c_double)


class _Result(ctypes.Structure):
    _fields_ = [("glb", ctypes.c_double), ("gub", ctypes.c_double),
                ("n_boxes", ctypes.c_int64),
                ("box_lo", _PD), ("box_hi", _PD), ("box_flo", _PD),
                ("box_cyc", ctypes.POINTER(ctypes.c_int32)),
                ("generations", ctypes.c_int64), ("evals32", ctypes.c_int64),
                ("evals64", ctypes.c_int64), ("mids", ctypes.c_int64),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n_trace", ctypes.c_int64),
                ("tr_parents", _P64), ("tr_children", _P64), ("tr_kept32", _P64),
                ("tr_kept", _P64), ("tr_pool", _P64), ("tr_gub", _PD)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, dp, ip = ctypes.c_void_p, _PD, ctypes.c_int
            L.oracle_create.restype = vp
            L.oracle_create.argtypes = [vp, ip, ip, ctypes.POINTER(dp), _P64, ip, ip,
                                        dp, dp, ip]
            L.oracle_destroy.argtypes = [vp]
            L.oracle_n_blocks.argtypes = [vp]
            L.oracle_n_blocks.restype = ip
            L.oracle_eval_box.argtypes = [vp, dp, dp, ip, ip, dp, dp, dp,
                                          ctypes.POINTER(ctypes.c_int32)]
            L.oracle_eval_box_dev.argtypes = [vp, dp, dp, ip, ip, dp, dp, dp, dp, dp, dp]
            L.oracle_set_extra_widening.argtypes = [ip]
            L.oracle_iv_op.argtypes = [ip, dp, dp, ctypes.c_double, ip, dp]
            L.oracle_tree_sum.argtypes = [dp, dp, ip, ip, dp]
            L.oracle_iv_op_batch.argtypes = [ip, dp, dp, dp, dp, dp, ctypes.c_int64, ip, dp]
            L.oracle_tree_prod.argtypes = [dp, dp, ip, ip, dp]
            L.oracle_tree_prod_adjoint.argtypes = [dp, dp, ip, ctypes.c_double, ctypes.c_double, ip, dp]
            L.oracle_solve.argtypes = [vp, ctypes.POINTER(_Opts), ctypes.POINTER(_Result)]
            L.oracle_solve.restype = ip
            L.oracle_free_result.argtypes = [ctypes.POINTER(_Result)]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def iv_op(op: str, x, y=(0.0, 0.0), c: float = 0.0, f32: bool = False):
    """One interval operation of the oracle, returned as (lo, hi)."""
    xa = np.asarray(x, dtype=np.float64)
    ya = np.asarray(y, dtype=np.float64)
    out = np.zeros(2)
    rc = lib().oracle_iv_op(OP[op], _dp(xa), _dp(ya), float(c), int(f32), _dp(out))
    if rc:
        raise ValueError(op)
    return float(out[0]), float(out[1])


def iv_op_batch(op: str, xlo, xhi, ylo=None, yhi=None, c=None, f32: bool = False) -> np.ndarray:
    """iv_op over arrays of operands; returns (count, 2) [lo, hi]."""
    xlo = np.ascontiguousarray(xlo, dtype=np.float64)
    xhi = np.ascontiguousarray(xhi, dtype=np.float64)
    ylo = np.ascontiguousarray(ylo if ylo is not None else np.zeros_like(xlo), dtype=np.float64)
    yhi = np.ascontiguousarray(yhi if yhi is not None else np.zeros_like(xlo), dtype=np.float64)
    cc = np.ascontiguousarray(c if c is not None else np.zeros_like(xlo), dtype=np.float64)
    out = np.zeros((len(xlo), 2))
    if lib().oracle_iv_op_batch(OP[op], _dp(xlo), _dp(xhi), _dp(ylo), _dp(yhi), _dp(cc), len(xlo), int(f32),
                                _dp(out)):
        raise ValueError(op)
    return out


def set_extra_widening(k: int) -> None:
    """Test hook: widen every transcendental endpoint by k more ulps (0: the
    oracle's own rule).  Used only to perturb library values when pinning
    the deviation bound."""
    lib().oracle_set_extra_widening(int(k))


def tree_sum(lo, hi, f32: bool = False):
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_tree_sum(_dp(lo), _dp(hi), len(lo), int(f32), _dp(out))
    return float(out[0]), float(out[1])


def tree_prod(lo, hi, f32: bool = False):
    """The IPROD reduction tree (the pairwise tree of tree_sum with products)."""
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_tree_prod(_dp(lo), _dp(hi), len(lo), int(f32), _dp(out))
    return float(out[0]), float(out[1])


def tree_prod_adjoint(lo, hi, seed=(1.0, 1.0), f32: bool = False):
    """Adjoint of every item of the IPROD tree for a product adjoint seed; (m, 2)."""
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = np.zeros((len(lo), 2))
    lib().oracle_tree_prod_adjoint(_dp(lo), _dp(hi), len(lo), float(seed[0]), float(seed[1]), int(f32),
                                   _dp(out))
    return out


@dataclass
class SolveResult:
    glb: float
    gub: float
    status: int
    box_lo: np.ndarray
    box_hi: np.ndarray
    box_flo: np.ndarray
    box_cyc: np.ndarray
    generations: int
    evals32: int
    evals64: int
    mids: int
    trace: dict


class Oracle:
    """Handle on one problem inside the C oracle."""

    def __init__(self, problem, block: int | None = None):
        self.p = problem
        self.B = int(block if block else problem.block)
        self._tabs = [np.ascontiguousarray(t, dtype=np.float64) for t in problem.tables]
        ptrs = (_PD * max(1, len(self._tabs)))(*[_dp(t) for t in self._tabs])
        lens = np.array([len(t) for t in self._tabs] or [0], dtype=np.int64)
        self._nodes = np.ascontiguousarray(problem.nodes)
        self._l = np.ascontiguousarray(problem.l, dtype=np.float64)
        self._u = np.ascontiguousarray(problem.u, dtype=np.float64)
        self.h = lib().oracle_create(self._nodes.ctypes.data, len(self._nodes), int(problem.root),
                                     ptrs, lens.ctypes.data_as(_P64), len(self._tabs),
                                     int(problem.n), _dp(self._l), _dp(self._u), self.B)
        if not self.h:
            raise ValueError("oracle rejected the problem")

    def close(self):
        if getattr(self, "h", None):
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def eval_box(self, lo, hi, blk: int = -1, f32: bool = False):
        """(F, Fmid, G[width], mono) for one box; G and mono only if blk >= 0."""
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        F = np.zeros(2)
        Fm = np.zeros(2)
        G = np.zeros(2 * self.B)
        mono = ctypes.c_int32(0)
        lib().oracle_eval_box(self.h, _dp(lo), _dp(hi), int(f32), int(blk), _dp(F), _dp(Fm),
                              _dp(G), ctypes.byref(mono))
        return F, Fm, G.reshape(self.B, 2), int(mono.value)

    def eval_box_dev(self, lo, hi, blk: int = -1, f32: bool = False):
        """eval_box's F, Fmid and G with their deviation bounds: (F, dF,
        Fmid, dFmid, G[width], dG[width]).  An implementation running the
        same operations whose exp / sin / cos endpoints are within a few ulps
        of the oracle's gives endpoints within these bounds (0 for
        objectives without transcendentals)."""
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        F, dF, Fm, dFm = np.zeros(2), np.zeros(1), np.zeros(2), np.zeros(1)
        G = np.zeros(2 * self.B)
        dG = np.zeros(self.B)
        lib().oracle_eval_box_dev(self.h, _dp(lo), _dp(hi), int(f32), int(blk), _dp(F), _dp(dF), _dp(Fm),
                                  _dp(dFm), _dp(G), _dp(dG))
        return F, float(dF[0]), Fm, float(dFm[0]), G.reshape(self.B, 2), dG

    def solve(self, tol_f: float | None = None, tol_x: float = 0.0, split_m: int = 2,
              split_d: int = 1, fp32: bool = False, max_gen: int = 10**9,
              max_parents: int = 1 << 20, cap: int = 1 << 40, samples: int = 0,
              mono_all: bool = False, threads: int = 1) -> SolveResult:
        """samples: 0 one midpoint sample per box, S > 0 the S interior diagonal
        points j / (S + 1); mono_all: first-order test on every coordinate
        (the paper's rule) instead of the active block; threads: threads for
        the per-child loops of a generation (the result does not depend on
        it)."""
        o = _Opts(tol_f=float(self.p.tol_f if tol_f is None else tol_f), tol_x=float(tol_x),
                  split_m=split_m, split_d=split_d, fp32=int(fp32), samples=int(samples),
                  max_gen=max_gen, max_parents=max_parents, cap=cap, mono_all=int(mono_all),
                  threads=int(threads))
        r = _Result()
        lib().oracle_solve(self.h, ctypes.byref(o), ctypes.byref(r))
        try:
            n, nb = self.p.n, r.n_boxes
            def arr(ptr, count, dt):
                if count == 0:
                    return np.zeros(0, dtype=dt)
                return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dt, copy=True)
            nt = r.n_trace
            res = SolveResult(
                glb=r.glb, gub=r.gub, status=r.status,
                box_lo=arr(r.box_lo, nb * n, np.float64).reshape(nb, n),
                box_hi=arr(r.box_hi, nb * n, np.float64).reshape(nb, n),
                box_flo=arr(r.box_flo, nb, np.float64),
                box_cyc=arr(r.box_cyc, nb, np.int32),
                generations=r.generations, evals32=r.evals32, evals64=r.evals64, mids=r.mids,
                trace=dict(parents=arr(r.tr_parents, nt, np.int64),
                           children=arr(r.tr_children, nt, np.int64),
                           kept32=arr(r.tr_kept32, nt, np.int64),
                           kept=arr(r.tr_kept, nt, np.int64),
                           pool=arr(r.tr_pool, nt, np.int64),
                           gub=arr(r.tr_gub, nt, np.float64)))
        finally:
            lib().oracle_free_result(ctypes.byref(r))
        return res
