"""CPU oracle for the SpTRSV hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import this package.  The product library never loads it and shares no
code with it; the only thing both sides consume is the seeded input generator module.

The arithmetic lives in ``sptrsv_oracle.c`` (plain serial C, fp64, compiled with
``-ffp-contract=off``); this module compiles it with gcc on first use and wraps it with
numpy arrays.  The MLP and feature oracles are in ``mlp.py`` and ``features.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sptrsv_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

NAIVE, DEPTH, CHOSEN, MANUAL, CHOSEN_THIN, ROWCAP = 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_lib/liboracle.so (plain gcc, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i64, i32, dbl, vp = C.c_int64, C.c_int32, C.c_double, C.c_void_p
        lib.orc_validate.argtypes = [i64, vp, vp, vp, C.POINTER(i64)]
        lib.orc_validate.restype = C.c_int
        lib.orc_forward_subst.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.orc_forward_subst.restype = None
        lib.orc_forward_subst_f32vals.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.orc_forward_subst_f32vals.restype = None
        lib.orc_backward_subst.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.orc_backward_subst.restype = None
        lib.orc_levels.argtypes = [i64, vp, vp, C.c_int, vp]
        lib.orc_levels.restype = i32
        lib.orc_level_stats.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        lib.orc_level_stats.restype = None
        lib.orc_plan.argtypes = [i64, vp, vp, vp, i32, C.c_int, i32, dbl, dbl, vp, vp, vp, vp, vp]
        lib.orc_plan.restype = C.c_int
        lib.orc_plan_rules.argtypes = [i64, vp, vp, vp, i32, C.c_int, i32, dbl, dbl, vp, vp, i32, i64, vp, vp, vp]
        lib.orc_plan_rules.restype = C.c_int
        lib.orc_plan_parts.argtypes = [i64, vp, vp, vp, i32, C.c_int, i32, dbl, dbl, vp, vp, i32, i64, i32, vp, vp,
                                       vp]
        lib.orc_plan_parts.restype = C.c_int
        lib.orc_rewrite.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.orc_rewrite.restype = vp
        lib.orc_system_free.argtypes = [vp]
        lib.orc_system_free.restype = None
        lib.orc_system_nnz_c.argtypes = [vp]
        lib.orc_system_nnz_c.restype = i64
        lib.orc_system_nnz_e.argtypes = [vp]
        lib.orc_system_nnz_e.restype = i64
        lib.orc_system_copy.argtypes = [vp] * 9
        lib.orc_system_copy.restype = None
        lib.orc_system_levels.argtypes = [vp, vp]
        lib.orc_system_levels.restype = i32
        lib.orc_solve_rewritten.argtypes = [vp, vp, vp]
        lib.orc_solve_rewritten.restype = None
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------------------------
# wrappers
# ------------------------------------------------------------------------------------

def validate(rowptr, colidx, vals) -> tuple[int, int]:
    """(code, first bad row); code 0 means the CSR contract of Algorithm 1 holds."""
    rp, ci, v = _i32(rowptr), _i32(colidx), _f64(vals)
    bad = C.c_int64(-1)
    code = _load().orc_validate(rp.size - 1, _p(rp), _p(ci), _p(v), C.byref(bad))
    return int(code), int(bad.value)


def forward_subst(rowptr, colidx, vals, b) -> np.ndarray:
    """Algorithm 1 for every right-hand side.  b: shape (n,) or (nrhs, n)."""
    lib = _load()
    rp, ci = _i32(rowptr), _i32(colidx)
    b = _f64(b)
    one = b.ndim == 1
    B = b[None, :] if one else b
    X = np.empty_like(B)
    n = rp.size - 1
    if np.asarray(vals).dtype == np.float32:
        v = np.ascontiguousarray(vals, dtype=np.float32)
        for k in range(B.shape[0]):
            bk, xk = np.ascontiguousarray(B[k]), np.empty(n)
            lib.orc_forward_subst_f32vals(n, _p(rp), _p(ci), _p(v), _p(bk), _p(xk))
            X[k] = xk
    else:
        v = _f64(vals)
        for k in range(B.shape[0]):
            bk, xk = np.ascontiguousarray(B[k]), np.empty(n)
            lib.orc_forward_subst(n, _p(rp), _p(ci), _p(v), _p(bk), _p(xk))
            X[k] = xk
    return X[0] if one else X


def backward_subst(rowptr, colidx, vals, b) -> np.ndarray:
    """x = U^{-1} b for an upper-triangular CSR U with the diagonal first in each row."""
    lib = _load()
    rp, ci, v = _i32(rowptr), _i32(colidx), _f64(vals)
    b = _f64(b)
    one = b.ndim == 1
    B = b[None, :] if one else b
    X = np.empty_like(B)
    n = rp.size - 1
    for k in range(B.shape[0]):
        bk, xk = np.ascontiguousarray(B[k]), np.empty(n)
        lib.orc_backward_subst(n, _p(rp), _p(ci), _p(v), _p(bk), _p(xk))
        X[k] = xk
    return X[0] if one else X


def levels(rowptr, colidx, diag_last: bool = True) -> tuple[np.ndarray, int]:
    """(level[n], m) by the definition level(i) = 1 + max level of its dependencies."""
    rp, ci = _i32(rowptr), _i32(colidx)
    n = rp.size - 1
    lev = np.empty(max(n, 1), dtype=np.int32)
    m = _load().orc_levels(n, _p(rp), _p(ci), 1 if diag_last else 0, _p(lev))
    return lev[:n], int(m)


def level_stats(rowptr, level, m) -> dict:
    rp, lv = _i32(rowptr), _i32(level)
    rows = np.empty(max(m, 1), np.int64)
    nnz = np.empty(max(m, 1), np.int64)
    cost = np.empty(max(m, 1), np.int64)
    _load().orc_level_stats(rp.size - 1, _p(rp), _p(lv), m, _p(rows), _p(nnz), _p(cost))
    return {"rows": rows[:m], "nnz": nnz[:m], "cost": cost[:m]}


@dataclass
class Plan:
    target: np.ndarray      # int32[n]: level each row ends on (original numbering)
    row_cost: np.ndarray    # int64[n]
    moved: int
    stored_nnz: int         # nnz(L') + nnz(E explicit rows)
    nnz_l: int
    levels_after: int       # non-empty levels after the moves
    avg: float
    targets: int


def plan(rowptr, colidx, level, m, kind: int, k: int = 0, avg: float = 0.0, cap: float = 0.0,
         injected_cost=None, depth_of_target=None, alpha: int = 0, beta: int = 0, parts: int = 1) -> Plan:
    """The Section III planner (NAIVE / DEPTH / CHOSEN / MANUAL / CHOSEN_THIN / ROWCAP), with the per-row rules of
    Section III.A (alpha: fewer dependencies than alpha; beta: dependency spread below beta); parts > 1 starts the
    walk at the beginning of every one of `parts` equal level ranges (2: from both ends, Section III)."""
    rp, ci, lv = _i32(rowptr), _i32(colidx), _i32(level)
    n = rp.size - 1
    tgt = np.empty(max(n, 1), np.int32)
    rc = np.empty(max(n, 1), np.int64)
    info = np.zeros(6, np.int64)
    inj = None if injected_cost is None else np.ascontiguousarray(injected_cost, dtype=np.int64)
    dot = None if depth_of_target is None else _i32(depth_of_target)
    rc_ = _load().orc_plan_parts(n, _p(rp), _p(ci), _p(lv), int(m), int(kind), int(k), float(avg), float(cap),
                                 None if inj is None else _p(inj), None if dot is None else _p(dot),
                                 int(alpha), int(beta), int(parts), _p(tgt), _p(rc), _p(info))
    if rc_ != 0:
        raise MemoryError("oracle planner allocation failed")
    return Plan(tgt[:n].copy(), rc[:n].copy(), int(info[0]), int(info[1]), int(info[2]), int(info[3]),
                info[4] / 1e6, int(info[5]))


@dataclass
class System:
    """A rewritten system in the original row numbering (see orc_system in the C file)."""
    n: int
    cptr: np.ndarray
    ccol: np.ndarray
    cval: np.ndarray
    dval: np.ndarray
    eptr: np.ndarray
    ecol: np.ndarray
    eval: np.ndarray
    moved: np.ndarray
    _h: int = 0

    def levels(self) -> tuple[np.ndarray, int]:
        lev = np.empty(max(self.n, 1), np.int32)
        m = _load().orc_system_levels(C.c_void_p(self._h), _p(lev))
        return lev[:self.n], int(m)

    def solve(self, b) -> np.ndarray:
        b = _f64(b)
        one = b.ndim == 1
        B = b[None, :] if one else b
        X = np.empty_like(B)
        for k in range(B.shape[0]):
            bk, xk = np.ascontiguousarray(B[k]), np.empty(self.n)
            _load().orc_solve_rewritten(C.c_void_p(self._h), _p(bk), _p(xk))
            X[k] = xk
        return X[0] if one else X

    def close(self):
        if self._h:
            _load().orc_system_free(C.c_void_p(self._h))
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rewrite(rowptr, colidx, vals, level, target) -> System:
    """Equation rewriting with rearrangement for the rows whose target is above their level."""
    lib = _load()
    rp, ci, v, lv, tg = _i32(rowptr), _i32(colidx), _f64(vals), _i32(level), _i32(target)
    n = rp.size - 1
    h = lib.orc_rewrite(n, _p(rp), _p(ci), _p(v), _p(lv), _p(tg))
    if not h:
        raise MemoryError("oracle rewrite allocation failed")
    nc, ne = lib.orc_system_nnz_c(h), lib.orc_system_nnz_e(h)
    cptr = np.empty(n + 1, np.int64); eptr = np.empty(n + 1, np.int64)
    ccol = np.empty(max(nc, 1), np.int32); cval = np.empty(max(nc, 1))
    ecol = np.empty(max(ne, 1), np.int32); evl = np.empty(max(ne, 1))
    dval = np.empty(max(n, 1)); moved = np.empty(max(n, 1), np.int32)
    lib.orc_system_copy(h, _p(cptr), _p(ccol), _p(cval), _p(dval), _p(eptr), _p(ecol), _p(evl), _p(moved))
    return System(n, cptr, ccol[:nc], cval[:nc], dval[:n], eptr, ecol[:ne], evl[:ne], moved[:n], h)
