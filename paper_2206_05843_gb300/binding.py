"""Thin Python binding of libsptrsv.so (the C ABI in include/sptrsv.h).

Argument marshalling only: torch supplies device memory and the current CUDA stream,
every step of analysis, rewriting and solving runs in the library's CUDA kernels.
Importing this module does not touch the GPU; the first call loads the library and
raises if it is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsptrsv.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC, ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "NUMERIC", 6: "UNSUPPORTED"}
F64, F32 = 0, 1
NONE, NAIVE, DEPTH_K, LEARNED, CHOSEN, MANUAL, ROWCAP, CHOSEN_THIN = 0, 1, 2, 3, 4, 5, 6, 7
PICKER_FEATURES, PICKER_HIDDEN = 12, 64
PICKER_PARAMS = 12 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1

# every symbol include/sptrsv.h declares
EXPORTED = [
    "sptrsv_last_error", "sptrsv_validate", "sptrsv_analyse", "sptrsv_levels_stats", "sptrsv_levels_export",
    "sptrsv_levels_destroy", "sptrsv_system_plain", "sptrsv_rewrite", "sptrsv_system_info_get",
    "sptrsv_system_export", "sptrsv_system_destroy", "sptrsv_solve", "sptrsv_solve_timed", "sptrsv_solve_status",
    "sptrsv_solve_noalloc", "sptrsv_system_autotune", "sptrsv_upper_to_lower", "sptrsv_system_reverse_rows",
    "sptrsv_debug_set_wait", "sptrsv_system_tune", "sptrsv_system_tune_cluster", "sptrsv_batch_create",
    "sptrsv_batch_solve",
    "sptrsv_batch_info_get", "sptrsv_batch_destroy", "sptrsv_picker_create", "sptrsv_picker_destroy",
    "sptrsv_picker_get_params", "sptrsv_picker_set_params", "sptrsv_picker_set_norm", "sptrsv_picker_save",
    "sptrsv_picker_load", "sptrsv_picker_features", "sptrsv_picker_infer", "sptrsv_picker_grad",
    "sptrsv_picker_train_step", "sptrsv_debug_run_blocks",
]


class SptrsvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("vals", C.c_void_p), ("dtype", C.c_int32)]


class LevelStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("nnz", C.c_int64), ("total_cost", C.c_int64),
                ("avg_cost", C.c_double), ("max_width", C.c_int64)]


class Strategy(C.Structure):
    _fields_ = [("kind", C.c_int32), ("k", C.c_int32), ("nnz_growth_cap", C.c_double),
                ("avg_override", C.c_double), ("growth_guard", C.c_double), ("picker", C.c_void_p),
                ("depth_of_target_host", C.c_void_p), ("depths_host", C.c_void_p), ("n_depths", C.c_int32),
                ("injected_cost_dev", C.c_void_p), ("max_deps", C.c_int32), ("max_spread", C.c_int64),
                ("learned_mode", C.c_int32), ("walk_parts", C.c_int32)]


class SystemInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("nnz_c", C.c_int64), ("nnz_e", C.c_int64),
                ("rows_moved", C.c_int64), ("stored_nnz", C.c_int64), ("nnz_l", C.c_int64),
                ("segments", C.c_int64), ("run_levels", C.c_int64), ("dtype", C.c_int32),
                ("rewritten", C.c_int32), ("avg_cost", C.c_double), ("block", C.c_int32),
                ("run_width", C.c_int32), ("lanes_per_row", C.c_int32), ("strategy_used", C.c_int32),
                ("launches", C.c_int32), ("ctas", C.c_int32), ("candidate_us", C.c_double * 4),
                ("cluster", C.c_int32), ("cluster_setting", C.c_int32), ("cluster_levels", C.c_int64),
                ("cluster_rows", C.c_int64), ("tiled_levels", C.c_int64), ("tiles_setting", C.c_int32),
                ("reserved0", C.c_int32), ("shared_x_levels", C.c_int64), ("shared_x_setting", C.c_int32),
                ("reserved1", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("count", C.c_int32), ("block", C.c_int32), ("lanes_per_row", C.c_int32), ("graph", C.c_int32),
                ("tuned_us", C.c_double), ("items", C.c_int32), ("split_policy", C.c_int32)]


_lib = None
_lock = threading.Lock()


def load():
    """Loads libsptrsv.so; raises when it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2206_05843_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "sptrsv_last_error": [C.c_char_p, C.c_size_t],
            "sptrsv_validate": [vp, vp],
            "sptrsv_analyse": [vp, C.POINTER(vp), vp],
            "sptrsv_levels_stats": [vp, vp],
            "sptrsv_levels_export": [vp, vp, vp, vp, vp, vp, vp, vp],
            "sptrsv_system_plain": [vp, vp, C.POINTER(vp), vp],
            "sptrsv_rewrite": [vp, vp, vp, C.POINTER(vp), vp],
            "sptrsv_system_info_get": [vp, vp],
            "sptrsv_system_export": [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "sptrsv_solve": [vp, vp, vp, i32, i64, vp],
            "sptrsv_solve_timed": [vp, vp, vp, i32, i64, vp, vp],
            "sptrsv_solve_status": [vp, vp],
            "sptrsv_solve_noalloc": [vp, vp, vp, i32, i64, vp],
            "sptrsv_debug_set_wait": [vp, i64, i64],
            "sptrsv_debug_run_blocks": [vp, i64, vp, i32, i32, i32, vp, i64, vp, vp],
            "sptrsv_system_tune": [vp, i32, i32, i32],
            "sptrsv_system_tune_cluster": [vp, i32, i64, i32, i32],
            "sptrsv_system_autotune": [vp, i32, vp, vp],
            "sptrsv_upper_to_lower": [vp, vp, vp, vp, vp],
            "sptrsv_system_reverse_rows": [vp, vp],
            "sptrsv_batch_create": [vp, vp, i32, C.POINTER(vp), vp],
            "sptrsv_batch_solve": [vp, vp, vp, vp],
            "sptrsv_batch_info_get": [vp, vp],
            "sptrsv_picker_create": [C.c_uint64, C.POINTER(vp)],
            "sptrsv_picker_get_params": [vp, vp],
            "sptrsv_picker_set_params": [vp, vp],
            "sptrsv_picker_set_norm": [vp, vp, vp, C.c_float],
            "sptrsv_picker_save": [vp, C.c_char_p],
            "sptrsv_picker_load": [vp, C.c_char_p],
            "sptrsv_picker_features": [vp, vp, vp, i32, vp, vp],
            "sptrsv_picker_infer": [vp, vp, i64, vp, i32, vp],
            "sptrsv_picker_grad": [vp, vp, vp, i64, i32, vp, vp, vp],
            "sptrsv_picker_train_step": [vp, vp, vp, i64, C.c_float, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        for name in ("sptrsv_levels_destroy", "sptrsv_system_destroy", "sptrsv_batch_destroy",
                     "sptrsv_picker_destroy"):
            f = getattr(lib, name)
            f.argtypes = [vp]
            f.restype = None
        _lib = lib
        return lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    load().sptrsv_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(code: int):
    if code != OK:
        raise SptrsvError(code, last_error())


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr() if t is not None else 0)


# ------------------------------------------------------------------------------------
# matrices
# ------------------------------------------------------------------------------------

class Matrix:
    """A lower-triangular CSR matrix resident on the GPU (tensors kept alive here)."""

    def __init__(self, n, rowptr, colidx, vals):
        torch = _torch()
        self.n = int(n)
        self.rowptr = rowptr
        self.colidx = colidx
        self.vals = vals
        self.dtype = F64 if vals.dtype == torch.float64 else F32
        self.csr = Csr(self.n, int(colidx.numel()), rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr(), self.dtype)

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    @classmethod
    def from_host(cls, m, device="cuda", dtype=None):
        """From a synth.LowerCsr (or anything with n/rowptr/colidx/vals numpy arrays)."""
        torch = _torch()
        vals = np.asarray(m.vals)
        if dtype is not None:
            vals = vals.astype(dtype)
        tdt = torch.float64 if vals.dtype == np.float64 else torch.float32
        rp = torch.from_numpy(np.ascontiguousarray(m.rowptr, dtype=np.int32)).to(device)
        ci = torch.from_numpy(np.ascontiguousarray(m.colidx, dtype=np.int32)).to(device)
        va = torch.from_numpy(np.ascontiguousarray(vals)).to(device=device, dtype=tdt)
        return cls(m.n, rp, ci, va)

    def validate(self):
        check(load().sptrsv_validate(C.byref(self.csr), _stream()))


def upper_to_lower(U: "Matrix") -> "Matrix":
    """The lower-triangular matrix of the reversed index order of an upper-triangular U
    (diagonal first in each row), computed on the device."""
    torch = _torch()
    rp = torch.empty_like(U.rowptr)
    ci = torch.empty_like(U.colidx)
    va = torch.empty_like(U.vals)
    check(load().sptrsv_upper_to_lower(C.byref(U.csr), _ptr(rp), _ptr(ci), _ptr(va), _stream()))
    return Matrix(U.n, rp, ci, va)


def solve_upper(U: "Matrix", b, kind=NONE, **kw):
    """x = U^{-1} b through the reversed lower-triangular system (plain or rewritten)."""
    L = upper_to_lower(U)
    lv = Levels(L)
    s = System(L, lv, kind, **kw).reverse_rows()
    return s.solve(b, check_status=True), s, (L, lv)


class Levels:
    def __init__(self, matrix: Matrix):
        h = C.c_void_p()
        check(load().sptrsv_analyse(C.byref(matrix.csr), C.byref(h), _stream()))
        self.h = h
        self.matrix = matrix
        st = LevelStats()
        check(load().sptrsv_levels_stats(h, C.byref(st)))
        self.n, self.m, self.nnz = st.n, st.m, st.nnz
        self.total_cost, self.avg_cost, self.max_width = st.total_cost, st.avg_cost, st.max_width

    def export(self) -> dict:
        torch = _torch()
        dev = self.matrix.rowptr.device
        n, m = self.n, self.m
        level = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        lptr = torch.empty(m + 1, dtype=torch.int32, device=dev)
        lrows = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        rows = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
        nnz = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
        cost = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
        check(load().sptrsv_levels_export(self.h, _ptr(level), _ptr(lptr), _ptr(lrows), _ptr(rows), _ptr(nnz),
                                          _ptr(cost), _stream()))
        return {"level": level[:n].cpu().numpy(), "level_ptr": lptr.cpu().numpy(), "level_rows": lrows[:n].cpu().numpy(),
                "rows": rows[:m].cpu().numpy(), "nnz": nnz[:m].cpu().numpy(), "cost": cost[:m].cpu().numpy()}

    def close(self):
        if getattr(self, "h", None):
            load().sptrsv_levels_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def strategy(kind=NONE, k=0, cap=0.0, avg=0.0, guard=0.0, picker=None, depth_of_target=None, depths=None,
             injected_cost=None, alpha=0, beta=0, model_only=False, walk_parts=1) -> tuple[Strategy, list]:
    """Builds an sptrsv_strategy; returns it with the objects that must stay alive."""
    keep = []
    s = Strategy()
    s.kind, s.k, s.nnz_growth_cap, s.avg_override, s.growth_guard = kind, k, cap, avg, guard
    s.max_deps, s.max_spread = alpha, beta
    s.learned_mode = 1 if model_only else 0
    s.walk_parts = int(walk_parts)
    s.picker = picker.h if picker is not None else None
    if depth_of_target is not None:
        a = np.ascontiguousarray(depth_of_target, dtype=np.int32)
        keep.append(a)
        s.depth_of_target_host = a.ctypes.data
    if depths is not None:
        a = np.ascontiguousarray(depths, dtype=np.int32)
        keep.append(a)
        s.depths_host = a.ctypes.data
        s.n_depths = a.size
    if injected_cost is not None:
        keep.append(injected_cost)
        s.injected_cost_dev = injected_cost.data_ptr()
    return s, keep


class System:
    """A stored system (plain or rewritten) that sptrsv_solve runs on."""

    def __init__(self, matrix: Matrix, levels: Levels, kind=NONE, **kw):
        h = C.c_void_p()
        if kind == NONE and not kw:
            check(load().sptrsv_system_plain(C.byref(matrix.csr), levels.h, C.byref(h), _stream()))
        else:
            s, keep = strategy(kind, **kw)
            check(load().sptrsv_rewrite(C.byref(matrix.csr), levels.h, C.byref(s), C.byref(h), _stream()))
            del keep
        self.h = h
        self.matrix = matrix
        self.dtype = matrix.dtype
        self.refresh()

    def refresh(self):
        inf = SystemInfo()
        check(load().sptrsv_system_info_get(self.h, C.byref(inf)))
        self.info = {f: (list(v) if isinstance(v, C.Array) else v)
                     for f, v in ((f, getattr(inf, f)) for f, _ in SystemInfo._fields_)}
        self.n, self.m = inf.n, inf.m
        return self.info

    def run_width(self) -> int:
        return int(self.refresh()["run_width"])

    def tune(self, block=0, run_width=0, lanes_per_row=0):
        check(load().sptrsv_system_tune(self.h, block, run_width, lanes_per_row))

    def tune_cluster(self, cluster=-1, cluster_rows=-1, tiles=-1, shared_x=-1):
        """CTAs per cluster for mid-width levels (0 automatic, 1 none), the widest such level,
        whether wide levels may stream through shared-memory tiles (0 automatic, 1 never), and
        whether cluster levels read the previous level's x from the cluster's shared memory
        (0 automatic, 1 never).  -1 keeps a setting."""
        check(load().sptrsv_system_tune_cluster(self.h, cluster, cluster_rows, tiles, shared_x))

    def autotune(self, nrhs=1) -> float:
        """Times candidate schedules and keeps the fastest; returns its time in us."""
        us = C.c_double(0)
        check(load().sptrsv_system_autotune(self.h, nrhs, C.byref(us), _stream()))
        self.refresh()
        return us.value

    def reverse_rows(self):
        """Re-index a system built from upper_to_lower(U) so that it solves U x = b."""
        check(load().sptrsv_system_reverse_rows(self.h, _stream()))
        return self

    def debug_set_wait(self, withhold_segment=-1, timeout_ns=0):
        check(load().sptrsv_debug_set_wait(self.h, withhold_segment, timeout_ns))

    def solve(self, b, x=None, stamps=None, check_status=False):
        """b: device tensor of shape (n,) or (nrhs, n) (column-major n x nrhs, ld = n)."""
        torch = _torch()
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        if x is None:
            x = torch.empty_like(b)
        if stamps is None:
            check(load().sptrsv_solve(self.h, _ptr(b), _ptr(x), nrhs, self.n, _stream()))
        else:
            check(load().sptrsv_solve_timed(self.h, _ptr(b), _ptr(x), nrhs, self.n, _ptr(stamps), _stream()))
        if check_status:
            self.status()
        return x

    def solve_noalloc(self, b, x):
        """The solve that allocates nothing (x preallocated; schedule prepared by solve())."""
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        check(load().sptrsv_solve_noalloc(self.h, _ptr(b), _ptr(x), nrhs, self.n, _stream()))
        return x

    def status(self):
        check(load().sptrsv_solve_status(self.h, _stream()))

    def export(self) -> dict:
        torch = _torch()
        self.refresh()
        dev = self.matrix.rowptr.device
        n, nc, ne = self.n, self.info["nnz_c"], self.info["nnz_e"]
        vt = torch.float64 if self.dtype == F64 else torch.float32
        target = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        level = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        cptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        ccol = torch.empty(max(nc, 1), dtype=torch.int32, device=dev)
        cval = torch.empty(max(nc, 1), dtype=vt, device=dev)
        dinv = torch.empty(max(n, 1), dtype=vt, device=dev)
        eptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        ecol = torch.empty(max(ne, 1), dtype=torch.int32, device=dev)
        evl = torch.empty(max(ne, 1), dtype=vt, device=dev)
        check(load().sptrsv_system_export(self.h, _ptr(target), _ptr(level), _ptr(cptr), _ptr(ccol), _ptr(cval),
                                          _ptr(dinv), _ptr(eptr), _ptr(ecol), _ptr(evl), _stream()))
        out = {"target": target[:n], "level": level[:n], "cptr": cptr, "ccol": ccol[:nc], "cval": cval[:nc],
               "dinv": dinv[:n], "eptr": eptr, "ecol": ecol[:ne], "eval": evl[:ne]}
        return {k: v.cpu().numpy() for k, v in out.items()}

    def close(self):
        if getattr(self, "h", None):
            load().sptrsv_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many systems solved in one graph-captured persistent launch."""

    def __init__(self, systems, nrhs):
        nrhs = [int(r) for r in nrhs]
        assert len(systems) == len(nrhs) and systems
        self.systems = list(systems)
        self.nrhs = nrhs
        arr = (C.c_void_p * len(systems))(*[s.h.value if isinstance(s.h, C.c_void_p) else s.h for s in systems])
        nr = (C.c_int32 * len(systems))(*nrhs)
        h = C.c_void_p()
        check(load().sptrsv_batch_create(arr, nr, len(systems), C.byref(h), _stream()))
        self.h = h
        inf = BatchInfo()
        check(load().sptrsv_batch_info_get(h, C.byref(inf)))
        self.info = {f: getattr(inf, f) for f, _ in BatchInfo._fields_}

    def solve(self, bs, xs=None):
        """bs: list of device tensors (nrhs_i, n_i) in each system's value type."""
        torch = _torch()
        if xs is None:
            xs = [torch.empty_like(b) for b in bs]
        n = len(self.systems)
        barr = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
        xarr = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        check(load().sptrsv_batch_solve(self.h, barr, xarr, _stream()))
        return xs

    def close(self):
        if getattr(self, "h", None):
            load().sptrsv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Picker:
    """The learned rewrite picker (MLP 12 -> 64 -> 64 -> 64 -> 1, bfloat16 weights)."""

    def __init__(self, seed: int = 0):
        h = C.c_void_p()
        check(load().sptrsv_picker_create(C.c_uint64(seed), C.byref(h)))
        self.h = h

    @classmethod
    def load(cls, path: str) -> "Picker":
        pk = cls(0)
        check(load().sptrsv_picker_load(pk.h, path.encode()))
        return pk

    def save(self, path: str):
        check(load().sptrsv_picker_save(self.h, path.encode()))

    def get_params(self) -> np.ndarray:
        out = np.empty(PICKER_PARAMS, dtype=np.float32)
        check(load().sptrsv_picker_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == PICKER_PARAMS
        check(load().sptrsv_picker_set_params(self.h, a.ctypes.data_as(C.c_void_p)))

    def set_norm(self, mean, std, target_scale=1.0):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(std, dtype=np.float32)
        check(load().sptrsv_picker_set_norm(self.h, m.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p),
                                            C.c_float(target_scale)))

    def infer(self, feat, bf16=True):
        torch = _torch()
        n = feat.shape[0]
        out = torch.empty(max(n, 1), dtype=torch.float32, device=feat.device)
        check(load().sptrsv_picker_infer(self.h, _ptr(feat), n, _ptr(out), 1 if bf16 else 0, _stream()))
        return out[:n]

    def grad(self, feat, target, bf16=True):
        torch = _torch()
        g = torch.empty(PICKER_PARAMS, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        check(load().sptrsv_picker_grad(self.h, _ptr(feat), _ptr(target), feat.shape[0], 1 if bf16 else 0, _ptr(g),
                                        _ptr(loss), _stream()))
        return g, loss

    def train_step(self, feat, target, lr):
        torch = _torch()
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        check(load().sptrsv_picker_train_step(self.h, _ptr(feat), _ptr(target), feat.shape[0], C.c_float(lr),
                                              _ptr(loss), _stream()))
        return loss

    def close(self):
        if getattr(self, "h", None):
            load().sptrsv_picker_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# candidates of the learned strategy: fixed depths, and row budgets as negative entries (a target
# takes the following levels while it holds at most r rows)
DEFAULT_DEPTHS = (1, 2, 4, 8, 16, 32, -16, -32, -64)


def features(matrix: Matrix, levels: Levels, depths=DEFAULT_DEPTHS):
    """Device tensor (m * len(depths), 12) of candidate features, row t * len(depths) + d."""
    torch = _torch()
    d = np.ascontiguousarray(depths, dtype=np.int32)
    out = torch.empty((max(levels.m * d.size, 1), PICKER_FEATURES), dtype=torch.float32,
                      device=matrix.rowptr.device)
    check(load().sptrsv_picker_features(C.byref(matrix.csr), levels.h, d.ctypes.data_as(C.c_void_p), d.size,
                                        _ptr(out), _stream()))
    return out[:levels.m * d.size]


def run_blocks(level_ptr, cptr, nrhs=1, lanes_per_row=1, value_bytes=8):
    """The host block cutter of the single-CTA executor (test hook): returns (blocks int32[k, 4],
    geometry {stage_rows, stage_entries, ring_rows, fast_records})."""
    lp = np.ascontiguousarray(level_ptr, dtype=np.int32)
    cp = np.ascontiguousarray(cptr, dtype=np.int32)
    geo = np.zeros(4, np.int32)
    cnt = C.c_int64(0)
    cap = max(16, lp.size)
    while True:
        out = np.zeros((cap, 4), np.int32)
        rc = load().sptrsv_debug_run_blocks(lp.ctypes.data, lp.size - 1, cp.ctypes.data, nrhs, lanes_per_row,
                                            value_bytes, out.ctypes.data, cap, C.byref(cnt), geo.ctypes.data)
        if rc == ERR_INVALID and cnt.value > cap:
            cap = cnt.value
            continue
        check(rc)
        break
    g = dict(zip(("stage_rows", "stage_entries", "ring_rows", "fast_records"), (int(v) for v in geo)))
    return out[:cnt.value].copy(), g
