"""Thin ctypes binding of the C ABI in ``include/basker.h``.

Argument marshalling only: every step of the factorization and solve runs in the
CUDA library ``libbasker_gb300.so``.  PyTorch supplies device memory and the
current stream.  If the library is missing or cannot load, calls raise; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_BTF", 3: "BAD_ND", 4: "SINGULAR", 5: "NAN", 6: "OOM",
          7: "TIMEOUT", 8: "CUDA", 9: "NOT_FACTORED"}


class BaskerError(RuntimeError):
    def __init__(self, status: int, where: str, column: int = -1):
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.column = column
        msg = f"{where}: {self.name}"
        if column >= 0:
            msg += f" (column {column})"
        super().__init__(msg)


class Options(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("slack", ctypes.c_double),
                ("wait_budget_cycles", ctypes.c_longlong), ("factor_mode", ctypes.c_int),
                ("timing", ctypes.c_int), ("precision", ctypes.c_int), ("ir_max_iter", ctypes.c_int),
                ("ir_tol", ctypes.c_double), ("growth_limit", ctypes.c_double), ("refactor_switch", ctypes.c_int),
                ("graphs", ctypes.c_int), ("symbolic_mode", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("nd_block", ctypes.c_int32),
                ("nd_leaves", ctypes.c_int32), ("nnz_a", ctypes.c_int64), ("nnz_l", ctypes.c_int64),
                ("nnz_u", ctypes.c_int64), ("nnz_l_sym", ctypes.c_int64), ("nnz_u_sym", ctypes.c_int64),
                ("flops", ctypes.c_double), ("failed_column", ctypes.c_int32),
                ("last_repivot_columns", ctypes.c_int32), ("off_diagonal_pivots", ctypes.c_int32),
                ("capacity_regrows", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("gp_launches", ctypes.c_int32), ("static_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("kernel_ms", ctypes.c_double * 10),
                ("internal_site", ctypes.c_int32), ("internal_col", ctypes.c_int32),
                ("last_rounds", ctypes.c_int32), ("ir_iterations", ctypes.c_int32),
                ("ir_fallbacks", ctypes.c_int32), ("precision_used", ctypes.c_int32),
                ("tuned_static_blocks", ctypes.c_int32), ("tuned_solve_blocks", ctypes.c_int32),
                ("ir_eta", ctypes.c_double), ("growth", ctypes.c_double),
                ("kernel_calls", ctypes.c_int32 * 10), ("cuda_error", ctypes.c_int32),
                ("cuda_line", ctypes.c_int32),
                ("rounds_columns", ctypes.c_int64), ("full_refactors", ctypes.c_int32), ("graph_launches", ctypes.c_int32),
                ("static_factors", ctypes.c_int32), ("pad1", ctypes.c_int32)]

KERNEL_KINDS = ["gather", "static_refactor", "dag_levels", "gp_in_node", "gp_descendant", "solve",
                "dense_node", "refactor_rounds", "rows_transpose", "refine"]


EXPORTED = ["basker_default_options", "basker_symbolic", "basker_factor", "basker_refactor",
            "basker_solve", "basker_refactor_solve_host", "basker_info", "basker_export",
            "basker_free", "basker_strerror", "basker_solve_noalloc", "basker_autotune",
            "basker_symbolic_counts", "basker_probe_latency"]


def library_path() -> str:
    return _build.library_path()


def load(path: Optional[str] = None):
    """Load the CUDA library (built in-tree by ``build()``); raise if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or library_path()
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
        L = ctypes.CDLL(p)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.basker_default_options.argtypes = [ctypes.POINTER(Options)]
        L.basker_default_options.restype = None
        L.basker_symbolic.argtypes = [i32, vp, vp, vp, vp, i32, vp, i32, i32, vp, ctypes.POINTER(Options),
                                      ctypes.POINTER(vp)]
        L.basker_symbolic.restype = ctypes.c_int
        for f in ("basker_factor", "basker_refactor"):
            getattr(L, f).argtypes = [vp, vp, vp]
            getattr(L, f).restype = ctypes.c_int
        L.basker_solve.argtypes = [vp, i32, vp, i32, vp, i32, vp]
        L.basker_solve.restype = ctypes.c_int
        L.basker_autotune.argtypes = [vp, vp, vp, vp]
        L.basker_autotune.restype = ctypes.c_int
        L.basker_solve_noalloc.argtypes = [vp, i32, vp, i32, vp, i32, vp]
        L.basker_solve_noalloc.restype = ctypes.c_int
        L.basker_refactor_solve_host.argtypes = [vp, vp, i32, vp, vp, vp]
        L.basker_refactor_solve_host.restype = ctypes.c_int
        L.basker_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.basker_info.restype = ctypes.c_int
        L.basker_export.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.basker_export.restype = ctypes.c_int
        L.basker_free.argtypes = [vp]
        L.basker_free.restype = None
        L.basker_strerror.argtypes = [ctypes.c_int]
        L.basker_strerror.restype = ctypes.c_char_p
        L.basker_symbolic_counts.argtypes = [i32, vp, vp, vp, vp, i32, vp, i32, i32, vp, ctypes.c_int, vp, vp]
        L.basker_symbolic_counts.restype = ctypes.c_int
        L.basker_probe_latency.argtypes = [vp]
        L.basker_probe_latency.restype = ctypes.c_int
        _lib = L
        return L


def symbolic_counts(prob, mode: int = 0):
    """basker_symbolic_counts on the host: per-column L and U counts of a problem's
    pattern (mode 0: structural pass under the natural pivots; 1: Algorithm 3's
    elimination-tree counts).  Needs no GPU."""
    L = load()
    arrs = [_i32(prob.colptr), _i32(prob.rowind), _i32(prob.P), _i32(prob.Q), _i32(prob.block_ptr),
            _i32(prob.nd_node_ptr if prob.nd_block >= 0 else [0])]
    n = int(prob.n)
    lc = np.zeros(max(n, 1), np.int32)
    uc = np.zeros(max(n, 1), np.int32)
    s = L.basker_symbolic_counts(n, *[_np_ptr(a) for a in arrs[:4]], len(arrs[4]) - 1, _np_ptr(arrs[4]),
                                 int(prob.nd_block), int(prob.nd_leaves), _np_ptr(arrs[5]), int(mode),
                                 _np_ptr(lc), _np_ptr(uc))
    if s != 0:
        raise BaskerError(s, "basker_symbolic_counts")
    return lc[:n], uc[:n]


def probe_latency() -> dict:
    """basker_probe_latency on the current device: ns of one flag handoff between
    two blocks, one dependent FP64 fma, one dependent FP64 division."""
    L = load()
    out = (ctypes.c_double * 3)()
    s = L.basker_probe_latency(ctypes.cast(out, ctypes.c_void_p))
    if s != 0:
        raise BaskerError(s, "basker_probe_latency")
    return {"flag_handoff_ns": out[0], "dfma_ns": out[1], "ddiv_ns": out[2]}


def default_options() -> Options:
    o = Options()
    load().basker_default_options(ctypes.byref(o))
    return o


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _stream_ptr(stream) -> ctypes.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dev_ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(int(t.data_ptr()))


class Handle:
    """One analysed pattern (``basker_symbolic``) and its factors on the device."""

    def __init__(self, n, colptr, rowind, P, Q, block_ptr, nd_block=-1, nd_leaves=0, nd_node_ptr=None,
                 tau: float = 1e-3, slack: Optional[float] = None, wait_budget_cycles: Optional[int] = None,
                 factor_mode: int = 0, timing: bool = False, precision: int = 0,
                 ir_max_iter: Optional[int] = None, ir_tol: Optional[float] = None,
                 growth_limit: Optional[float] = None, refactor_switch: Optional[int] = None,
                 graphs: Optional[bool] = None, symbolic_mode: Optional[int] = None):
        self.lib = load()
        opt = default_options()
        if symbolic_mode is not None:
            opt.symbolic_mode = int(symbolic_mode)
        if graphs is not None:
            opt.graphs = 1 if graphs else 0
        if refactor_switch is not None:
            opt.refactor_switch = int(refactor_switch)
        opt.tau = float(tau)
        opt.precision = int(precision)
        if ir_max_iter is not None:
            opt.ir_max_iter = int(ir_max_iter)
        if ir_tol is not None:
            opt.ir_tol = float(ir_tol)
        if growth_limit is not None:
            opt.growth_limit = float(growth_limit)
        if slack is not None:
            opt.slack = float(slack)
        if wait_budget_cycles is not None:
            opt.wait_budget_cycles = int(wait_budget_cycles)
        opt.factor_mode = int(factor_mode)
        opt.timing = 1 if timing else 0
        self.n = int(n)
        arrs = [_i32(colptr), _i32(rowind), _i32(P), _i32(Q), _i32(block_ptr),
                _i32(nd_node_ptr if (nd_node_ptr is not None and nd_block >= 0) else [0])]
        self.nnz = int(arrs[0][-1]) if len(arrs[0]) else 0
        self.nblocks = len(arrs[4]) - 1
        h = ctypes.c_void_p()
        s = self.lib.basker_symbolic(self.n, *[_np_ptr(a) for a in arrs[:4]], self.nblocks, _np_ptr(arrs[4]),
                                     int(nd_block), int(nd_leaves), _np_ptr(arrs[5]), ctypes.byref(opt),
                                     ctypes.byref(h))
        if s != 0:
            raise BaskerError(s, "basker_symbolic")
        self.h = h
        self._dev_index = None
        try:
            import torch
            if torch.cuda.is_available():
                self._dev_index = torch.cuda.current_device()
        except Exception:
            pass

    @classmethod
    def from_problem(cls, prob, **kw) -> "Handle":
        return cls(prob.n, prob.colptr, prob.rowind, prob.P, prob.Q, prob.block_ptr, prob.nd_block,
                   prob.nd_leaves, prob.nd_node_ptr, **kw)

    def _check(self, s: int, where: str):
        if s != 0:
            inf = self.info()
            col = inf["failed_column"] if s in (4, 5) else -1
            err = BaskerError(s, where, col)
            if inf["internal_site"]:
                err.args = (err.args[0] + f" [internal check {inf['internal_site']} at column {inf['internal_col']}]",)
            if s == 8 and inf["cuda_error"]:
                err.args = (err.args[0] + f" [cuda error {inf['cuda_error']} at api.cu:{inf['cuda_line']}]",)
            raise err

    def factor(self, values, stream=None) -> None:
        """values: CUDA float64 tensor of nnz(A) entries in A's CSC order."""
        self._check(self.lib.basker_factor(self.h, _dev_ptr(values), _stream_ptr(stream)), "basker_factor")

    def refactor(self, values, stream=None) -> None:
        self._check(self.lib.basker_refactor(self.h, _dev_ptr(values), _stream_ptr(stream)), "basker_refactor")

    def solve(self, b, x=None, stream=None):
        """b: CUDA float64 (n,) or (n, nrhs).  Returns x of the same shape."""
        import torch
        if b.dim() == 1:
            bt = b.contiguous().view(1, -1)
        else:
            bt = b.t().contiguous()            # (nrhs, n) row-major = column-major n x nrhs
        nrhs = bt.shape[0]
        xt = torch.empty_like(bt)
        s = self.lib.basker_solve(self.h, nrhs, _dev_ptr(bt), self.n, _dev_ptr(xt), self.n, _stream_ptr(stream))
        self._check(s, "basker_solve")
        out = xt.view(-1) if b.dim() == 1 else xt.t()
        if x is not None:
            x.copy_(out)
            return x
        return out

    def solve_noalloc(self, b, x):
        """basker_solve_noalloc: like solve(), for callers that cannot allocate
        device memory; b and x are CUDA float64 (n,) or column-major (n, nrhs)
        buffers the caller owns (x is written in place)."""
        import torch
        for nm, t in (("b", b), ("x", x)):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float64:
                raise ValueError(f"{nm} must be a float64 tensor")
            if not t.is_cuda or t.device.index != self.device_index():
                raise ValueError(f"{nm} must live on the handle's device (cuda:{self.device_index()})")
            if t.dim() not in (1, 2) or t.shape[0] != self.n:
                raise ValueError(f"{nm} must have shape (n,) or (n, nrhs) with n = {self.n}")
        if b.dim() != x.dim() or tuple(b.shape) != tuple(x.shape):
            raise ValueError("b and x must have the same shape")
        nrhs = 1 if b.dim() == 1 else b.shape[1]

        def lead(t):
            if t.dim() == 1 or t.shape[1] == 1:
                if t.dim() == 2 and t.stride(0) != 1:
                    raise ValueError("b and x must be column-major (n, nrhs) views")
                return self.n
            if not (t.stride(0) == 1 and t.stride(1) >= self.n):
                raise ValueError("b and x must be column-major (n, nrhs) views")
            return t.stride(1)
        ldb, ldx = lead(b), lead(x)
        s = self.lib.basker_solve_noalloc(self.h, nrhs, _dev_ptr(b), ldb, _dev_ptr(x), ldx, _stream_ptr(None))
        self._check(s, "basker_solve_noalloc")
        return x

    def device_index(self) -> int:
        """CUDA device the handle's memory lives on (current at basker_symbolic)."""
        if getattr(self, "_dev_index", None) is None:
            import torch
            self._dev_index = torch.cuda.current_device()
        return self._dev_index

    def autotune(self, values, b, stream=None) -> dict:
        """basker_autotune: values and b CUDA float64 tensors (nnz(A), n).  Returns the
        chosen launch sizes."""
        self._check(self.lib.basker_autotune(self.h, _dev_ptr(values), _dev_ptr(b), _stream_ptr(stream)),
                    "basker_autotune")
        inf = self.info()
        return {"static_blocks": inf["tuned_static_blocks"], "solve_blocks": inf["tuned_solve_blocks"]}

    def refactor_solve_host(self, values: np.ndarray, b: np.ndarray, stream=None) -> np.ndarray:
        """Host arrays in, host solution out (copies inside the call)."""
        v = np.ascontiguousarray(values, np.float64)
        b2 = np.asfortranarray(b.reshape(self.n, -1), np.float64)
        x = np.empty_like(b2, order="F")
        s = self.lib.basker_refactor_solve_host(self.h, _np_ptr(v), b2.shape[1], _np_ptr(b2), _np_ptr(x),
                                                _stream_ptr(stream))
        self._check(s, "basker_refactor_solve_host")
        return x.reshape(b.shape)

    def info(self) -> dict:
        inf = Info()
        s = self.lib.basker_info(self.h, ctypes.byref(inf))
        if s != 0:
            raise BaskerError(s, "basker_info")
        out = {k: getattr(inf, k) for k, _ in Info._fields_ if k not in ("reserved", "pad1", "kernel_ms",
                                                                          "kernel_calls")}
        out["kernel_calls"] = {KERNEL_KINDS[i]: inf.kernel_calls[i] for i in range(len(KERNEL_KINDS))}
        out["kernel_ms"] = {KERNEL_KINDS[i]: inf.kernel_ms[i] for i in range(len(KERNEL_KINDS))}
        return out

    def export(self):
        """(prow, L, U) as host scipy CSC matrices in B's coordinates (steps as rows)."""
        import scipy.sparse as sp
        nl, nu = ctypes.c_int64(), ctypes.c_int64()
        s = self.lib.basker_export(self.h, None, None, None, None, None, None, None, ctypes.byref(nl),
                                   ctypes.byref(nu))
        self._check(s, "basker_export")
        n = self.n
        prow = np.empty(n, np.int32)
        Lp, Up = np.empty(n + 1, np.int64), np.empty(n + 1, np.int64)
        Li, Lx = np.empty(max(nl.value, 1), np.int32), np.empty(max(nl.value, 1), np.float64)
        Ui, Ux = np.empty(max(nu.value, 1), np.int32), np.empty(max(nu.value, 1), np.float64)
        s = self.lib.basker_export(self.h, _np_ptr(prow), _np_ptr(Lp), _np_ptr(Li), _np_ptr(Lx), _np_ptr(Up),
                                   _np_ptr(Ui), _np_ptr(Ux), ctypes.byref(nl), ctypes.byref(nu))
        self._check(s, "basker_export")
        L = sp.csc_matrix((Lx[:nl.value], Li[:nl.value], Lp), shape=(n, n))
        U = sp.csc_matrix((Ux[:nu.value], Ui[:nu.value], Up), shape=(n, n))
        return prow, L, U

    def free(self) -> None:
        h = getattr(self, "h", None)
        if h:
            self.lib.basker_free(h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
