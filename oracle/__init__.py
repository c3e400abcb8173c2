"""The oracle: plain serial CPU FP64 reference of the numeric sparse LU.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library and the library never calls it.

``basker_oracle.c`` holds the arithmetic (Algorithm 1 per column over the BTF
diagonal blocks, pivots confined to the ND node, Sec. II-III); this module only
compiles it with gcc and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "basker_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbasker_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "INVALID", 2: "NOT_BTF", 3: "BAD_ND", 4: "SINGULAR", 5: "NAN", 6: "NOMEM"}
ORDER = {"ascending": 0, "dfs": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, ip, dp = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
        lib.oracle_analyze.restype = vp
        lib.oracle_analyze.argtypes = [ctypes.c_int, ip, ip, ip, ip, ctypes.c_int, ip,
                                       ctypes.c_int, ctypes.c_int, ip]
        lib.oracle_factor.restype = ctypes.c_int
        lib.oracle_factor.argtypes = [vp, dp, ctypes.c_double, ip, ctypes.c_int]
        lib.oracle_status.restype = ctypes.c_int
        lib.oracle_status.argtypes = [vp, ip]
        lib.oracle_sizes.argtypes = [vp, ip, ip]
        lib.oracle_export.restype = ctypes.c_int
        lib.oracle_export.argtypes = [vp, ip, ip, ip, dp, ip, ip, dp]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
        lib.oracle_bsizes.argtypes = [vp, ip]
        lib.oracle_bexport.argtypes = [vp, ip, ip, dp]
        lib.oracle_free.argtypes = [vp]
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclasses.dataclass
class Factors:
    """LU of the diagonal blocks of B = A(P,Q), in B's coordinates.

    ``prow[k]`` is the B row pivoted at step k; ``L`` (unit diagonal not stored) and
    ``U`` (diagonal stored) are scipy CSC matrices whose row indices are pivot steps,
    so that ``B[prow][:, :]`` restricted to the diagonal blocks equals ``(I + L) U``.
    """
    prow: np.ndarray
    L: "object"
    U: "object"


class OracleLU:
    """One analysed pattern (``oracle_analyze``) and its latest factorization."""

    def __init__(self, prob):
        self.lib = _load()
        self.prob = prob
        self.n = int(prob.n)
        self._keep = [_i32(prob.colptr), _i32(prob.rowind), _i32(prob.P), _i32(prob.Q),
                      _i32(prob.block_ptr), _i32(prob.nd_node_ptr if prob.nd_block >= 0 else [0])]
        Ap, Ai, P, Q, bp, ndp = self._keep
        self.h = self.lib.oracle_analyze(self.n, _ptr(Ap), _ptr(Ai), _ptr(P), _ptr(Q),
                                         int(prob.nblocks), _ptr(bp), int(prob.nd_block),
                                         int(prob.nd_leaves), _ptr(ndp))
        if not self.h:
            raise MemoryError("oracle_analyze")
        self.status, self.info_col = self._status()

    def _status(self):
        col = ctypes.c_int(-1)
        s = self.lib.oracle_status(self.h, ctypes.byref(col))
        return STATUS.get(s, str(s)), col.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_free(h)
            self.h = None

    def factor(self, values: Optional[np.ndarray] = None, tau: float = 1e-3,
               pref: Optional[np.ndarray] = None, order: str = "ascending") -> str:
        """Numeric factorization; ``pref`` = B rows preferred as pivots (refactor)."""
        v = np.ascontiguousarray(self.prob.values if values is None else values, np.float64)
        pr = None if pref is None else _i32(pref)
        self.lib.oracle_factor(self.h, _ptr(v), float(tau), _ptr(pr), ORDER[order])
        self.status, self.info_col = self._status()
        return self.status

    def refactor(self, values: np.ndarray, prev: Factors, tau: float = 1e-3) -> str:
        """Same pattern, new values, previous pivots preferred."""
        return self.factor(values, tau=tau, pref=prev.prow)

    def factors(self) -> Factors:
        import scipy.sparse as sp
        if self.status != "OK":
            raise RuntimeError(f"oracle status {self.status} (column {self.info_col})")
        lnz, unz = ctypes.c_int64(), ctypes.c_int64()
        self.lib.oracle_sizes(self.h, ctypes.byref(lnz), ctypes.byref(unz))
        n = self.n
        prow = np.empty(n, np.int32)
        Lp = np.empty(n + 1, np.int64)
        Up = np.empty(n + 1, np.int64)
        Li = np.empty(max(lnz.value, 1), np.int32)
        Lx = np.empty(max(lnz.value, 1), np.float64)
        Ui = np.empty(max(unz.value, 1), np.int32)
        Ux = np.empty(max(unz.value, 1), np.float64)
        self.lib.oracle_export(self.h, _ptr(prow), _ptr(Lp), _ptr(Li), _ptr(Lx), _ptr(Up),
                               _ptr(Ui), _ptr(Ux))
        L = sp.csc_matrix((Lx[:lnz.value], Li[:lnz.value], Lp), shape=(n, n))
        U = sp.csc_matrix((Ux[:unz.value], Ui[:unz.value], Up), shape=(n, n))
        return Factors(prow=prow, L=L, U=U)

    def B(self):
        """B = A(P,Q) with the values of the latest factorization."""
        import scipy.sparse as sp
        nnz = ctypes.c_int64()
        self.lib.oracle_bsizes(self.h, ctypes.byref(nnz))
        Bp = np.empty(self.n + 1, np.int64)
        Bi = np.empty(max(nnz.value, 1), np.int32)
        Bx = np.empty(max(nnz.value, 1), np.float64)
        self.lib.oracle_bexport(self.h, _ptr(Bp), _ptr(Bi), _ptr(Bx))
        return sp.csc_matrix((Bx[:nnz.value], Bi[:nnz.value], Bp), shape=(self.n, self.n))

    def solve(self, b: np.ndarray) -> np.ndarray:
        """x = A^{-1} b; ``b`` is (n,) or (n, nrhs)."""
        b2 = np.asfortranarray(b.reshape(self.n, -1), np.float64)
        x = np.zeros_like(b2, order="F")
        s = self.lib.oracle_solve(self.h, b2.shape[1], _ptr(b2), self.n, _ptr(x), self.n)
        if s != 0:
            raise RuntimeError(f"oracle_solve: {STATUS.get(s, s)}")
        return x.reshape(b.shape)
