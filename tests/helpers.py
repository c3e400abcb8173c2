"""Test-side helpers: independent references written from textbook definitions.

Nothing here calls the CUDA library; the dense eliminations below are the
textbook right-looking Gaussian elimination (a different algorithm from the
left-looking Gilbert-Peierls method under test).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import scipy.sparse as sp


def block_of(block_ptr: np.ndarray, n: int) -> np.ndarray:
    return np.repeat(np.arange(len(block_ptr) - 1), np.diff(block_ptr))


def diag_blocks(B: sp.csc_matrix, block_ptr: np.ndarray) -> sp.csc_matrix:
    """The block-diagonal part of B (the part that is factored)."""
    blk = block_of(block_ptr, B.shape[0])
    C = B.tocoo()
    m = blk[C.row] == blk[C.col]
    return sp.csc_matrix((C.data[m], (C.row[m], C.col[m])), shape=B.shape)


def candidate_range(prob, c: int):
    """Rows a pivot of column c may come from: its BTF block, or its ND node."""
    bp = prob.block_ptr
    d = int(np.searchsorted(bp, c, side="right") - 1)
    if d == prob.nd_block:
        ptr = prob.nd_node_ptr
        t = int(np.searchsorted(ptr, c, side="right") - 1)
        return int(ptr[t]), int(ptr[t + 1])
    return int(bp[d]), int(bp[d + 1])


def dense_threshold_lu(M: np.ndarray, tau: float, ranges, pref=None):
    """Textbook right-looking elimination with threshold partial pivoting.

    ``ranges[k]`` = (lo, hi): rows column k may take its pivot from.  The
    preferred row (``pref[k]`` or k) is kept if |a| >= tau * max, else the lowest
    row index holding the maximum.  Returns (prow, L, U) with P M = L U,
    ``prow[k]`` the original row pivoted at step k.
    """
    n = M.shape[0]
    A = M.astype(float).copy()
    rows = np.arange(n)            # rows[i] = original row now at position i
    for k in range(n):
        lo, hi = ranges[k]
        cand = [i for i in range(k, n) if lo <= rows[i] < hi]
        vals = np.abs(A[cand, k])
        m = vals.max()
        pr = k if pref is None else pref[k]
        pos = {rows[i]: i for i in cand}
        if pr in pos and abs(A[pos[pr], k]) >= tau * m:
            i = pos[pr]
        else:
            best = min(rows[i] for i in cand if abs(A[i, k]) == m)
            i = pos[best]
        A[[k, i]] = A[[i, k]]
        rows[[k, i]] = rows[[i, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    L = np.tril(A, -1)
    U = np.triu(A)
    return rows, L, U


def exact_lu(M, ranges=None):
    """Exact rational LU without row exchanges (diagonal pivots), Fractions."""
    n = len(M)
    A = [[Fraction(v) for v in row] for row in M]
    for k in range(n):
        for i in range(k + 1, n):
            if A[i][k] != 0:
                f = A[i][k] / A[k][k]
                A[i][k] = f
                for j in range(k + 1, n):
                    A[i][j] -= f * A[k][j]
    return A


def boolean_fill(S: np.ndarray) -> np.ndarray:
    """Structural LU of a boolean matrix without exchanges (fill-path theorem)."""
    M = S.astype(bool).copy()
    n = M.shape[0]
    for k in range(n):
        rows = np.flatnonzero(M[k + 1:, k]) + k + 1
        cols = np.flatnonzero(M[k, k + 1:]) + k + 1
        if rows.size and cols.size:
            M[np.ix_(rows, cols)] = True
    return M


def factor_backward_error(Bd: sp.csc_matrix, f) -> float:
    """|| P B_diag - (I+L) U ||_1 / || B ||_1 (column sums)."""
    n = Bd.shape[0]
    LU = (sp.identity(n, format="csc") + f.L) @ f.U
    R = Bd[f.prow, :] - LU
    num = np.abs(R).sum(axis=0).max() if R.nnz else 0.0
    return float(num / max(np.abs(Bd).sum(axis=0).max(), 1e-300))


def solve_backward_error(A: sp.csc_matrix, x: np.ndarray, b: np.ndarray) -> float:
    """eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) per right-hand side (max)."""
    x2 = x.reshape(A.shape[0], -1)
    b2 = b.reshape(A.shape[0], -1)
    r = b2 - A @ x2
    anorm = np.abs(A).sum(axis=1).max()
    eta = np.abs(r).max(axis=0) / (anorm * np.abs(x2).max(axis=0) + np.abs(b2).max(axis=0))
    return float(eta.max())


def forward_error(x: np.ndarray, xo: np.ndarray) -> float:
    """max over right-hand sides of ||x - xo||_inf / ||xo||_inf."""
    x2 = np.asarray(x).reshape(len(x), -1)
    o2 = np.asarray(xo).reshape(len(xo), -1)
    return float((np.abs(x2 - o2).max(axis=0) / np.abs(o2).max(axis=0)).max())


def oracle_solution(prob, values, b) -> np.ndarray:
    """The FP64 oracle's solution of A(values) x = b (a factorization from scratch)."""
    import oracle
    o = oracle.OracleLU(prob)
    assert o.factor(values) == "OK"
    return o.solve(b)


def kappa_inf_blocks(prob) -> float:
    """kappa_inf(A) of a block-diagonal B = A(P, Q): ||A||_inf times the largest
    ||B_d^-1||_inf over the diagonal blocks (dense inverses; small blocks)."""
    B = sp.csc_matrix((prob.values, (np.argsort(prob.P)[prob.rowind],
                                     np.argsort(prob.Q)[np.repeat(np.arange(prob.n), np.diff(prob.colptr))])),
                      shape=(prob.n, prob.n)).tocsr()
    bp = np.asarray(prob.block_ptr)
    inv = 0.0
    for d in range(len(bp) - 1):
        lo, hi = bp[d], bp[d + 1]
        Bd = B[lo:hi, lo:hi].toarray()
        inv = max(inv, float(np.abs(np.linalg.inv(Bd)).sum(axis=1).max()))
    return float(np.abs(B).sum(axis=1).max() * inv)


def kappa_inf(A: sp.csc_matrix) -> float:
    """kappa_inf(A) = ||A||_inf ||A^-1||_inf, the inverse's norm by the 1-norm
    estimate of A^-T (Hager-Higham, scipy's onenormest; small matrices)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(A.T.tocsc())
    inv_t = spla.LinearOperator(A.shape, matvec=lu.solve, rmatvec=lambda y: lu.solve(y, trans="T"),
                                dtype=np.float64)
    return float(np.abs(A).sum(axis=1).max() * spla.onenormest(inv_t))


def a_matrix(prob) -> sp.csc_matrix:
    return sp.csc_matrix((prob.values, prob.rowind, prob.colptr), shape=(prob.n, prob.n))


def flops(f) -> int:
    """sum_j l_j (2 u_j + 1): l_j below-diagonal entries of L(:,j), u_j right of the
    diagonal in U(j,:)."""
    lj = np.diff(f.L.indptr)
    uj = np.bincount(f.U.indices, minlength=f.U.shape[0]) - 1
    return int((lj * (2 * uj + 1)).sum())


def make_problem(Bmat, block_ptr=None, nd_block=-1, nd_leaves=0, nd_node_ptr=None,
                 scramble_seed=None, name="case"):
    """A Problem whose permuted matrix is exactly ``Bmat`` (A = B scrambled)."""
    from paper_1601_05725_gb300.inputs import Problem
    B = sp.csc_matrix(Bmat)
    n = B.shape[0]
    if scramble_seed is None:
        P = np.arange(n, dtype=np.int32)
        Q = np.arange(n, dtype=np.int32)
    else:
        rng = np.random.default_rng(scramble_seed)
        P = rng.permutation(n).astype(np.int32)
        Q = rng.permutation(n).astype(np.int32)
    C = B.tocoo()
    A = sp.csc_matrix((C.data, (P[C.row], Q[C.col])), shape=(n, n))
    A.sort_indices()
    bp = np.array([0, n] if block_ptr is None else block_ptr, np.int32)
    ndp = np.zeros(0, np.int32) if nd_node_ptr is None else np.asarray(nd_node_ptr, np.int32)
    return Problem(name=name, n=n, colptr=A.indptr.astype(np.int32),
                   rowind=A.indices.astype(np.int32), values=A.data.astype(np.float64),
                   P=P, Q=Q, block_ptr=bp, nd_block=nd_block, nd_leaves=nd_leaves,
                   nd_node_ptr=ndp, meta={"seed": 0})


def b_matrix(prob, values=None) -> sp.csc_matrix:
    """B = A(P,Q), formed with scipy indexing (independent of the code under test)."""
    v = prob.values if values is None else values
    A = sp.csc_matrix((v, prob.rowind, prob.colptr), shape=(prob.n, prob.n))
    return A[prob.P, :][:, prob.Q].tocsc()


def reference_block_lu(prob, tau, values=None, pref=None):
    """Textbook dense LU of every diagonal block of B with the library's pivot rule
    (candidates confined to the BTF block or ND node).  Returns (prow, L, U) dense
    over the whole matrix, L strictly lower and U upper in pivot-step rows."""
    B = b_matrix(prob, values).toarray()
    n = prob.n
    prow = np.zeros(n, np.int64)
    L = np.zeros((n, n))
    U = np.zeros((n, n))
    bp = prob.block_ptr
    for d in range(len(bp) - 1):
        k0, k1 = int(bp[d]), int(bp[d + 1])
        ranges = [tuple(v - k0 for v in candidate_range(prob, c)) for c in range(k0, k1)]
        pr = None if pref is None else [int(p) - k0 for p in pref[k0:k1]]
        rows, Lb, Ub = dense_threshold_lu(B[k0:k1, k0:k1], tau, ranges, pr)
        prow[k0:k1] = rows + k0
        L[k0:k1, k0:k1] = Lb
        U[k0:k1, k0:k1] = Ub
    return prow, L, U
