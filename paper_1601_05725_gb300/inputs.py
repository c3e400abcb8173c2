"""Seeded synthetic inputs for the sparse LU hot path, and the harness's own orderings.

This module builds matrices and permutations only; it holds none of the
factorization's arithmetic, so the CPU oracle and the CUDA path can both take
their inputs from it.

The paper's test suite (Table I, Sec. V-A) is made of circuit and power-grid
matrices that are not available here.  The generators below stand in for their
shape classes:

* ``netlist`` blocks: nodes on a ring (ring edges always present, which keeps the
  block strongly connected), extra links to ``i +- d`` with ``d`` log-uniform in
  ``[2, 64]`` (circuit locality), 5% of the non-ring links keep only one
  direction, off-diagonal conductances log-uniform in ``[1e-3, 1e3]`` with a
  random sign, diagonal = (row abs-sum) x U(0.5, 1.5).
* ``grid``: a five-point power-grid mesh, edge conductance ``g`` log-uniform in
  ``[1e-2, 1e2]``, ``a_ij = -g U(0.9,1.1)`` and ``a_ji = -g U(0.9,1.1)`` drawn
  independently, diagonal = row abs-sum + U(0, 1e-3).

Orderings (inputs of the method, Sec. III-A and III-C; the library does not
compute them): the block triangular form is built by construction, nested
dissection (ND) is geometric for the grid and by position bisection on the ring
for netlists ("cut the ring, the separator is one endpoint of every crossing
edge"), and each leaf is ordered by continued bisection of the same kind.

``B`` denotes the matrix in BTF + ND order.  The input ``A`` is ``B`` with its rows
and columns scrambled by random permutations; ``P`` and ``Q`` (new -> old) recover
it: ``B[i, j] = A[P[i], Q[j]]``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Problem", "config1", "config2", "config3", "small_problem", "grid_problem",
    "netlist_problem", "block_diagonal_problem", "refactor_values", "rhs_ones", "config4",
    "rhs_normal", "rail_links",
    "CONFIG_SEEDS",
]

CONFIG_SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}


@dataclasses.dataclass
class Problem:
    """One sparse system in the library's input form (CSC, 0-based, rows sorted)."""
    name: str
    n: int
    colptr: np.ndarray      # int32 [n+1]   pattern of A
    rowind: np.ndarray      # int32 [nnz]
    values: np.ndarray      # float64 [nnz] values of A in CSC order
    P: np.ndarray           # int32 [n] row permutation, new -> old
    Q: np.ndarray           # int32 [n] column permutation, new -> old
    block_ptr: np.ndarray   # int32 [nblocks+1] BTF block boundaries in B's numbering
    nd_block: int = -1      # index of the BTF block that carries the ND structure, -1 if none
    nd_leaves: int = 0      # number of ND leaves (power of two), 0 if none
    nd_node_ptr: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    @property
    def nblocks(self) -> int:
        return len(self.block_ptr) - 1

    def dense(self) -> np.ndarray:
        """Dense copy of A (small problems only)."""
        D = np.zeros((self.n, self.n))
        for j in range(self.n):
            s, e = self.colptr[j], self.colptr[j + 1]
            D[self.rowind[s:e], j] = self.values[s:e]
        return D

    def with_values(self, values: np.ndarray, name: Optional[str] = None) -> "Problem":
        return dataclasses.replace(self, values=np.ascontiguousarray(values, np.float64),
                                   name=name or self.name)


# ----------------------------------------------------------------------------------------
# elementary draws


def _log_uniform(rng: np.random.Generator, lo: float, hi: float, size) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _random_sign(rng: np.random.Generator, size) -> np.ndarray:
    return np.where(rng.random(size) < 0.5, -1.0, 1.0)


# ----------------------------------------------------------------------------------------
# netlist blocks


def netlist_pattern(rng: np.random.Generator, m: int, extra: Tuple[int, int] = (0, 1),
                    W: int = 64, drop: float = 0.05, nonlocal_links: bool = False
                    ) -> Tuple[np.ndarray, np.ndarray]:
    """Directed off-diagonal entries (rows, cols) of an m-node netlist block.

    Every node i initiates one ring link to i+1 (mod m) and U{extra} further links
    to i +- d, d log-uniform in [2, W] (``nonlocal_links`` draws uniform targets
    instead, a stress case with large separators).  Each undirected link is stored
    in both directions, except that 5% of the non-ring links lose one direction.
    """
    if m <= 1:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    i_ring = np.arange(m, dtype=np.int64)
    j_ring = (i_ring + 1) % m
    if m == 2:
        i_ring, j_ring = i_ring[:1], j_ring[:1]
    src = [i_ring]
    dst = [j_ring]
    if m >= 4 and extra[1] > 0:
        e = rng.integers(extra[0], extra[1] + 1, m)
        s = np.repeat(np.arange(m, dtype=np.int64), e)
        if nonlocal_links:
            t = rng.integers(0, m, s.size)
        else:
            dmax = max(2, min(W, m // 2))
            d = np.rint(_log_uniform(rng, 2.0, float(dmax), s.size)).astype(np.int64)
            t = (s + d * np.where(rng.random(s.size) < 0.5, -1, 1)) % m
        src.append(s)
        dst.append(t)
    s = np.concatenate(src)
    t = np.concatenate(dst)
    keep = s != t
    s, t = s[keep], t[keep]
    lo, hi = np.minimum(s, t), np.maximum(s, t)
    key = np.unique(lo * m + hi)
    lo, hi = key // m, key % m
    ring = (hi - lo == 1) | (hi - lo == m - 1)
    nonring = np.flatnonzero(~ring)
    dropped = nonring[rng.random(nonring.size) < drop]
    keep_fwd = np.ones(lo.size, bool)
    keep_bwd = np.ones(lo.size, bool)
    which = rng.random(dropped.size) < 0.5
    keep_fwd[dropped[which]] = False
    keep_bwd[dropped[~which]] = False
    rows = np.concatenate([lo[keep_fwd], hi[keep_bwd]])
    cols = np.concatenate([hi[keep_fwd], lo[keep_bwd]])
    return rows, cols


def netlist_values(rng: np.random.Generator, rows: np.ndarray, cols: np.ndarray, m: int,
                   diag_scale: Tuple[float, float] = (0.5, 1.5),
                   extra_rowabs: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Off-diagonal values (log-uniform 1e-3..1e3, random sign) and the diagonal.

    diagonal = (row abs-sum) x U(diag_scale); ``extra_rowabs`` adds the abs-sum of
    entries of the same rows that lie outside the block (coupling entries).
    """
    off = _log_uniform(rng, 1e-3, 1e3, rows.size) * _random_sign(rng, rows.size)
    rowabs = np.bincount(rows, weights=np.abs(off), minlength=m)
    if extra_rowabs is not None:
        rowabs = rowabs + extra_rowabs
    diag = rowabs * rng.uniform(diag_scale[0], diag_scale[1], m)
    empty = rowabs == 0
    if empty.any():
        diag[empty] = _log_uniform(rng, 1e-3, 1e3, int(empty.sum()))
    return off, diag


# ----------------------------------------------------------------------------------------
# orderings (harness side; inputs of the method)


def _sym_adjacency(m: int, rows: np.ndarray, cols: np.ndarray):
    import scipy.sparse as sp
    r = np.concatenate([rows, cols])
    c = np.concatenate([cols, rows])
    G = sp.csr_matrix((np.ones(r.size, np.int8), (r, c)), shape=(m, m))
    G.sum_duplicates()
    return G


def _vertex_cover_cut(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """One endpoint of every crossing edge (u, v): the endpoint with more crossings."""
    if u.size == 0:
        return np.zeros(0, np.int64)
    ends = np.concatenate([u, v])
    _, inv = np.unique(ends, return_inverse=True)
    cnt = np.bincount(inv)
    pick = np.where(cnt[inv[:u.size]] > cnt[inv[u.size:]], u, v)
    return np.unique(pick)


def bisection_order(m: int, rows: np.ndarray, cols: np.ndarray, pos: np.ndarray,
                    depth: int, leaf_min: int = 8) -> Tuple[np.ndarray, List[int]]:
    """Nested dissection by position bisection.

    ``pos`` gives each node's position (ring index, or a grid coordinate key).
    Each step splits the current node set at its median position; the separator is
    one endpoint of every edge joining the halves.  Returns ``(perm, sizes)``:
    ``perm`` lists node ids in postorder (left subtree, right subtree, separator)
    and ``sizes`` gives the row count of each of the ``2**(depth+1)-1`` tree nodes in
    postorder.  Leaves are themselves ordered by continued bisection down to
    ``leaf_min`` nodes (an ordering only: those inner levels are not reported).
    """
    r0 = np.concatenate([rows, cols]).astype(np.int64)
    c0 = np.concatenate([cols, rows]).astype(np.int64)
    side = np.full(max(m, 1), -1, np.int8)
    inS = np.zeros(max(m, 1), bool)

    def split(nodes, er, ec):
        order = nodes[np.argsort(pos[nodes], kind="stable")]
        half = order.size // 2
        left, right = order[:half], order[half:]
        side[left] = 0
        side[right] = 1
        sr, sc = side[er], side[ec]
        cross = (sr == 0) & (sc == 1)
        S = _vertex_cover_cut(er[cross], ec[cross])
        inS[S] = True
        keep = ~inS[er] & ~inS[ec]
        mL = (sr == 0) & (sc == 0) & keep
        mR = (sr == 1) & (sc == 1) & keep
        L, R = left[~inS[left]], right[~inS[right]]
        side[nodes] = -1
        inS[S] = False
        S_sorted = S[np.argsort(pos[S], kind="stable")]
        return (L, er[mL], ec[mL]), (R, er[mR], ec[mR]), S_sorted

    def leaf_order(nodes, er, ec):
        if nodes.size <= leaf_min:
            return nodes[np.argsort(pos[nodes], kind="stable")]
        a, b, S = split(nodes, er, ec)
        return np.concatenate([leaf_order(*a), leaf_order(*b), S])

    sizes: List[int] = []

    def rec(nodes, er, ec, d):
        if d == 0:
            sizes.append(int(nodes.size))
            return leaf_order(nodes, er, ec)
        a, b, S = split(nodes, er, ec)
        pa = rec(*a, d - 1)
        pb = rec(*b, d - 1)
        sizes.append(int(S.size))
        return np.concatenate([pa, pb, S])

    perm = rec(np.arange(m, dtype=np.int64), r0, c0, depth)
    return perm, sizes


def continued_bisection(m: int, rows: np.ndarray, cols: np.ndarray, pos: np.ndarray,
                        leaf_min: int = 8) -> np.ndarray:
    """Fill-reducing ordering of a whole block by continued position bisection."""
    perm, _ = bisection_order(m, rows, cols, pos, 0, leaf_min)
    return perm


# ----------------------------------------------------------------------------------------
# assembly


class _Builder:
    """Collects B's entries in BTF + ND order, then scrambles B into A."""

    def __init__(self):
        self.r: List[np.ndarray] = []
        self.c: List[np.ndarray] = []
        self.v: List[np.ndarray] = []
        self.n = 0
        self.block_ptr = [0]

    def add_block(self, m: int, rows, cols, off, diag, perm: Optional[np.ndarray] = None) -> int:
        """Append an m x m diagonal block; ``perm`` (new -> old local) reorders it."""
        o = self.n
        if perm is not None:
            inv = np.empty(m, np.int64)
            inv[perm] = np.arange(m)
            rows, cols = inv[rows], inv[cols]
            diag = diag[perm]
        idx = np.arange(m, dtype=np.int64)
        self.r += [rows + o, idx + o]
        self.c += [cols + o, idx + o]
        self.v += [off, diag]
        self.n += m
        self.block_ptr.append(self.n)
        return o

    def add_entries(self, rows, cols, vals):
        self.r.append(np.asarray(rows, np.int64))
        self.c.append(np.asarray(cols, np.int64))
        self.v.append(np.asarray(vals, np.float64))

    def finish(self, rng: np.random.Generator, name: str, scramble: bool = True, **kw) -> Problem:
        import scipy.sparse as sp
        n = self.n
        r = np.concatenate(self.r)
        c = np.concatenate(self.c)
        v = np.concatenate(self.v)
        if scramble:
            P = rng.permutation(n).astype(np.int32)
            Q = rng.permutation(n).astype(np.int32)
        else:
            P = np.arange(n, dtype=np.int32)
            Q = np.arange(n, dtype=np.int32)
        A = sp.csc_matrix((v, (P[r], Q[c])), shape=(n, n))
        A.sum_duplicates()
        A.sort_indices()
        return Problem(name=name, n=n, colptr=A.indptr.astype(np.int32),
                       rowind=A.indices.astype(np.int32), values=A.data.astype(np.float64),
                       P=P, Q=Q, block_ptr=np.asarray(self.block_ptr, np.int32), **kw)


def _small_blocks(rng: np.random.Generator, total: int, sizes: Tuple[int, int]) -> List[int]:
    out: List[int] = []
    left = total
    while left > 0:
        s = int(rng.integers(sizes[0], sizes[1] + 1))
        s = min(s, left)
        out.append(s)
        left -= s
    return out


def rail_links(rng: np.random.Generator, m_ring: int, n_rails: int, deg: Tuple[int, int],
               drop: float = 0.05) -> Tuple[np.ndarray, np.ndarray]:
    """Directed entries (rows, cols) joining ``n_rails`` rail nodes (ids m_ring ..
    m_ring + n_rails - 1) to ring nodes: rail k is tied to round(log-uniform(deg))
    distinct random ring nodes, each tie stored in both directions except that
    ``drop`` of them keep only one (as the netlist's non-ring links)."""
    src, dst = [], []
    for k in range(n_rails):
        cnt = int(min(m_ring, round(float(_log_uniform(rng, deg[0], deg[1], 1)[0]))))
        t = np.unique(rng.integers(0, m_ring, 2 * cnt))
        t = rng.permutation(t)[:cnt]
        src.append(np.full(t.size, m_ring + k, np.int64))
        dst.append(t.astype(np.int64))
    if not src:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    r = np.concatenate(src)
    t = np.concatenate(dst)
    dropped = rng.random(r.size) < drop
    which = rng.random(r.size) < 0.5
    keep_fwd = ~(dropped & which)          # rail row, ring column
    keep_bwd = ~(dropped & ~which)         # ring row, rail column
    rows = np.concatenate([r[keep_fwd], t[keep_bwd]])
    cols = np.concatenate([t[keep_fwd], r[keep_bwd]])
    return rows, cols


def _nd_netlist(rng, m, depth, extra=(0, 1), nonlocal_links=False, n_rails=0, rail_deg=(1000, 50000)):
    m_ring = m - n_rails
    rows, cols = netlist_pattern(rng, m_ring, extra=extra, nonlocal_links=nonlocal_links)
    perm, sizes = bisection_order(m_ring, rows, cols, np.arange(m_ring), depth)
    if n_rails > 0:
        # rails join nodes on both sides of every cut: they belong to the root separator
        rr, rc = rail_links(rng, m_ring, n_rails, rail_deg)
        rows, cols = np.concatenate([rows, rr]), np.concatenate([cols, rc])
        perm = np.concatenate([perm, np.arange(m_ring, m, dtype=np.int64)])
        sizes = list(sizes)
        sizes[-1] += n_rails
    return rows, cols, perm, sizes


def netlist_problem(seed: int, n_small: int = 800, small_sizes=(1, 2), m_netlist: int = 1200,
                    depth: int = 2, extra=(0, 1), nonlocal_links: bool = False,
                    name: str = "netlist", scramble: bool = True, n_rails: int = 0,
                    rail_deg=(1000, 50000), coupling_to: str = "next") -> Problem:
    """Circuit-like matrix in the shape of Fig. 2a: small BTF blocks (D1), one
    strongly connected netlist block in ND order (D2), small BTF blocks (D3).

    Small blocks have U{small_sizes} rows (full, so irreducible); each small block has
    one coupling entry (strictly above the diagonal) into the columns of the next
    block (``coupling_to="next"``: the blocks form one chain) or of a uniformly random
    later block (``"random"``: a shallow DAG of blocks).
    The netlist block is ND-ordered into ``2**depth`` leaves (``depth=0``: no ND).
    ``n_rails`` of the netlist's nodes are supply rails tied to many random nodes
    (``rail_links``); they are ordered last, in the root separator (ND required).
    """
    if n_rails and depth <= 0:
        raise ValueError("rails need an ND ordering")
    rng = np.random.default_rng(seed)
    sizes = _small_blocks(rng, n_small, small_sizes) if n_small > 0 else []
    nb_above = len(sizes) // 2
    layout = sizes[:nb_above] + [-1] + sizes[nb_above:]   # -1 marks the netlist block
    if m_netlist <= 0:
        layout = sizes
    b = _Builder()
    nd_block = -1
    nd_ptr = np.zeros(0, np.int32)
    # coupling entries: one per small block into a later block
    coupling = []
    block_sizes = [m_netlist if s < 0 else s for s in layout]
    offsets = np.concatenate([[0], np.cumsum(block_sizes)]).astype(np.int64)
    for k, s in enumerate(layout):
        if s > 0 and k + 1 < len(layout):
            e = k + 1 if coupling_to == "next" else int(rng.integers(k + 1, len(layout)))
            row = offsets[k] + rng.integers(0, s)
            col = offsets[e] + rng.integers(0, block_sizes[e])
            coupling.append((row, col, float(_log_uniform(rng, 1e-3, 1e3, 1)[0] * _random_sign(rng, 1)[0])))
    cabs = np.zeros(int(offsets[-1]))
    for row, col, val in coupling:
        cabs[row] += abs(val)
    for k, s in enumerate(layout):
        o = int(offsets[k])
        if s < 0:
            if depth > 0:
                rows, cols, perm, nsz = _nd_netlist(rng, m_netlist, depth, extra, nonlocal_links,
                                                    n_rails, rail_deg)
            else:
                rows, cols = netlist_pattern(rng, m_netlist, extra=extra, nonlocal_links=nonlocal_links)
                perm = continued_bisection(m_netlist, rows, cols, np.arange(m_netlist))
                nsz = None
            off, diag = netlist_values(rng, rows, cols, m_netlist)
            b.add_block(m_netlist, rows, cols, off, diag, perm)
            if nsz is not None:
                nd_block = k
                nd_ptr = (o + np.concatenate([[0], np.cumsum(nsz)])).astype(np.int32)
        else:
            if s == 1:
                rows = cols = np.zeros(0, np.int64)
            else:
                rows, cols = netlist_pattern(rng, s, extra=(0, 0))
            off, diag = netlist_values(rng, rows, cols, s, extra_rowabs=cabs[o:o + s])
            b.add_block(s, rows, cols, off, diag)
    if coupling:
        cr, cc, cv = zip(*coupling)
        b.add_entries(cr, cc, cv)
    leaves = 2 ** depth if nd_block >= 0 else 0
    prob = b.finish(rng, name, scramble=scramble, nd_block=nd_block, nd_leaves=leaves,
                    nd_node_ptr=nd_ptr)
    prob.meta.update(seed=seed, n_small_blocks=len(sizes), m_netlist=m_netlist, depth=depth, n_rails=n_rails,
                     nd_node_sizes=np.diff(nd_ptr).tolist() if nd_block >= 0 else [])
    return prob


def grid_problem(seed: int, k: int = 316, depth: int = 4, name: str = "grid",
                 scramble: bool = True) -> Problem:
    """Five-point power-grid mesh, k x k nodes, geometric ND into 2**depth leaves,
    each leaf ordered by continued geometric bisection.  One BTF block."""
    rng = np.random.default_rng(seed)
    n = k * k
    idx = np.arange(n, dtype=np.int64).reshape(k, k)
    e_u = np.concatenate([idx[:-1, :].ravel(), idx[:, :-1].ravel()])
    e_v = np.concatenate([idx[1:, :].ravel(), idx[:, 1:].ravel()])
    g = _log_uniform(rng, 1e-2, 1e2, e_u.size)
    a_uv = -g * rng.uniform(0.9, 1.1, e_u.size)
    a_vu = -g * rng.uniform(0.9, 1.1, e_u.size)
    rows = np.concatenate([e_u, e_v])
    cols = np.concatenate([e_v, e_u])
    off = np.concatenate([a_uv, a_vu])
    diag = np.bincount(rows, weights=np.abs(off), minlength=n) + rng.uniform(0.0, 1e-3, n)
    perm, sizes = _grid_nd(k, depth)
    b = _Builder()
    b.add_block(n, rows, cols, off, diag, perm)
    nd_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    prob = b.finish(rng, name, scramble=scramble, nd_block=0, nd_leaves=2 ** depth,
                    nd_node_ptr=nd_ptr)
    prob.meta.update(seed=seed, k=k, depth=depth, nd_node_sizes=list(map(int, sizes)))
    return prob


def _grid_nd(k: int, depth: int, leaf_min: int = 4) -> Tuple[np.ndarray, List[int]]:
    """Geometric nested dissection of a k x k grid: split the longer side of the
    current rectangle at its middle line, which is the separator.  Leaves are
    ordered by continued bisection of the same kind."""
    sizes: List[int] = []

    def ids(x0, x1, y0, y1):
        xs, ys = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1), indexing="ij")
        return (xs * k + ys).ravel().astype(np.int64)

    def halves(x0, x1, y0, y1):
        w, h = x1 - x0, y1 - y0
        if w >= h:
            xm = x0 + w // 2
            return (x0, xm, y0, y1), (xm + 1, x1, y0, y1), (xm, xm + 1, y0, y1)
        ym = y0 + h // 2
        return (x0, x1, y0, ym), (x0, x1, ym + 1, y1), (x0, x1, ym, ym + 1)

    def order(x0, x1, y0, y1):
        w, h = x1 - x0, y1 - y0
        if w <= 0 or h <= 0:
            return np.zeros(0, np.int64)
        if w * h <= leaf_min:
            return ids(x0, x1, y0, y1)
        a, b, s = halves(x0, x1, y0, y1)
        return np.concatenate([order(*a), order(*b), ids(*s)])

    def rec(x0, x1, y0, y1, d):
        w, h = x1 - x0, y1 - y0
        if w <= 0 or h <= 0:
            sizes.extend([0] * (2 ** (d + 1) - 1))
            return np.zeros(0, np.int64)
        if d == 0:
            sizes.append(w * h)
            return order(x0, x1, y0, y1)
        a, b, s = halves(x0, x1, y0, y1)
        pa = rec(*a, d - 1)
        pb = rec(*b, d - 1)
        sep = ids(*s)
        sizes.append(int(sep.size))
        return np.concatenate([pa, pb, sep])

    perm = rec(0, k, 0, k, depth)
    assert perm.size == k * k
    return perm, sizes


def block_diagonal_problem(seed: int, nblocks: int = 8192, size_range=(4, 1024),
                           extra=(0, 2), name: str = "batched", scramble: bool = True) -> Problem:
    """Independent netlist blocks (no coupling, no ND), sizes round(log-uniform
    size_range), each ordered by continued bisection."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(_log_uniform(rng, size_range[0], size_range[1], nblocks)).astype(np.int64)
    b = _Builder()
    for s in sizes:
        s = int(s)
        rows, cols = netlist_pattern(rng, s, extra=extra)
        perm = continued_bisection(s, rows, cols, np.arange(s))
        off, diag = netlist_values(rng, rows, cols, s)
        b.add_block(s, rows, cols, off, diag, perm)
    prob = b.finish(rng, name, scramble=scramble)
    prob.meta.update(seed=seed, block_sizes=sizes.tolist())
    return prob


# ----------------------------------------------------------------------------------------
# the workloads


def config1(seed: int = CONFIG_SEEDS[1]) -> Problem:
    """n = 2,000 circuit matrix: 800 rows of U{1,2} BTF blocks around a 1,200-row
    netlist block ND-ordered into 4 leaves."""
    return netlist_problem(seed, n_small=800, small_sizes=(1, 2), m_netlist=1200, depth=2,
                           name="circuit_n2000")


def config2(seed: int = CONFIG_SEEDS[2], k: int = 316) -> Problem:
    """316 x 316 power-grid mesh (n = 99,856), ND depth 4 (16 leaves)."""
    return grid_problem(seed, k=k, depth=4, name=f"powergrid_{k}x{k}")


def config3(seed: int = CONFIG_SEEDS[3], nblocks: int = 8192) -> Problem:
    """8,192 independent netlist blocks of log-uniform 4..1,024 rows."""
    return block_diagonal_problem(seed, nblocks=nblocks, name=f"batched_{nblocks}")


def config4(seed: int = CONFIG_SEEDS[4], n: int = 2_000_000, n_rails: int = 200,
            rail_deg=(1000, 50000)) -> Problem:
    """Large circuit: 30% of the n rows in BTF blocks of U{1..16} rows, the rest one
    netlist block with ``n_rails`` supply rails (each tied to log-uniform
    1e3..5e4 random nodes) in the root separator, ND depth 5 (32 leaves).
    Each small block has one coupling entry into a uniformly random later block.
    Smaller ``n`` / ``n_rails`` / ``rail_deg`` give the same structure scaled down."""
    n_small = int(round(0.3 * n))
    return netlist_problem(seed, n_small=n_small, small_sizes=(1, 16), m_netlist=n - n_small, depth=5,
                           n_rails=n_rails, rail_deg=rail_deg, coupling_to="random",
                           name=f"circuit_rails_n{n}")


def rhs_normal(prob: Problem, nrhs: int, seed: int = 0) -> np.ndarray:
    """n x nrhs right-hand sides drawn N(0, 1) (column-major: one column per system)."""
    rng = np.random.default_rng(int(prob.meta.get("seed", 0)) + 7919 + seed)
    return np.asfortranarray(rng.standard_normal((prob.n, nrhs)))


def small_problem(seed: int, kind: str = "netlist", **kw) -> Problem:
    """Small cases for the parity tests (several tiles, ragged tails)."""
    if kind == "netlist":
        args = dict(n_small=60, small_sizes=(1, 3), m_netlist=300, depth=2)
        args.update(kw)
        return netlist_problem(seed, name=f"small_netlist_{seed}", **args)
    if kind == "grid":
        args = dict(k=24, depth=3)
        args.update(kw)
        return grid_problem(seed, name=f"small_grid_{seed}", **args)
    if kind == "blocks":
        args = dict(nblocks=64, size_range=(1, 200))
        args.update(kw)
        return block_diagonal_problem(seed, name=f"small_blocks_{seed}", **args)
    raise ValueError(kind)


def refactor_values(prob: Problem, k: int, sigma: float = 0.05) -> np.ndarray:
    """Values of the k-th matrix of a same-pattern sequence: each stored value of
    the base matrix times (1 + N(0, sigma)), drawn from the base (not compounding);
    seeded by (seed + 100 k)."""
    seed = int(prob.meta.get("seed", 0)) + 100 * k
    rng = np.random.default_rng(seed)
    return prob.values * (1.0 + sigma * rng.standard_normal(prob.values.size))


def rhs_ones(prob: Problem, values: Optional[np.ndarray] = None) -> np.ndarray:
    """b = A * ones (so x = ones is the exact solution)."""
    v = prob.values if values is None else values
    return np.bincount(prob.rowind, weights=v, minlength=prob.n)
