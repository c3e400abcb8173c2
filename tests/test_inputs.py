"""The synthetic inputs have the structure the method assumes (CPU only).

Checked with scipy, independently of the oracle: B = A(P,Q) is block upper
triangular (Sec. II), every diagonal block is irreducible (strongly connected,
Sec. III-A), and in the ND block each separator disconnects its two halves
(Sec. III-C).
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from paper_1601_05725_gb300 import inputs as I
from tests import helpers as H


def _nd_first(leaves):
    first = []

    def rec(d):
        start = len(first)
        if d > 0:
            rec(d - 1)
            rec(d - 1)
        first.append(start)
    depth = int(np.log2(leaves))
    rec(depth)
    return np.array(first)


def _check_structure(prob, check_scc=True):
    B = H.b_matrix(prob)
    n = prob.n
    blk = H.block_of(prob.block_ptr, n)
    C = B.tocoo()
    assert (blk[C.row] <= blk[C.col]).all(), "entry below the diagonal blocks"
    if check_scc:
        for d in range(prob.nblocks):
            k0, k1 = prob.block_ptr[d], prob.block_ptr[d + 1]
            if k1 - k0 > 1:
                ncomp, _ = connected_components(B[k0:k1, k0:k1], directed=True, connection="strong")
                assert ncomp == 1, f"block {d} is reducible"
    if prob.nd_block >= 0:
        ptr = prob.nd_node_ptr
        k0, k1 = prob.block_ptr[prob.nd_block], prob.block_ptr[prob.nd_block + 1]
        assert ptr[0] == k0 and ptr[-1] == k1
        first = _nd_first(prob.nd_leaves)
        m = (C.row >= k0) & (C.col >= k0) & (C.row < k1) & (C.col < k1)
        tr = np.searchsorted(ptr, C.row[m], side="right") - 1
        tc = np.searchsorted(ptr, C.col[m], side="right") - 1
        related = ((first[tr] <= tc) & (tc <= tr)) | ((first[tc] <= tr) & (tr <= tc))
        assert related.all(), "an entry crosses a separator"
    return B


def test_config1_shape():
    p = I.config1()
    assert p.n == 2000
    assert p.nd_leaves == 4 and len(p.nd_node_ptr) == 8
    sizes = np.diff(p.block_ptr)
    big = int(np.argmax(sizes))
    assert sizes[big] == 1200 and big == p.nd_block
    assert set(np.unique(np.delete(sizes, big))) <= {1, 2}
    B = _check_structure(p)
    # one coupling entry from each small block into the next block
    blk = H.block_of(p.block_ptr, p.n)
    C = B.tocoo()
    off = blk[C.row] < blk[C.col]
    assert np.all(blk[C.col[off]] == blk[C.row[off]] + 1)
    assert off.sum() == p.nblocks - 1 - 1   # every small block except the last; none from D2


def test_config2_shape():
    p = I.config2()
    assert p.n == 316 * 316 and p.nnz == 498016
    assert p.nblocks == 1 and p.nd_leaves == 16
    _check_structure(p, check_scc=False)
    B = H.b_matrix(p)
    assert connected_components(B, directed=True, connection="strong")[0] == 1
    # M-matrix signs: positive diagonal, negative off-diagonals
    assert (B.diagonal() > 0).all()
    C = B.tocoo()
    assert (C.data[C.row != C.col] < 0).all()


@pytest.mark.parametrize("kind,seed", [("netlist", 1), ("netlist", 2), ("grid", 3), ("blocks", 4)])
def test_small_cases_structure(kind, seed):
    _check_structure(I.small_problem(seed, kind))


def test_seeded_and_reproducible():
    a, b = I.config1(), I.config1()
    np.testing.assert_array_equal(a.values, b.values)
    np.testing.assert_array_equal(a.P, b.P)
    v1, v2 = I.refactor_values(a, 1), I.refactor_values(a, 2)
    assert not np.array_equal(v1, v2)
    np.testing.assert_array_equal(v1, I.refactor_values(b, 1))


def test_config4_shape_scaled():
    """The large-circuit generator at a tenth of its size: 30% of the rows in BTF
    blocks of 1..16 rows, one netlist block in 32 ND leaves whose rails sit in the
    root separator and are tied to the requested number of nodes."""
    n, rails, deg = 200_000, 20, (100, 5000)
    p = I.config4(n=n, n_rails=rails, rail_deg=deg)
    assert p.n == n and p.nd_leaves == 32 and len(p.nd_node_ptr) == 64
    sizes = np.diff(p.block_ptr)
    big = int(np.argmax(sizes))
    assert big == p.nd_block and sizes[big] == n - int(round(0.3 * n))
    assert set(np.unique(np.delete(sizes, big))) <= set(range(1, 17))
    B = _check_structure(p)
    # the last `rails` rows of the ND block are the rails: in the root separator,
    # each tied (in at least one direction) to deg[0]..deg[1] ring nodes
    k1 = p.block_ptr[p.nd_block + 1]
    root_lo = p.nd_node_ptr[-2]
    assert k1 - root_lo > rails
    Bd = B[p.block_ptr[p.nd_block]:k1, p.block_ptr[p.nd_block]:k1]
    S = ((Bd != 0).astype(np.int8) + (Bd != 0).T.astype(np.int8)).tocsr()
    m = Bd.shape[0]
    deg_rails = np.diff(S.indptr)[m - rails:] - 1       # minus the diagonal
    assert (deg_rails >= 0.9 * deg[0]).all() and (deg_rails <= deg[1]).all()
    deg_ring = np.diff(S.indptr)[: m - rails]
    assert np.median(deg_ring) < 10


def test_config4_coupling_is_a_shallow_dag_of_blocks():
    """Config 4's small blocks couple into uniformly random later blocks: the
    longest chain of coupled blocks (the solve's critical path through the BTF
    blocks) stays logarithmic, unlike config 1's block-to-next-block chain."""
    p = I.config4(n=40_000, n_rails=4, rail_deg=(20, 1000))
    B = H.b_matrix(p).tocoo()
    blk = H.block_of(p.block_ptr, p.n)
    off = blk[B.row] < blk[B.col]
    src, dst = blk[B.row[off]], blk[B.col[off]]
    assert (dst > src).all()
    depth = np.zeros(p.nblocks, np.int64)
    order = np.argsort(-src, kind="stable")
    for k in order:                      # later blocks first
        depth[src[k]] = max(depth[src[k]], depth[dst[k]] + 1)
    assert depth.max() < 40, depth.max()
    c1 = I.config1()
    B1 = H.b_matrix(c1).tocoo()
    b1 = H.block_of(c1.block_ptr, c1.n)
    o1 = b1[B1.row] < b1[B1.col]
    assert (b1[B1.col[o1]] == b1[B1.row[o1]] + 1).all()


@pytest.mark.slow
def test_config4_full_size_counts():
    p = I.config4()
    assert p.n == 2_000_000 and 11e6 < p.nnz < 14e6
    assert 60_000 < p.nblocks < 80_000
    assert p.meta["nd_node_sizes"][-1] >= 200
