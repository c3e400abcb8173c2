"""Symbolic counts on the host (basker_symbolic_counts, no device; CPU only).

Mode 0 is the structural Gilbert-Peierls pass under the natural pivots; mode 1 is
Algorithm 3's elimination-tree counts of the symmetric structure (Sec. III-C);
mode 2 is Algorithm 3 with its interval estimates for the separators.
Pins, independent of the library's arithmetic:
* mode 1 equals the column counts of the boolean elimination of B_dd + B_dd^T
  (the fill-path theorem; the Cholesky structure of the symmetric pattern);
* mode 0 equals the boolean elimination of B_dd itself (no exchanges) and the
  oracle's factors of a matrix whose natural pivots are all kept;
* mode 1 >= mode 0 column by column, with equality for a symmetric pattern;
* mode 2 equals mode 1 on the ND leaves and BTF blocks, bounds it from above
  on the separators, and equals the interval rule written out here from the
  boolean elimination's patterns (each separator column dense, per node,
  between the lowest and the highest row of the ranges that reach it).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I
from tests import helpers as H


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    basker.load()


def _blockwise_boolean_counts(prob, symmetric):
    """L (strictly lower) and U (diagonal included) column counts of the boolean
    elimination of each diagonal block of B (or of B_dd + B_dd^T)."""
    B = H.b_matrix(prob)
    lc = np.zeros(prob.n, np.int64)
    uc = np.zeros(prob.n, np.int64)
    for d in range(prob.nblocks):
        k0, k1 = prob.block_ptr[d], prob.block_ptr[d + 1]
        S = (B[k0:k1, k0:k1].toarray() != 0)
        if symmetric:
            S = S | S.T
        S = S | np.eye(k1 - k0, dtype=bool)
        F = H.boolean_fill(S)
        lc[k0:k1] = np.tril(F, -1).sum(axis=0)
        uc[k0:k1] = np.triu(F).sum(axis=0)
    return lc, uc


SMALL = [
    ("netlist", 1, dict(n_small=30, m_netlist=120, depth=2)),
    ("netlist", 2, dict(n_small=40, small_sizes=(1, 9), m_netlist=200, depth=3)),
    ("grid", 3, dict(k=12, depth=2)),
    ("blocks", 4, dict(nblocks=30, size_range=(1, 40))),
]


@pytest.mark.parametrize("kind,seed,kw", SMALL)
def test_tree_counts_equal_the_symmetric_boolean_elimination(kind, seed, kw):
    prob = I.small_problem(seed, kind, **kw)
    l1, u1 = basker.symbolic_counts(prob, 1)
    lb, ub = _blockwise_boolean_counts(prob, symmetric=True)
    np.testing.assert_array_equal(l1, lb)
    np.testing.assert_array_equal(u1, ub)


@pytest.mark.parametrize("kind,seed,kw", SMALL)
def test_structural_counts_equal_the_boolean_elimination(kind, seed, kw):
    prob = I.small_problem(seed, kind, **kw)
    l0, u0 = basker.symbolic_counts(prob, 0)
    lb, ub = _blockwise_boolean_counts(prob, symmetric=False)
    np.testing.assert_array_equal(l0, lb)
    np.testing.assert_array_equal(u0, ub)


@pytest.mark.parametrize("prob", [I.small_problem(5, "netlist"), I.small_problem(6, "grid"), I.config1(),
                                  I.config4(n=40_000, n_rails=4, rail_deg=(20, 1000))],
                         ids=["netlist", "grid", "config1", "config4_small"])
def test_tree_counts_bound_the_structural_counts(prob):
    l0, u0 = basker.symbolic_counts(prob, 0)
    l1, u1 = basker.symbolic_counts(prob, 1)
    assert (l1 >= l0).all() and (u1 >= u0).all()


def test_symmetric_pattern_gives_equal_counts_and_the_oracle_agrees():
    # the power-grid mesh has a symmetric pattern and keeps its natural pivots
    prob = I.small_problem(7, "grid", k=20, depth=2)
    l0, u0 = basker.symbolic_counts(prob, 0)
    l1, u1 = basker.symbolic_counts(prob, 1)
    np.testing.assert_array_equal(l0, l1)
    np.testing.assert_array_equal(u0, u1)
    o = oracle.OracleLU(prob)
    assert o.factor() == "OK"
    f = o.factors()
    assert (f.prow == np.arange(prob.n)).all()
    np.testing.assert_array_equal(np.diff(f.L.indptr), l0)
    np.testing.assert_array_equal(np.diff(f.U.indptr), u0)


def test_structure_errors_on_the_host():
    prob = I.small_problem(8, "netlist", n_small=20, m_netlist=100, depth=2)
    B = H.b_matrix(prob).tolil()
    # an entry below the diagonal blocks
    k = prob.block_ptr[1]
    B[k, 0] = 1.0
    bad = H.make_problem(B.tocsc(), block_ptr=prob.block_ptr, nd_block=prob.nd_block, nd_leaves=prob.nd_leaves,
                         nd_node_ptr=prob.nd_node_ptr)
    for mode in (0, 1, 2):
        with pytest.raises(basker.BaskerError) as e:
            basker.symbolic_counts(bad, mode)
        assert e.value.name == "NOT_BTF"
    with pytest.raises(basker.BaskerError) as e:
        basker.symbolic_counts(prob, 3)
    assert e.value.name == "INVALID_ARG"


def _nd_nodes(prob):
    """Heights and ancestor lists of the ND nodes (postorder: left, right, parent)."""
    heights, parent = [], []

    def rec(d):
        if d == 0:
            heights.append(0)
            parent.append(-1)
            return len(heights) - 1
        a, b = rec(d - 1), rec(d - 1)
        heights.append(d)
        parent.append(-1)
        parent[a] = parent[b] = len(heights) - 1
        return len(heights) - 1
    rec(int(round(np.log2(prob.nd_leaves))))
    anc = []
    for i in range(len(heights)):
        chain, p = [], parent[i]
        while p >= 0:
            chain.append(p)
            p = parent[p]
        anc.append(chain)
    return heights, anc


def _interval_rule_counts(prob):
    """Algorithm 3's interval estimates written out from the boolean elimination
    of the symmetric structure: the leaves and the BTF blocks count exactly, and
    each of their columns keeps the rows of its L pattern in every ancestor node
    as a range; then, node by node up the tree, separator column c is reached by
    every earlier row t whose range in c's node covers c, and its rows in each
    node are dense between the lowest and the highest row of those rows' ranges
    (above c in its own node) and of its own entries."""
    B = H.b_matrix(prob)
    n = prob.n
    lc = np.zeros(n, np.int64)
    uc = np.zeros(n, np.int64)
    for d in range(prob.nblocks):
        k0, k1 = prob.block_ptr[d], prob.block_ptr[d + 1]
        S = (B[k0:k1, k0:k1].toarray() != 0)
        S = S | S.T | np.eye(k1 - k0, dtype=bool)
        F = H.boolean_fill(S)
        if d != prob.nd_block:
            lc[k0:k1] = np.tril(F, -1).sum(axis=0)
            uc[k0:k1] = np.triu(F).sum(axis=0)
            continue
        heights, anc = _nd_nodes(prob)
        ptr = np.asarray(prob.nd_node_ptr) - k0
        node_of = np.repeat(np.arange(len(heights)), np.diff(ptr))
        m = k1 - k0
        rng = {}                                     # (column, node) -> [lowest, highest] row
        for c in range(m):
            node = node_of[c]
            if heights[node] > 0:
                continue
            lc[k0 + c] = F[c + 1:, c].sum()
            uc[k0 + c] = F[:c + 1, c].sum()
            rows = np.nonzero(F[c + 1:, c])[0] + c + 1
            for q in anc[node]:
                rq = rows[node_of[rows] == q]
                if rq.size:
                    rng[(c, q)] = [int(rq.min()), int(rq.max())]
        for node in range(len(heights)):            # children before parents
            if heights[node] == 0:
                continue
            lo, hi = ptr[node], ptr[node + 1]
            below = [t for t in range(lo) if node in anc[node_of[t]]]
            for c in range(lo, hi):
                reach = [t for t in below + list(range(lo, c))
                         if (t, node) in rng and rng[(t, node)][0] <= c <= rng[(t, node)][1]]
                uc[k0 + c] = len(reach) + 1
                total = 0
                for q in anc[node] + [node]:
                    lows, highs = [], []
                    for t in reach:
                        if (t, q) in rng:
                            a, b = rng[(t, q)]
                            a = max(a, c + 1) if q == node else a
                            if a <= b:
                                lows.append(a)
                                highs.append(b)
                    own = np.nonzero(S[:, c])[0]
                    own = own[(own > c) & (node_of[own] == q)]
                    lows += own.tolist()
                    highs += own.tolist()
                    if lows:
                        rng[(c, q)] = [min(lows), max(highs)]
                        total += max(highs) - min(lows) + 1
                lc[k0 + c] = total
    return lc, uc


@pytest.mark.parametrize("kind,seed,kw", [SMALL[0], SMALL[1], SMALL[2]])
def test_interval_estimates_equal_the_written_out_rule(kind, seed, kw):
    prob = I.small_problem(seed, kind, **kw)
    l2, u2 = basker.symbolic_counts(prob, 2)
    lr, ur = _interval_rule_counts(prob)
    np.testing.assert_array_equal(l2, lr)
    np.testing.assert_array_equal(u2, ur)


@pytest.mark.parametrize("prob", [I.small_problem(5, "netlist"), I.small_problem(6, "grid"), I.config1(),
                                  I.small_problem(9, "blocks", nblocks=40, size_range=(1, 50)),
                                  I.config4(n=40_000, n_rails=4, rail_deg=(20, 1000))],
                         ids=["netlist", "grid", "config1", "blocks", "config4_small"])
def test_interval_estimates_bound_the_tree_counts(prob):
    l0, u0 = basker.symbolic_counts(prob, 0)
    l1, u1 = basker.symbolic_counts(prob, 1)
    l2, u2 = basker.symbolic_counts(prob, 2)
    assert (l2 >= l1).all() and (u2 >= u1).all()
    assert (l2 >= l0).all() and (u2 >= u0).all()
    # equal at the leaves and the BTF blocks (tree levels -1 and 0: exact counts)
    exact = np.ones(prob.n, bool)
    if prob.nd_block >= 0:
        heights, _ = _nd_nodes(prob)
        ptr = np.asarray(prob.nd_node_ptr)
        for node, h in enumerate(heights):
            if h > 0:
                exact[ptr[node]:ptr[node + 1]] = False
    np.testing.assert_array_equal(l2[exact], l1[exact])
    np.testing.assert_array_equal(u2[exact], u1[exact])
