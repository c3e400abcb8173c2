"""Symbolic counts on the host (basker_symbolic_counts, no device; CPU only).

Mode 0 is the structural Gilbert-Peierls pass under the natural pivots; mode 1 is
Algorithm 3's elimination-tree counts of the symmetric structure (Sec. III-C).
Pins, independent of the library's arithmetic:
* mode 1 equals the column counts of the boolean elimination of B_dd + B_dd^T
  (the fill-path theorem; the Cholesky structure of the symmetric pattern);
* mode 0 equals the boolean elimination of B_dd itself (no exchanges) and the
  oracle's factors of a matrix whose natural pivots are all kept;
* mode 1 >= mode 0 column by column, with equality for a symmetric pattern.
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
    for mode in (0, 1):
        with pytest.raises(basker.BaskerError) as e:
            basker.symbolic_counts(bad, mode)
        assert e.value.name == "NOT_BTF"
    with pytest.raises(basker.BaskerError) as e:
        basker.symbolic_counts(prob, 2)
    assert e.value.name == "INVALID_ARG"
