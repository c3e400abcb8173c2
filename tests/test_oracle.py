"""Pins of the oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something it does not share code with:
LAPACK's partial-pivoting LU, a textbook right-looking elimination, exact rational
arithmetic, boolean elimination (fill-path theorem), closed forms, exact
power-of-two scaling, and the paper's own structural facts (Sec. II-III).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_1601_05725_gb300 import inputs as I
from tests import helpers as H


def _factor(prob, tau=1e-3, values=None, pref=None, order="ascending"):
    o = oracle.OracleLU(prob)
    assert o.status == "OK", o.status
    s = o.factor(values, tau=tau, pref=pref, order=order)
    assert s == "OK", (s, o.info_col)
    return o, o.factors()


# ---------------------------------------------------------------------------- LAPACK


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (16, 3), (16, 4)])
def test_dense_matches_lapack_partial_pivoting(n, seed):
    """tau = 1 on a full matrix is classical partial pivoting (LAPACK getrf)."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    prob = H.make_problem(sp.csc_matrix(np.where(M == 0, 1e-300, M)))
    _, f = _factor(prob, tau=1.0)
    lu, piv = sla.lu_factor(M)
    perm = np.arange(n)
    for i, p in enumerate(piv):
        perm[[i, p]] = perm[[p, i]]
    np.testing.assert_array_equal(f.prow, perm)
    np.testing.assert_allclose(f.L.toarray(), np.tril(lu, -1), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(f.U.toarray(), np.triu(lu), rtol=1e-12, atol=1e-14)


def test_sparse_partial_pivoting_matches_lapack_on_dense_copy():
    """A sparse matrix (one block, tau=1): same pivots and factors as getrf on its dense copy."""
    rng = np.random.default_rng(11)
    n = 40
    S = sp.random(n, n, density=0.12, random_state=rng, data_rvs=rng.standard_normal)
    S = (S + sp.diags(rng.standard_normal(n))).tocsc()
    prob = H.make_problem(S, scramble_seed=5)
    _, f = _factor(prob, tau=1.0)
    B = H.b_matrix(prob).toarray()
    lu, piv = sla.lu_factor(B)
    perm = np.arange(n)
    for i, p in enumerate(piv):
        perm[[i, p]] = perm[[p, i]]
    np.testing.assert_array_equal(f.prow, perm)
    scale = np.abs(lu).max()
    np.testing.assert_allclose(f.U.toarray(), np.triu(lu), rtol=1e-10, atol=1e-13 * scale)
    np.testing.assert_allclose(f.L.toarray(), np.tril(lu, -1), rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------- textbook elimination


@pytest.mark.parametrize("kind,seed,tau", [("netlist", 3, 1e-3), ("netlist", 4, 0.5),
                                           ("netlist", 5, 1.0), ("grid", 6, 1e-3),
                                           ("blocks", 7, 0.1)])
def test_matches_textbook_threshold_lu(kind, seed, tau):
    """Per BTF block, pivots confined to the block / ND node: identical pivot
    sequence and factors equal to a right-looking dense elimination."""
    kw = {"netlist": dict(n_small=30, m_netlist=120), "grid": dict(k=10, depth=2),
          "blocks": dict(nblocks=12, size_range=(1, 30))}[kind]
    prob = I.small_problem(seed, kind, **kw)
    _, f = _factor(prob, tau=tau)
    prow, L, U = H.reference_block_lu(prob, tau)
    np.testing.assert_array_equal(f.prow, prow)
    scale = max(np.abs(U).max(), 1.0)
    np.testing.assert_allclose(f.U.toarray(), U, rtol=1e-9, atol=1e-12 * scale)
    np.testing.assert_allclose(f.L.toarray(), L, rtol=1e-9, atol=1e-12)


def test_refactor_preference_matches_textbook():
    """With new values and the previous pivots preferred, the pivot sequence and
    factors match the textbook elimination given the same preferences."""
    prob = I.small_problem(8, "netlist", n_small=20, m_netlist=150)
    o, f = _factor(prob)
    v = I.refactor_values(prob, 1, sigma=0.3)
    assert o.factor(v, tau=0.1, pref=f.prow) == "OK"
    g = o.factors()
    prow, L, U = H.reference_block_lu(prob, 0.1, values=v, pref=f.prow)
    np.testing.assert_array_equal(g.prow, prow)
    np.testing.assert_allclose(g.U.toarray(), U, rtol=1e-9, atol=1e-12 * np.abs(U).max())


def test_nd_pivot_stays_in_node():
    """A leaf column whose largest entry sits in a separator row still pivots inside
    the leaf (Sec. III-C: the leaves and separators are the pivoting blocks)."""
    # two leaves {0,1}, {2,3}, separator {4}
    M = np.array([[1e-2, 1.0, 0.0, 0.0, 2.0],
                  [1.0, 3.0, 0.0, 0.0, 1.0],
                  [0.0, 0.0, 2.0, 1.0, 1.0],
                  [0.0, 0.0, 1.0, 4.0, 1.0],
                  [9.0, 1.0, 1.0, 1.0, 5.0]])
    prob = H.make_problem(M, nd_block=0, nd_leaves=2, nd_node_ptr=[0, 2, 4, 5])
    _, f = _factor(prob, tau=0.5)
    # column 0: candidates rows {0, 1}; |x_0| = 1e-2 < 0.5 * 1 -> row 1, never row 4
    assert f.prow[0] == 1
    prow, L, U = H.reference_block_lu(prob, 0.5)
    np.testing.assert_array_equal(f.prow, prow)
    np.testing.assert_allclose(f.U.toarray(), U, rtol=1e-13)
    # without the node restriction classical pivoting would pick row 4
    free = H.make_problem(M)
    _, g = _factor(free, tau=0.5)
    assert g.prow[0] == 4


# -------------------------------------------------------------------- exact values


def test_exact_rational_lu():
    """Integer, diagonally dominant matrix: every computed entry is the exact
    rational LU entry rounded to within a few ulps."""
    M = np.array([[10, -2, 0, 1, 0, 3],
                  [-1, 12, 4, 0, 0, 0],
                  [0, 3, 9, -2, 1, 0],
                  [2, 0, -1, 11, 0, -3],
                  [0, 0, 2, 0, 8, 1],
                  [1, 0, 0, -4, 2, 13]], dtype=float)
    prob = H.make_problem(M, scramble_seed=2)
    _, f = _factor(prob, tau=1e-3)
    B = H.b_matrix(prob).toarray()
    np.testing.assert_array_equal(f.prow, np.arange(6))   # dominant: diagonal pivots
    E = H.exact_lu(B.tolist())
    Ld, Ud = f.L.toarray(), f.U.toarray()
    for i in range(6):
        for j in range(6):
            ex = float(E[i][j])
            got = Ld[i, j] if i > j else Ud[i, j]
            assert abs(got - ex) <= 8 * np.finfo(float).eps * max(abs(ex), 1.0), (i, j, got, ex)


# ---------------------------------------------------------------- patterns (fill-path)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_patterns_equal_boolean_elimination(seed):
    """Pattern of L+U per block == structural elimination of P B_dd (Sec. III-C,
    the fill-path identities).  Entries that cancel to zero are kept."""
    prob = I.small_problem(20 + seed, "netlist", n_small=24, m_netlist=90)
    o, f = _factor(prob)
    B = H.b_matrix(prob)
    bp = prob.block_ptr
    LU = (f.L + f.U).tocsc()
    LU.data[:] = 1.0
    for d in range(len(bp) - 1):
        k0, k1 = bp[d], bp[d + 1]
        S = (B[f.prow[k0:k1], :][:, k0:k1].toarray() != 0)
        fill = H.boolean_fill(S)
        got = LU[k0:k1, k0:k1].toarray() != 0
        np.testing.assert_array_equal(got, fill)


# ----------------------------------------------------------------------- closed forms


def test_diagonal_matrix():
    d = np.array([3.0, -2.0, 0.5, 7.0])
    prob = H.make_problem(np.diag(d), scramble_seed=1)
    _, f = _factor(prob)
    assert f.L.nnz == 0
    np.testing.assert_array_equal(f.U.diagonal(), H.b_matrix(prob).diagonal())


def test_upper_triangular_is_its_own_u():
    rng = np.random.default_rng(3)
    M = np.triu(rng.standard_normal((9, 9)))
    M[np.abs(M) < 0.5] = 0.0
    np.fill_diagonal(M, rng.uniform(1, 2, 9))
    prob = H.make_problem(M, scramble_seed=4)
    _, f = _factor(prob)
    assert f.L.nnz == 0
    B = H.b_matrix(prob)
    np.testing.assert_array_equal(f.U.toarray(), B.toarray())


def test_tridiagonal_thomas_bitwise():
    """Diagonally dominant tridiagonal: L and U follow the Thomas recurrence
    u_{k+1} = fma(-l_k, c_k, a_{k+1}), l_k = b_k / u_k, bit for bit."""
    rng = np.random.default_rng(5)
    n = 50
    lo, up = rng.uniform(-1, 1, n - 1), rng.uniform(-1, 1, n - 1)
    dg = 3.0 + rng.uniform(0, 1, n)
    M = sp.diags([lo, dg, up], [-1, 0, 1]).tocsc()
    prob = H.make_problem(M)
    _, f = _factor(prob)
    u = np.empty(n)
    l = np.empty(n - 1)
    u[0] = dg[0]
    for k in range(n - 1):
        l[k] = lo[k] / u[k]
        u[k + 1] = _fma(-l[k], up[k], dg[k + 1])
    np.testing.assert_array_equal(f.U.diagonal(), u)
    np.testing.assert_array_equal(f.L.diagonal(-1), l)
    np.testing.assert_array_equal(f.U.diagonal(1), up)


def _fma(a, b, c):
    """Correctly rounded a*b+c from exact rationals."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def test_block_diagonal_concatenates():
    """Factors of a block-diagonal matrix are the per-block factors, bit for bit."""
    p1 = I.small_problem(31, "blocks", nblocks=5, size_range=(3, 25))
    p2 = I.small_problem(32, "blocks", nblocks=4, size_range=(3, 25))
    B1, B2 = H.b_matrix(p1), H.b_matrix(p2)
    both = H.make_problem(sp.block_diag([B1, B2]).tocsc(),
                          block_ptr=np.concatenate([p1.block_ptr, p1.n + p2.block_ptr[1:]]))
    _, f = _factor(both)
    _, f1 = _factor(H.make_problem(B1, block_ptr=p1.block_ptr))
    _, f2 = _factor(H.make_problem(B2, block_ptr=p2.block_ptr))
    np.testing.assert_array_equal(f.prow, np.concatenate([f1.prow, f2.prow + p1.n]))
    np.testing.assert_array_equal(f.U.toarray(), sp.block_diag([f1.U, f2.U]).toarray())
    np.testing.assert_array_equal(f.L.toarray(), sp.block_diag([f1.L, f2.L]).toarray())


# -------------------------------------------------------------- exact scaling invariants


def test_power_of_two_scaling_is_exact():
    prob = I.small_problem(40, "netlist", n_small=20, m_netlist=100)
    _, f = _factor(prob)
    _, g = _factor(prob.with_values(prob.values * 2.0 ** 7))
    np.testing.assert_array_equal(g.prow, f.prow)
    np.testing.assert_array_equal(g.L.data, f.L.data)
    np.testing.assert_array_equal(g.U.data, f.U.data * 2.0 ** 7)


def test_column_scaling_scales_one_column_of_u():
    prob = I.small_problem(41, "netlist", n_small=20, m_netlist=100)
    _, f = _factor(prob)
    j = 57                                            # a column of B
    v = prob.values.copy()
    qa = prob.Q[j]                                    # the same column of A
    v[prob.colptr[qa]:prob.colptr[qa + 1]] *= 2.0 ** -5
    _, g = _factor(prob.with_values(v))
    np.testing.assert_array_equal(g.prow, f.prow)
    np.testing.assert_array_equal(g.L.data, f.L.data)
    Ug, Uf = g.U.toarray(), f.U.toarray()
    Uf[:, j] *= 2.0 ** -5
    np.testing.assert_array_equal(Ug, Uf)


# ------------------------------------------------------------------------- invariants


@pytest.mark.parametrize("make", [lambda: I.config1(), lambda: I.small_problem(9, "grid")])
def test_invariants(make):
    prob = make()
    tau = 1e-3
    o, f = _factor(prob, tau=tau)
    n = prob.n
    Lc = f.L.tocoo()
    assert (Lc.row > Lc.col).all()                              # strictly lower
    # |l_rc| <= 1/tau for rows the pivot was chosen among (the block / ND node);
    # rows of ancestor separators (the L_kj blocks) are not candidates and are not bounded
    brow = f.prow[Lc.row]
    inside = np.array([H.candidate_range(prob, c)[0] <= r < H.candidate_range(prob, c)[1]
                       for r, c in zip(brow, Lc.col)], bool)
    assert np.abs(Lc.data[inside]).max() <= 1.0 / tau
    Uc = f.U.tocoo()
    assert (Uc.row <= Uc.col).all()
    np.testing.assert_array_equal(np.sort(f.prow), np.arange(n))
    for c in range(n):                                          # pivot in the node / block
        lo, hi = H.candidate_range(prob, c)
        assert lo <= f.prow[c] < hi
    Bd = H.diag_blocks(H.b_matrix(prob), prob.block_ptr)
    assert H.factor_backward_error(Bd, f) < 1e-13
    B = o.B()
    assert abs(B - H.b_matrix(prob)).max() == 0


def test_solve_ones_and_scipy():
    prob = I.config1()
    o, f = _factor(prob)
    A = H.a_matrix(prob)
    b = I.rhs_ones(prob)
    x = o.solve(b)
    assert H.solve_backward_error(A, x, b) < 1e-12     # the metric's bar
    np.testing.assert_allclose(x, 1.0, rtol=1e-8)
    rng = np.random.default_rng(0)
    B4 = rng.standard_normal((prob.n, 4))
    X4 = o.solve(B4)
    ref = spla.spsolve(A, B4)
    np.testing.assert_allclose(X4, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


# -------------------------------------------------------------------- structure checks


def _nd_case():
    """4 leaves of 2 rows, separators of 1 row: 11 rows in postorder 1..7 (Fig. 3)."""
    sizes = [2, 2, 1, 2, 2, 1, 1]
    ptr = np.concatenate([[0], np.cumsum(sizes)])
    n = int(ptr[-1])
    return n, ptr


def test_nd_golden_tree_numbering():
    """Which node pairs may hold entries, from the paper's four-leaf example."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "nd_tree_4_leaves.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    n, ptr = _nd_case()
    for a, b, allowed in rows:
        M = np.eye(n) * 4.0
        M[ptr[a - 1], ptr[b - 1]] = 1.0
        prob = H.make_problem(M, nd_block=0, nd_leaves=4, nd_node_ptr=ptr, scramble_seed=a * 10 + b)
        o = oracle.OracleLU(prob)
        assert o.status == ("OK" if allowed else "BAD_ND"), (a, b, o.status)


def test_not_btf_detected():
    M = np.eye(6) * 3.0
    M[4, 1] = 1.0                                         # below the diagonal blocks
    prob = H.make_problem(M, block_ptr=[0, 2, 4, 6], scramble_seed=3)
    o = oracle.OracleLU(prob)
    assert o.status == "NOT_BTF" and o.info_col == 1
    M2 = np.eye(6) * 3.0
    M2[1, 4] = 1.0                                        # above: fine
    assert oracle.OracleLU(H.make_problem(M2, block_ptr=[0, 2, 4, 6])).status == "OK"


def test_invalid_inputs():
    prob = I.small_problem(1, "blocks", nblocks=4, size_range=(2, 5))
    bad = prob.with_values(prob.values)
    bad.P = prob.P.copy()
    bad.P[0] = bad.P[1]
    assert oracle.OracleLU(bad).status == "INVALID"
    bad2 = prob.with_values(prob.values)
    bad2.block_ptr = np.array([0, prob.n + 1], np.int32)
    assert oracle.OracleLU(bad2).status == "INVALID"


def test_singular_and_nan():
    M = np.array([[2.0, 1.0, 0.0], [1.0, 0.5, 0.0], [0.0, 0.0, 3.0]])   # columns 0, 1 dependent
    prob = H.make_problem(M)
    o = oracle.OracleLU(prob)
    assert o.factor(tau=1.0) == "SINGULAR" and o.info_col == 1
    M2 = np.array([[2.0, 1.0], [1.0, 3.0]])
    prob2 = H.make_problem(M2)
    v = prob2.values.copy()
    v[2] = np.nan
    o2 = oracle.OracleLU(prob2)
    assert o2.factor(v) == "NAN" and o2.info_col == 1


# ------------------------------------------------------------ determinism and orders


def test_refactor_same_values_bitwise_and_dfs_order_close():
    prob = I.config1()
    o, f = _factor(prob)
    assert o.refactor(prob.values, f) == "OK"
    g = o.factors()
    np.testing.assert_array_equal(g.prow, f.prow)
    np.testing.assert_array_equal(g.L.data, f.L.data)
    np.testing.assert_array_equal(g.U.data, f.U.data)
    # Algorithm 1's DFS order instead of ascending steps: same pivots, rounding-level change
    o2, h = _factor(prob, order="dfs")
    np.testing.assert_array_equal(h.prow, f.prow)
    np.testing.assert_array_equal(h.U.indices, f.U.indices)
    np.testing.assert_allclose(h.U.data, f.U.data, rtol=1e-10, atol=1e-12 * np.abs(f.U.data).max())
