"""GPU parity: the CUDA library against the oracle, through the C ABI.

Pivots and L/U patterns must match bit for bit; FP64 values within 1e-12
relative per entry (the design keeps the oracle's per-entry operation order, so
they are in fact compared for exact equality too); solves by backward error and
agreement with the oracle's solution.
"""
import numpy as np
import pytest

import oracle
from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    basker.load()


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _oracle(prob, tau=1e-3, values=None, pref=None):
    o = oracle.OracleLU(prob)
    assert o.status == "OK"
    s = o.factor(values, tau=tau, pref=pref)
    return o, s


def assert_same_factors(h, f, exact=True):
    prow, L, U = h.export()
    np.testing.assert_array_equal(prow, f.prow, err_msg="pivot sequence")
    np.testing.assert_array_equal(L.indptr, f.L.indptr, err_msg="L column counts")
    np.testing.assert_array_equal(L.indices, f.L.indices, err_msg="L pattern")
    np.testing.assert_array_equal(U.indptr, f.U.indptr, err_msg="U column counts")
    np.testing.assert_array_equal(U.indices, f.U.indices, err_msg="U pattern")
    for got, ref, name in ((L.data, f.L.data, "L"), (U.data, f.U.data, "U")):
        bad = np.abs(got - ref) > 1e-12 * np.abs(ref)
        assert not bad.any(), f"{name}: {bad.sum()} entries beyond 1e-12 relative"
        if exact:
            assert np.array_equal(got, ref), f"{name}: not bitwise equal (max diff {np.abs(got - ref).max()})"


CASES = [
    ("netlist", 1, {}, 1e-3),
    ("netlist", 2, dict(n_small=100, small_sizes=(1, 40), m_netlist=500, depth=3), 1e-3),
    ("netlist", 3, dict(n_small=0, m_netlist=700, depth=1), 0.1),
    ("netlist", 4, dict(n_small=50, m_netlist=400, depth=2), 1.0),
    ("grid", 5, dict(k=30, depth=3), 1e-3),
    ("grid", 6, dict(k=17, depth=2), 0.5),
    ("blocks", 7, dict(nblocks=200, size_range=(1, 300)), 1e-3),
    ("blocks", 8, dict(nblocks=40, size_range=(30, 700)), 1.0),
]


@pytest.mark.parametrize("kind,seed,kw,tau", CASES)
def test_factor_matches_oracle(kind, seed, kw, tau):
    prob = I.small_problem(seed, kind, **kw)
    o, s = _oracle(prob, tau)
    assert s == "OK"
    h = basker.Handle.from_problem(prob, tau=tau)
    h.factor(_dev(prob.values))
    assert_same_factors(h, o.factors())


def test_info_counts_and_flops_match_the_oracle():
    prob = I.small_problem(17, "netlist", n_small=60, m_netlist=500, depth=3)
    o, s = _oracle(prob)
    f = o.factors()
    h = basker.Handle.from_problem(prob)
    for values in (prob.values, I.refactor_values(prob, 1, sigma=0.3)):
        if values is not prob.values:
            assert o.factor(values, pref=f.prow) == "OK"
            f = o.factors()
            h.refactor(_dev(values))
        else:
            h.factor(_dev(values))
        inf = h.info()
        assert inf["nnz_l"] == f.L.nnz and inf["nnz_u"] == f.U.nnz
        assert inf["flops"] == H.flops(f)
        assert inf["off_diagonal_pivots"] == int((f.prow != np.arange(prob.n)).sum())


def test_config1_factor_solve():
    prob = I.config1()
    o, s = _oracle(prob)
    f = o.factors()
    h = basker.Handle.from_problem(prob)
    h.factor(_dev(prob.values))
    assert_same_factors(h, f)
    b = I.rhs_ones(prob)
    x = h.solve(_dev(b)).cpu().numpy()
    A = H.a_matrix(prob)
    assert H.solve_backward_error(A, x, b) <= 1e-12
    # the solve keeps the oracle's per-entry operation order: equal bit for bit
    np.testing.assert_array_equal(x, o.solve(b))


@pytest.mark.parametrize("kind,seed,kw,sigma,tau", [
    ("netlist", 11, dict(n_small=60, m_netlist=400, depth=2), 0.05, 1e-3),
    ("netlist", 12, dict(n_small=60, m_netlist=400, depth=2), 0.5, 0.3),
    ("grid", 13, dict(k=30, depth=3), 0.05, 1e-3),
    ("grid", 14, dict(k=24, depth=3), 0.3, 0.2),
    ("blocks", 15, dict(nblocks=100, size_range=(2, 200)), 0.5, 0.3),
])
def test_refactor_sequence_matches_oracle(kind, seed, kw, sigma, tau):
    """Same pattern, new values, previous pivots preferred; both the stored-pattern
    path and the repivoting path are exercised (large sigma forces repivots)."""
    prob = I.small_problem(seed, kind, **kw)
    o, s = _oracle(prob, tau)
    f = o.factors()
    h = basker.Handle.from_problem(prob, tau=tau)
    h.factor(_dev(prob.values))
    assert_same_factors(h, f)
    repivots = 0
    for k in range(1, 5):
        v = I.refactor_values(prob, k, sigma=sigma)
        assert o.factor(v, tau=tau, pref=f.prow) == "OK"
        f = o.factors()
        h.refactor(_dev(v))
        repivots += h.info()["last_repivot_columns"]
        assert_same_factors(h, f)
        b = I.rhs_ones(prob, v)
        x = h.solve(_dev(b)).cpu().numpy()
        assert H.solve_backward_error(H.a_matrix(prob.with_values(v)), x, b) <= 1e-12
    if sigma >= 0.3:
        # rounds (columns recomputed by the reach) or, when the stored-pattern pass
        # rejects many pivots, the complete pass with the previous pivots preferred
        assert repivots > 0 or h.info()["full_refactors"] > 0, "the repivoting path was not exercised"


@pytest.mark.parametrize("kind,seed,kw", [
    ("netlist", 71, dict(n_small=60, m_netlist=900, depth=3)),
    ("grid", 72, dict(k=40, depth=3)),
    ("netlist", 73, dict(n_small=0, m_netlist=3000, depth=4, nonlocal_links=True)),
])
def test_dense_separator_elimination_equals_column_by_column(kind, seed, kw):
    """factor_mode 0 runs each separator's in-node phase as one dense
    right-looking elimination, factor_mode 1 column by column in one warp: the
    same factors as the oracle's, in FP64 and (between the two modes) in FP32,
    for the factorization and a refactorization that repivots."""
    prob = I.small_problem(seed, kind, **kw)
    o, s = _oracle(prob)
    f = o.factors()
    hd = basker.Handle.from_problem(prob, factor_mode=0)
    hw = basker.Handle.from_problem(prob, factor_mode=1)
    for h in (hd, hw):
        h.factor(_dev(prob.values))
        assert_same_factors(h, f)
    assert hd.info()["kernel_calls"]["dense_node"] > 0
    assert hw.info()["kernel_calls"]["dense_node"] == 0
    v = I.refactor_values(prob, 1, sigma=0.3)
    assert o.factor(v, pref=f.prow) == "OK"
    g = o.factors()
    for h in (hd, hw):
        h2 = basker.Handle.from_problem(prob, factor_mode=h is hw, refactor_switch=2)
        h2.factor(_dev(prob.values))
        h2.refactor(_dev(v))
        assert_same_factors(h2, g)
    f32 = []
    for mode in (0, 1):
        h = basker.Handle.from_problem(prob, factor_mode=mode, precision=1)
        h.factor(_dev(prob.values))
        f32.append(h.export())
    np.testing.assert_array_equal(f32[0][0], f32[1][0])
    for a, b in zip(f32[0][1:], f32[1][1:]):
        np.testing.assert_array_equal(a.indptr, b.indptr)
        np.testing.assert_array_equal(a.indices, b.indices)
        assert np.array_equal(a.data, b.data)


@pytest.mark.parametrize("kind,seed,kw,dominant", [
    ("grid", 91, dict(k=40, depth=3), True),
    ("netlist", 92, dict(n_small=60, m_netlist=800, depth=3), False),
])
def test_factorization_by_the_stored_pattern_path(kind, seed, kw, dominant):
    """basker_factor first tries the refactorization's path from the symbolic
    arena (natural rows preferred); with few rejected natural pivots it is kept,
    else the complete pass runs.  Either way the factors are the oracle's, also
    when the handle is factored again after refactorizations moved its pivots."""
    prob = I.small_problem(seed, kind, **kw)
    o, s = _oracle(prob)
    f = o.factors()
    h = basker.Handle.from_problem(prob)
    h.factor(_dev(prob.values))
    assert_same_factors(h, f)
    if dominant:
        assert h.info()["static_factors"] == 1
    v = I.refactor_values(prob, 1, sigma=0.3)
    h.refactor(_dev(v))
    assert o.factor(v) == "OK"
    h.factor(_dev(v))
    assert_same_factors(h, o.factors())
    b = I.rhs_ones(prob, v)
    np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), o.solve(b))


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("kind,seed,kw", [
    ("netlist", 95, dict(n_small=60, m_netlist=800, depth=3)),
    ("grid", 96, dict(k=36, depth=3)),
    ("blocks", 97, dict(nblocks=60, size_range=(2, 300))),
])
def test_tree_count_sizing_gives_the_same_factors(kind, seed, kw, mode):
    """options.symbolic_mode 1 sizes L and U by Algorithm 3's elimination-tree
    counts, mode 2 by Algorithm 3's interval estimates for the separators (no
    pattern stored, every factorization a complete pass): the factors,
    refactorizations and solves are the oracle's."""
    prob = I.small_problem(seed, kind, **kw)
    o, s = _oracle(prob)
    f = o.factors()
    h = basker.Handle.from_problem(prob, symbolic_mode=mode)
    inf = h.info()
    l1, u1 = basker.symbolic_counts(prob, mode)
    assert inf["nnz_l_sym"] == l1.sum() and inf["nnz_u_sym"] == u1.sum()
    h.factor(_dev(prob.values))
    assert_same_factors(h, f)
    assert h.info()["static_factors"] == 0
    for k in (1, 2):
        v = I.refactor_values(prob, k, sigma=0.3)
        assert o.factor(v, pref=f.prow) == "OK"
        f = o.factors()
        h.refactor(_dev(v))
        assert_same_factors(h, f)
        b = I.rhs_ones(prob, v)
        np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), o.solve(b))


def test_graph_replay_equals_direct_launches():
    """options.graphs replays the post-factorization launches from a captured
    CUDA graph (slack 0: columns move to the spill pools between replays): the
    solves equal those of direct launches and the oracle's, bit for bit."""
    prob = I.small_problem(81, "netlist", n_small=60, m_netlist=700, depth=3)
    o, s = _oracle(prob)
    f = o.factors()
    hg = basker.Handle.from_problem(prob, slack=0.0, graphs=True)
    hd = basker.Handle.from_problem(prob, slack=0.0, graphs=False)
    for h in (hg, hd):
        h.factor(_dev(prob.values))
        assert_same_factors(h, f)
    for k in range(1, 4):
        v = I.refactor_values(prob, k, sigma=0.3)
        assert o.factor(v, pref=f.prow) == "OK"
        f = o.factors()
        b = I.rhs_ones(prob, v)
        xo = o.solve(b)
        for h in (hg, hd):
            h.refactor(_dev(v))
            np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), xo)
    ig, idd = hg.info(), hd.info()
    assert ig["graph_launches"] == 4 and idd["graph_launches"] == 0


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_refactor_switch_modes_give_the_same_factors(mode):
    """Rounds with the switch to a complete pass (0), rounds only (1), one complete
    pass with the previous pivots preferred (2) and the repair pass in column
    order on the device (3) all compute the refactorization's definition: the
    oracle's factors."""
    prob = I.small_problem(61, "netlist", n_small=80, m_netlist=600, depth=3)
    o, s = _oracle(prob)
    f = o.factors()
    h = basker.Handle.from_problem(prob, refactor_switch=mode)
    h.factor(_dev(prob.values))
    rounds = 0
    for k in range(1, 4):
        v = I.refactor_values(prob, k, sigma=0.3)
        assert o.factor(v, pref=f.prow) == "OK"
        f = o.factors()
        h.refactor(_dev(v))
        rounds += h.info()["last_rounds"]
        assert_same_factors(h, f)
        b = I.rhs_ones(prob, v)
        np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), o.solve(b))
    inf = h.info()
    if mode == 3:
        # one repair pass per refactorization that repivots, no complete pass
        assert rounds == 3 and inf["full_refactors"] == 0
    elif mode == 0:
        assert rounds > 0
    elif mode == 1:
        assert rounds > 0 and inf["full_refactors"] == 0
    else:
        assert rounds == 0 and inf["full_refactors"] == 3   # every step repivots (checked on the oracle)


def test_config2_factor_refactor_solve():
    """The power-grid workload at full size: every pivot, pattern entry and value."""
    prob = I.config2()
    o, s = _oracle(prob)
    f = o.factors()
    h = basker.Handle.from_problem(prob)
    h.factor(_dev(prob.values))
    assert_same_factors(h, f)
    # draw 4 rejects a cascade of consecutive pivots in one leaf
    for k in (1, 2, 3, 4, 5):
        v = I.refactor_values(prob, k)
        assert o.factor(v, pref=f.prow) == "OK"
        f = o.factors()
        h.refactor(_dev(v))
        assert_same_factors(h, f)
        b = I.rhs_ones(prob, v)
        x = h.solve(_dev(b)).cpu().numpy()
        assert H.solve_backward_error(H.a_matrix(prob.with_values(v)), x, b) <= 1e-12


def test_multiple_rhs_and_host_entry_point():
    prob = I.small_problem(21, "netlist", n_small=80, m_netlist=300, depth=2)
    o, _ = _oracle(prob)
    h = basker.Handle.from_problem(prob)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((prob.n, 4))
    X = h.refactor_solve_host(prob.values, B)            # first call factors
    np.testing.assert_array_equal(X, o.solve(B))
    v = I.refactor_values(prob, 1)
    X2 = h.refactor_solve_host(v, B)                     # then refactors
    assert H.solve_backward_error(H.a_matrix(prob.with_values(v)), X2, B) <= 1e-12
    Xd = h.solve(_dev(B)).cpu().numpy()
    np.testing.assert_array_equal(Xd, X2)


def test_edge_cases_small_and_ragged():
    # n = 1
    p1 = H.make_problem(np.array([[3.0]]))
    h = basker.Handle.from_problem(p1)
    h.factor(_dev(p1.values))
    x = h.solve(_dev(np.array([6.0]))).cpu().numpy()
    assert x[0] == 2.0
    # a 33-row dense-ish block (crosses a warp) and 1-row blocks, empty ND separator
    rng = np.random.default_rng(3)
    M = rng.standard_normal((33, 33)) * (rng.random((33, 33)) < 0.3) + np.eye(33) * 4
    blocks = H.make_problem(np.kron(np.eye(1), M), scramble_seed=1)
    o, _ = _oracle(blocks, 0.5)
    h = basker.Handle.from_problem(blocks, tau=0.5)
    h.factor(_dev(blocks.values))
    assert_same_factors(h, o.factors())
    # ND with an empty separator between two leaves that do not touch
    M2 = np.diag([2.0, 3.0, 4.0, 5.0])
    M2[0, 1] = M2[1, 0] = 1.0
    M2[2, 3] = 1.0
    nd = H.make_problem(M2, nd_block=0, nd_leaves=2, nd_node_ptr=[0, 2, 4, 4], scramble_seed=2)
    o, _ = _oracle(nd)
    h = basker.Handle.from_problem(nd)
    h.factor(_dev(nd.values))
    assert_same_factors(h, o.factors())


def test_singular_and_nan_columns_match_oracle():
    prob = I.small_problem(31, "netlist", n_small=40, m_netlist=200, depth=2)
    B = H.b_matrix(prob)
    # zero one column of B inside the ND block: singular at (or before) it
    j = int(prob.nd_node_ptr[2]) + 1
    v = prob.values.copy()
    qa = prob.Q[j]
    v[prob.colptr[qa]:prob.colptr[qa + 1]] = 0.0
    o, s = _oracle(prob, values=v)
    assert s == "SINGULAR"
    h = basker.Handle.from_problem(prob)
    with pytest.raises(basker.BaskerError) as e:
        h.factor(_dev(v))
    assert e.value.name == "SINGULAR" and e.value.column == o.info_col
    v2 = prob.values.copy()
    v2[prob.colptr[qa]] = np.nan
    o2, s2 = _oracle(prob, values=v2)
    assert s2 == "NAN"
    with pytest.raises(basker.BaskerError) as e2:
        h.factor(_dev(v2))
    assert e2.value.name == "NAN" and e2.value.column == o2.info_col
    # the handle recovers
    h.factor(_dev(prob.values))
    o3, _ = _oracle(prob)
    assert_same_factors(h, o3.factors())


def test_structure_errors_at_symbolic():
    M = np.eye(6) * 3.0
    M[4, 1] = 1.0
    with pytest.raises(basker.BaskerError) as e:
        basker.Handle.from_problem(H.make_problem(M, block_ptr=[0, 2, 4, 6], scramble_seed=3))
    assert e.value.name == "NOT_BTF"
    M2 = np.eye(5) * 3.0
    M2[0, 2] = 1.0                                     # leaf 0 to leaf 1: crosses the separator
    with pytest.raises(basker.BaskerError) as e:
        basker.Handle.from_problem(H.make_problem(M2, nd_block=0, nd_leaves=2, nd_node_ptr=[0, 2, 4, 5]))
    assert e.value.name == "BAD_ND"
    prob = I.small_problem(1, "blocks", nblocks=4, size_range=(2, 5))
    P = prob.P.copy()
    P[0] = P[1]
    with pytest.raises(basker.BaskerError) as e:
        basker.Handle(prob.n, prob.colptr, prob.rowind, P, prob.Q, prob.block_ptr)
    assert e.value.name == "INVALID_ARG"


def test_wait_budget_gives_timeout_not_hang():
    """A one-cycle wait budget: the dataflow refactor reports TIMEOUT and returns;
    the device stays usable."""
    prob = I.small_problem(41, "grid", k=40, depth=3)
    seen = False
    for _ in range(5):
        h = basker.Handle.from_problem(prob, wait_budget_cycles=1)
        h.factor(_dev(prob.values))
        try:
            h.refactor(_dev(I.refactor_values(prob, 1, sigma=0.0)))
        except basker.BaskerError as e:
            assert e.name == "TIMEOUT"
            seen = True
        h.free()
        if seen:
            break
    assert seen
    o, _ = _oracle(prob)
    h2 = basker.Handle.from_problem(prob)
    h2.factor(_dev(prob.values))
    h2.refactor(_dev(prob.values))
    assert_same_factors(h2, o.factors())
