"""FP32 factorization with FP64 iterative refinement (options.precision = 1).

The FP32 factors are checked by their own backward error; every solve by the
FP64 backward error eta <= 1e-12 of the refined solution, computed here on the
host from A, x and b, and by its error against the FP64 oracle's solution,
bounded by 2 kappa(A) eta (with slack for the estimate of kappa).  The fallbacks to an FP64 factorization (pivot growth
above the limit, a refinement that stalls) must give the FP64 handle's result.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I
from tests import helpers as H

pytestmark = pytest.mark.gpu

ETA = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    basker.load()


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _solve(h, b):
    return h.solve(_dev(b)).cpu().numpy()


CASES = [
    ("netlist", 11, {}),
    ("netlist", 12, dict(n_small=100, small_sizes=(1, 40), m_netlist=500, depth=3)),
    ("grid", 13, dict(k=30, depth=3)),
    ("blocks", 14, dict(nblocks=200, size_range=(1, 300))),
]


@pytest.mark.parametrize("kind,seed,kw", CASES)
def test_fp32_factors_and_refined_solve(kind, seed, kw):
    prob = I.small_problem(seed, kind, **kw)
    A = H.a_matrix(prob)
    h = basker.Handle.from_problem(prob, precision=1)
    h.factor(_dev(prob.values))
    inf = h.info()
    assert inf["ir_fallbacks"] == 0 and np.isfinite(inf["growth"]) and inf["growth"] > 0
    # the FP32 factors: P B_diag = (I + L) U to FP32 accuracy (times the growth)
    prow, L, U = h.export()
    Bd = H.diag_blocks(H.b_matrix(prob), prob.block_ptr)
    from types import SimpleNamespace
    be = H.factor_backward_error(Bd, SimpleNamespace(prow=prow, L=L, U=U))
    assert be <= 64 * np.finfo(np.float32).eps * max(1.0, inf["growth"]), be
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(prob.n)
    x = _solve(h, b)
    inf = h.info()
    assert inf["precision_used"] == 1 and inf["ir_iterations"] >= 1
    eta = H.solve_backward_error(A, x, b)
    assert eta <= ETA
    assert inf["ir_eta"] <= 1e-13
    # the error against the FP64 oracle's solution, within what eta allows
    err = H.forward_error(x, H.oracle_solution(prob, prob.values, b))
    kappa = H.kappa_inf(A)
    print(f"{kind} {seed}: FP32+IR vs FP64 oracle rel err {err:.2e} (eta {eta:.1e}, kappa {kappa:.1e})")
    assert err <= 20.0 * kappa * max(eta, 1e-16)


def test_fp32_refactor_sequence_and_multiple_rhs():
    prob = I.small_problem(21, "netlist", n_small=60, m_netlist=400, depth=2)
    h = basker.Handle.from_problem(prob, precision=1)
    h.factor(_dev(prob.values))
    rng = np.random.default_rng(21)
    for k in range(1, 5):
        v = I.refactor_values(prob, k, sigma=0.3)
        h.refactor(_dev(v))
        A = sp.csc_matrix((v, prob.rowind, prob.colptr), shape=(prob.n, prob.n))
        B = rng.standard_normal((prob.n, 3))
        X = h.solve(_dev(B)).cpu().numpy()
        eta = H.solve_backward_error(A, X, B)
        assert eta <= ETA
        err = H.forward_error(X, H.oracle_solution(prob, v, B))
        assert err <= 20.0 * H.kappa_inf(A) * max(eta, 1e-16), err
    # the host entry point refines the same way
    v = I.refactor_values(prob, 9, sigma=0.05)
    b = rng.standard_normal(prob.n)
    x = h.refactor_solve_host(v, b).reshape(-1)
    A = sp.csc_matrix((v, prob.rowind, prob.colptr), shape=(prob.n, prob.n))
    assert H.solve_backward_error(A, x, b) <= ETA


def test_growth_limit_hands_the_matrix_to_fp64():
    prob = I.small_problem(31, "grid", k=20, depth=2)
    h32 = basker.Handle.from_problem(prob, precision=1, growth_limit=1e-300)
    h64 = basker.Handle.from_problem(prob)
    h32.factor(_dev(prob.values))
    h64.factor(_dev(prob.values))
    b = np.random.default_rng(31).standard_normal(prob.n)
    x32, x64 = _solve(h32, b), _solve(h64, b)
    inf = h32.info()
    assert inf["ir_fallbacks"] == 1 and inf["precision_used"] == 0
    # the FP64 twin factors the same values from scratch: the same result as a plain FP64 handle
    np.testing.assert_array_equal(x32, x64)


def test_stalled_refinement_falls_back_to_fp64():
    prob = I.small_problem(32, "netlist", n_small=40, m_netlist=300, depth=2)
    A = H.a_matrix(prob)
    h = basker.Handle.from_problem(prob, precision=1, ir_max_iter=1, ir_tol=1e-300)
    h.factor(_dev(prob.values))
    b = np.random.default_rng(32).standard_normal(prob.n)
    x = _solve(h, b)
    inf = h.info()
    assert inf["ir_fallbacks"] == 1 and inf["precision_used"] == 0 and inf["ir_iterations"] == 1
    assert H.solve_backward_error(A, x, b) <= ETA
    # the next factorization starts in FP32 again (and stalls again)
    v = I.refactor_values(prob, 1, sigma=0.05)
    h.refactor(_dev(v))
    x = _solve(h, b)
    inf = h.info()
    assert inf["ir_fallbacks"] == 2 and inf["precision_used"] == 0
    A = sp.csc_matrix((v, prob.rowind, prob.colptr), shape=(prob.n, prob.n))
    assert H.solve_backward_error(A, x, b) <= ETA


def test_precision_option_is_validated():
    prob = I.small_problem(33, "grid", k=10, depth=1)
    for kw in (dict(precision=3), dict(refactor_switch=4), dict(factor_mode=2), dict(symbolic_mode=3), dict(precision=1, ir_max_iter=0), dict(precision=1, ir_tol=0.0),
               dict(precision=1, growth_limit=-1.0)):
        with pytest.raises(basker.BaskerError) as e:
            basker.Handle.from_problem(prob, **kw)
        assert e.value.name == "INVALID_ARG"


def test_fp64_refined_solve_meets_the_bar_and_equals_plain_fp64_when_one_step_suffices():
    prob = I.small_problem(41, "netlist", n_small=60, m_netlist=400, depth=2)
    A = H.a_matrix(prob)
    h2 = basker.Handle.from_problem(prob, precision=2, ir_tol=1e-12)
    h0 = basker.Handle.from_problem(prob)
    for h in (h2, h0):
        h.factor(_dev(prob.values))
    b = np.random.default_rng(41).standard_normal(prob.n)
    x2, x0 = _solve(h2, b), _solve(h0, b)
    inf = h2.info()
    assert inf["precision_used"] == 0 and inf["ir_iterations"] >= 1 and inf["ir_fallbacks"] == 0
    assert H.solve_backward_error(A, x2, b) <= ETA
    if inf["ir_iterations"] == 1:
        np.testing.assert_array_equal(x2, x0)
    # a stricter target takes further steps and still converges
    h3 = basker.Handle.from_problem(prob, precision=2, ir_tol=1e-16)
    h3.factor(_dev(prob.values))
    x3 = _solve(h3, b)
    assert H.solve_backward_error(A, x3, b) <= ETA
