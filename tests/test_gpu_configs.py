"""The benchmark configurations at full size, through the C ABI.

Config 3 (8,192 independent netlist blocks, n = 1.5e6, |L+U| = 4.6e7): the
factorization, a refactorization with new values and the solve against the
oracle, bit for bit; the FP32 factorization with FP64 refinement by backward
error.  Config 2 (the power grid) is covered by test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I
from tests import helpers as H

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c3():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    basker.load()
    return I.config3()


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _same(h, f):
    prow, L, U = h.export()
    np.testing.assert_array_equal(prow, f.prow)
    for got, ref in ((L, f.L), (U, f.U)):
        np.testing.assert_array_equal(got.indptr, ref.indptr)
        np.testing.assert_array_equal(got.indices, ref.indices)
        assert np.array_equal(got.data, ref.data)


def test_config3_factor_refactor_solve_bitwise(c3):
    prob = c3
    o = oracle.OracleLU(prob)
    assert o.factor() == "OK"
    f0 = o.factors()
    h = basker.Handle.from_problem(prob)
    h.factor(_dev(prob.values))
    _same(h, f0)
    b = I.rhs_ones(prob, prob.values)
    np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), o.solve(b))
    v = I.refactor_values(prob, 1)
    assert o.factor(v, pref=f0.prow) == "OK"
    h.refactor(_dev(v))
    _same(h, o.factors())
    b = I.rhs_ones(prob, v)
    np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), o.solve(b))


def test_config3_fp32_refined(c3):
    prob = c3
    A = H.a_matrix(prob)
    h = basker.Handle.from_problem(prob, precision=1)
    h.factor(_dev(prob.values))
    b = I.rhs_ones(prob, prob.values)
    x = h.solve(_dev(b)).cpu().numpy()
    assert H.solve_backward_error(A, x, b) <= 1e-12
    assert h.info()["precision_used"] == 1
    # against the FP64 oracle's solution (independent blocks of at most 1,024 rows)
    # the error against the FP64 oracle's solution, within 2 kappa_inf(A) eta
    eta = H.solve_backward_error(A, x, b)
    err = H.forward_error(x, H.oracle_solution(prob, prob.values, b))
    kappa = H.kappa_inf_blocks(prob)
    print(f"config 3 FP32+IR vs FP64 oracle rel err {err:.2e} (eta {eta:.1e}, kappa {kappa:.1e})")
    assert err <= 2.0 * kappa * max(eta, 1e-16)


@pytest.mark.parametrize("switch", [0, 3])
def test_large_netlist_refactor_sequence_bitwise(switch):
    """An 81,219-row netlist block in 32 ND leaves: every refactorization that
    repivots runs the rounds kernel with its largest shared-memory footprint
    (switch 0) or the repair pass (switch 3)."""
    prob = I.netlist_problem(2001, n_small=0, m_netlist=81219, depth=5, name="netlist_81k")
    o = oracle.OracleLU(prob)
    assert o.factor() == "OK"
    f = o.factors()
    h = basker.Handle.from_problem(prob, refactor_switch=switch)
    h.factor(_dev(prob.values))
    _same(h, f)
    for k in (1, 2, 4):
        v = I.refactor_values(prob, k)
        assert o.factor(v, pref=f.prow) == "OK"
        f = o.factors()
        h.refactor(_dev(v))
        _same(h, f)
        b = I.rhs_ones(prob, v)
        np.testing.assert_array_equal(h.solve(_dev(b)).cpu().numpy(), o.solve(b))
