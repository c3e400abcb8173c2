"""Launch-size autotuning: the choices are valid and change nothing in the results."""
import numpy as np
import pytest

from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("kind,seed,kw", [("grid", 81, dict(k=60, depth=3)),
                                           ("netlist", 82, dict(n_small=100, m_netlist=2000, depth=3))])
def test_autotune_keeps_results_bit_for_bit(kind, seed, kw):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    prob = I.small_problem(seed, kind, **kw)
    tuned, plain = (basker.Handle.from_problem(prob) for _ in range(2))
    for h in (tuned, plain):
        h.factor(_dev(prob.values))
    choice = tuned.autotune(_dev(prob.values), _dev(I.rhs_ones(prob)))
    assert choice["static_blocks"] > 0 and choice["solve_blocks"] > 0
    plain.refactor(_dev(prob.values))       # the same history as the tuning runs
    for k in (1, 2, 3):
        v = I.refactor_values(prob, k, sigma=0.3)
        for h in (tuned, plain):
            h.refactor(_dev(v))
        a, b = tuned.export(), plain.export()
        np.testing.assert_array_equal(a[0], b[0])
        for ma, mb in ((a[1], b[1]), (a[2], b[2])):
            np.testing.assert_array_equal(ma.indptr, mb.indptr)
            np.testing.assert_array_equal(ma.indices, mb.indices)
            assert np.array_equal(ma.data, mb.data)
        rhs = _dev(I.rhs_ones(prob, v))
        np.testing.assert_array_equal(tuned.solve(rhs).cpu().numpy(), plain.solve(rhs).cpu().numpy())
