"""basker_solve_noalloc against basker_solve, through the C ABI.

Some callers cannot allocate device memory when they solve: a simulator whose
time-step loop runs on a pool or caching allocator that reserved the device
memory up front, where a cudaMalloc can fail and a cudaFree stalls the whole
device.  basker_solve_noalloc serves them from a fixed array compiled into the
library.  Two calls in a row must give what the allocating solve gives, and a
request larger than the array must be refused cleanly.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _colmajor(A, torch):
    """(n, k) CUDA float64 tensor with column-major strides."""
    return torch.as_tensor(np.ascontiguousarray(A.T), device="cuda").t()


@pytest.mark.parametrize("kind,seed,kw,nrhs", [
    ("netlist", 51, dict(n_small=60, m_netlist=400, depth=2), 3),
    ("grid", 52, dict(k=60, depth=3), 1),
])
def test_noalloc_solve_matches_solve_on_two_calls(kind, seed, kw, nrhs):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    prob = I.small_problem(seed, kind, **kw)
    h = basker.Handle.from_problem(prob)
    h.factor(torch.as_tensor(prob.values, device="cuda"))
    rng = np.random.default_rng(seed)
    for _ in range(2):
        B = rng.standard_normal((prob.n, nrhs))
        b = _colmajor(B, torch)
        ref = h.solve(b).cpu().numpy()
        x = _colmajor(np.full((prob.n, nrhs), np.nan), torch)
        h.solve_noalloc(b, x)
        got = x.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_noalloc_solve_refuses_more_than_its_array():
    import torch
    build.build()
    prob = I.small_problem(53, "blocks", nblocks=20, size_range=(5, 60))
    h = basker.Handle.from_problem(prob)
    h.factor(torch.as_tensor(prob.values, device="cuda"))
    nrhs = (1 << 20) // prob.n + 1
    b = _colmajor(np.ones((prob.n, nrhs)), torch)
    x = _colmajor(np.zeros((prob.n, nrhs)), torch)
    with pytest.raises(basker.BaskerError) as e:
        h.solve_noalloc(b, x)
    assert e.value.name == "INVALID_ARG"
    # a fitting request still works afterwards
    x1 = _colmajor(np.zeros((prob.n, 1)), torch)
    h.solve_noalloc(_colmajor(np.ones((prob.n, 1)), torch), x1)
    np.testing.assert_allclose(x1.cpu().numpy(), h.solve(_colmajor(np.ones((prob.n, 1)), torch)).cpu().numpy(),
                               rtol=1e-12)
