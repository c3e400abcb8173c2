"""basker_solve_noalloc against basker_solve and the oracle, through the C ABI.

Some callers cannot allocate device memory when they solve: a simulator whose
time-step loop runs on a pool or caching allocator that reserved the device
memory up front, where a cudaMalloc can fail and a cudaFree stalls the whole
device.  basker_solve_noalloc serves them from a fixed array compiled into the
library.  Each test below starts from a freshly factored handle that has never
solved, so an entry point that allocated its work vectors would show up in the
handle's device bytes.  Two calls in a row must give exactly what the
allocating solve and the oracle give (the solve keeps the oracle's per-entry
operation order, so the results are equal bit for bit), and a request larger
than the array must be refused cleanly.

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

    import oracle
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    prob = I.small_problem(seed, kind, **kw)
    o = oracle.OracleLU(prob)
    assert o.factor() == "OK"
    h = basker.Handle.from_problem(prob)
    h.factor(torch.as_tensor(prob.values, device="cuda"))
    rng = np.random.default_rng(seed)
    for call in range(2):
        B = rng.standard_normal((prob.n, nrhs))
        b = _colmajor(B, torch)
        x = _colmajor(np.full((prob.n, nrhs), np.nan), torch)
        torch.cuda.synchronize()
        dev_bytes = h.info()["device_bytes"]
        torch_allocs = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        h.solve_noalloc(b, x)
        torch.cuda.synchronize()
        # nothing allocated: the handle's arena did not grow and torch's allocator
        # served no request during the call
        assert h.info()["device_bytes"] == dev_bytes
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == torch_allocs
        got = x.cpu().numpy()
        np.testing.assert_array_equal(got, o.solve(B).reshape(prob.n, nrhs))
        if call == 1:
            # the allocating solve afterwards (it makes its buffers now) agrees bit for bit
            np.testing.assert_array_equal(got, h.solve(b).cpu().numpy())


def test_noalloc_solve_refuses_what_it_cannot_serve():
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
    # buffers the entry point would overrun are refused on the host, before the call
    one = _colmajor(np.ones((prob.n, 1)), torch)
    with pytest.raises(ValueError):
        h.solve_noalloc(_colmajor(np.ones((prob.n, 3)), torch), one)            # x narrower than b
    with pytest.raises(ValueError):
        h.solve_noalloc(one.float(), one)                                        # not float64
    with pytest.raises(ValueError):
        h.solve_noalloc(_colmajor(np.ones((prob.n + 1, 1)), torch), one)        # wrong n
    # a fitting request still works afterwards
    x1 = _colmajor(np.zeros((prob.n, 1)), torch)
    h.solve_noalloc(one, x1)
    np.testing.assert_array_equal(x1.cpu().numpy(), h.solve(one).cpu().numpy())
    # refined handles are refused (their refinement needs buffers of its own)
    for prec in (1, 2):
        hr = basker.Handle.from_problem(prob, precision=prec)
        hr.factor(torch.as_tensor(prob.values, device="cuda"))
        with pytest.raises(basker.BaskerError) as e:
            hr.solve_noalloc(one, x1)
        assert e.value.name == "INVALID_ARG"
        hr.free()
