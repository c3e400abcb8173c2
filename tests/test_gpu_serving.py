"""The serving loop on the GPU: continuous batching over several patterns.

Requests of four netlist patterns arrive faster than they are served, so they
queue and overlap on the device (three slots, one stream each).  Every FP64
result must equal, bit for bit, the result of the same pattern's requests run
alone in order on a fresh handle, and the oracle's along the same sequence;
every FP32-refined result must meet the backward-error bar, and its error
against the FP64 oracle's solution is stated and bounded by the condition
number times the backward error.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1601_05725_gb300 import basker, build
from paper_1601_05725_gb300 import inputs as I
from paper_1601_05725_gb300.serve import Request, Server, latency_summary, poisson_arrivals
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream_of_requests():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    basker.load()
    sizes = [(800, 2), (1500, 2), (2500, 3), (4000, 3)]
    pats = {f"p{k}": I.netlist_problem(60 + k, n_small=0, m_netlist=m, depth=dep, name=f"serve_{k}")
            for k, (m, dep) in enumerate(sizes)}
    rng = np.random.default_rng(7)
    count = 30
    arr = poisson_arrivals(rng, count, 2000.0)
    names = sorted(pats)
    reqs = []
    for i in range(count):
        name = names[int(rng.integers(0, len(names)))]
        prob = pats[name]
        v = I.refactor_values(prob, 1 + i, sigma=0.05)
        reqs.append(Request(i, name, v, I.rhs_ones(prob, v), float(arr[i])))
    return pats, reqs


def test_mixed_results_equal_alone_fp64(stream_of_requests):
    pats, reqs = stream_of_requests
    srv = Server(pats, slots=3, mem_cap=100e9)
    res = srv.run(reqs)
    srv.close()
    assert all(r.error is None for r in res), [r.error for r in res if r.error]
    # overlap: some request started before another one finished
    iv = sorted((r.start, r.finish) for r in res)
    assert any(b[0] < a[1] for a, b in zip(iv, iv[1:]))
    # alone: each pattern's requests in arrival order on a fresh handle; and the
    # oracle along the same sequence (a factorization, then refactorizations with
    # the previous pivots preferred), bit for bit
    for name, prob in pats.items():
        h = basker.Handle.from_problem(prob)
        o = oracle.OracleLU(prob)
        f = None
        for r in sorted((q for q in reqs if q.pattern == name), key=lambda q: (q.arrival, q.rid)):
            x = h.refactor_solve_host(r.values, r.b)
            np.testing.assert_array_equal(res[r.rid].x, x)
            assert (o.factor(r.values) if f is None else o.refactor(r.values, f)) == "OK"
            f = o.factors()
            np.testing.assert_array_equal(res[r.rid].x, o.solve(r.b))
        h.free()
    s = latency_summary(res)
    assert s["errors"] == 0 and s["p99_ms"] >= s["p50_ms"] > 0


def test_mixed_fp32_refined_meets_the_bar(stream_of_requests):
    pats, reqs = stream_of_requests
    srv = Server(pats, slots=3, mem_cap=100e9, precision=1)
    res = srv.run(reqs)
    srv.close()
    assert all(r.error is None for r in res), [r.error for r in res if r.error]
    errs = []
    for r in res:
        q = reqs[r.rid]
        prob = pats[q.pattern]
        A = sp.csc_matrix((q.values, prob.rowind, prob.colptr), shape=(prob.n, prob.n))
        eta = H.solve_backward_error(A, r.x, q.b)
        assert eta <= 1e-12
        # the error against the FP64 oracle's solution of the same system, within
        # what the backward error allows: |dx| / |x| <= 2 kappa_inf(A) eta (kappa
        # from a norm estimate, so with a factor 10 of slack)
        err = H.forward_error(r.x, H.oracle_solution(prob, q.values, q.b))
        kappa = H.kappa_inf(A)
        assert err <= 20.0 * kappa * max(eta, 1e-16), (err, kappa, eta)
        errs.append(err)
    print(f"FP32+IR served results vs the FP64 oracle: max rel err {max(errs):.2e}, median {np.median(errs):.2e}")


def test_memory_cap_evicts_and_results_stay_exact(stream_of_requests):
    pats, reqs = stream_of_requests
    # room for about two of the four patterns
    one = basker.Handle.from_problem(pats["p3"])
    cap = 2.2 * one.info()["device_bytes"]
    one.free()
    srv = Server(pats, slots=2, mem_cap=cap)
    res = srv.run(reqs)
    srv.close()
    assert all(r.error is None for r in res), [r.error for r in res if r.error][:3]
    assert srv.evictions > 0 and srv.peak_bytes <= cap
    # an evicted pattern restarts from a factorization: its sequence is split there
    errs = []
    for r in res:
        q = reqs[r.rid]
        prob = pats[q.pattern]
        A = sp.csc_matrix((q.values, prob.rowind, prob.colptr), shape=(prob.n, prob.n))
        eta = H.solve_backward_error(A, r.x, q.b)
        assert eta <= 1e-12
        # the error against the FP64 oracle's solution of the same system, within
        # what the backward error allows: |dx| / |x| <= 2 kappa_inf(A) eta (kappa
        # from a norm estimate, so with a factor 10 of slack)
        err = H.forward_error(r.x, H.oracle_solution(prob, q.values, q.b))
        kappa = H.kappa_inf(A)
        assert err <= 20.0 * kappa * max(eta, 1e-16), (err, kappa, eta)
        errs.append(err)
    print(f"FP32+IR served results vs the FP64 oracle: max rel err {max(errs):.2e}, median {np.median(errs):.2e}")
