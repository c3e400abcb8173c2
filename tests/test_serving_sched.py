"""The serving loop's scheduling and memory admission, on the CPU.

Fake handles stand in for the library: each request sleeps a little and returns
a value that depends on its pattern's request count, so the tests can check
that every pattern's requests run in arrival order on one handle at a time,
that different patterns overlap, and that the memory cap holds.
"""
import threading
import time

import numpy as np

from paper_1601_05725_gb300.serve import Request, Server, latency_summary, poisson_arrivals


class FakeHandle:
    def __init__(self, name, nbytes):
        self.name, self.nbytes, self.count, self.freed = name, nbytes, 0, False

    def free(self):
        self.freed = True


def _server(sizes, slots, cap, log, work=0.004):
    lock = threading.Lock()

    def make(prob):
        return FakeHandle(prob, sizes[prob])

    def run(handle, req, slot):
        assert not handle.freed
        with lock:
            log.append(("start", req.pattern, req.rid, time.perf_counter()))
        time.sleep(work)
        handle.count += 1
        with lock:
            log.append(("end", req.pattern, req.rid, time.perf_counter()))
        return np.array([handle.count], float)

    return Server({k: k for k in sizes}, slots=slots, mem_cap=cap, make_handle=make,
                  handle_bytes=lambda h: h.nbytes, run_request=run)


def _requests(names, count, rate, seed):
    rng = np.random.default_rng(seed)
    arr = poisson_arrivals(rng, count, rate)
    pick = rng.integers(0, len(names), size=count)
    return [Request(i, names[pick[i]], np.zeros(1), np.zeros(1), float(arr[i])) for i in range(count)]


def test_pattern_order_and_exclusivity_with_overlap_across_patterns():
    sizes = {"a": 10, "b": 20, "c": 30, "d": 40}
    log = []
    srv = _server(sizes, slots=3, cap=1e9, log=log)
    reqs = _requests(list(sizes), 60, 2000.0, 1)
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    # each pattern's requests in arrival order: the fake handle counts them
    for name in sizes:
        mine = sorted((r for r in res if r.pattern == name), key=lambda r: (r.arrival, r.rid))
        assert [int(r.x[0]) for r in mine] == list(range(1, len(mine) + 1))
    # never two requests of one pattern at once
    active = {}
    overlap_other = False
    running = set()
    for kind, name, rid, t in sorted(log, key=lambda e: (e[3], e[0] == "start")):
        if kind == "start":
            assert not active.get(name)
            active[name] = True
            if running:
                overlap_other = True
            running.add(rid)
        else:
            active[name] = False
            running.discard(rid)
    assert overlap_other, "requests of different patterns should overlap"
    s = latency_summary(res)
    assert s["errors"] == 0 and s["p99_ms"] >= s["p50_ms"] > 0


def test_memory_cap_evicts_idle_patterns_least_recently_used():
    sizes = {"a": 40, "b": 40, "c": 40}
    log = []
    srv = _server(sizes, slots=2, cap=85, log=log)
    reqs = _requests(list(sizes), 30, 5000.0, 2)
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    assert srv.peak_bytes <= 85
    assert srv.evictions > 0
    # an evicted pattern starts again from a new handle: counts restart, order kept
    for name in sizes:
        mine = sorted((r for r in res if r.pattern == name), key=lambda r: (r.arrival, r.rid))
        counts = [int(r.x[0]) for r in mine]
        assert counts[0] == 1 and all(c == 1 or c == p + 1 for p, c in zip(counts, counts[1:]))


def test_pattern_larger_than_the_cap_still_runs_alone():
    sizes = {"big": 500, "small": 10}
    log = []
    srv = _server(sizes, slots=2, cap=100, log=log)
    reqs = [Request(i, "big" if i % 2 == 0 else "small", np.zeros(1), np.zeros(1), 0.001 * i) for i in range(8)]
    res = srv.run(reqs)
    assert all(r.error is None for r in res)
    assert {r.pattern for r in res} == {"big", "small"}
