"""A serving loop for streams of refactor+solve requests on one GPU.

Each request names a sparsity pattern, carries new values of A (same pattern)
and one right-hand side, and asks for x = A^{-1} b.  The server keeps, per
pattern, a library handle with its symbolic data, pivots and L/U resident on
the device; the first request of a pattern factors, later ones refactor with
the previous pivots preferred (the matrix-sequence case of Sec. V).

Continuous batching: ``slots`` worker threads each drive one CUDA stream.  A
free slot takes the earliest request that has arrived and whose pattern is not
being served by another slot, so requests of different patterns run at the same
time on the device while each pattern's requests keep their arrival order.
Admission is by device memory: a pattern's handle is created only when the
handles held stay under ``mem_cap`` bytes, evicting idle handles least recently
used first; a request whose handle does not fit waits for memory.  Because a
pattern's requests are served in order by one handle, every result is the one
the same sequence gives alone.

The compute runs in the library's kernels; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    pattern: str
    values: np.ndarray          # nnz(A) float64, A's CSC order
    b: np.ndarray               # n float64
    arrival: float = 0.0        # seconds after the start of the run


@dataclasses.dataclass
class Result:
    rid: int
    pattern: str
    x: np.ndarray
    arrival: float
    start: float
    finish: float
    slot: int
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class _Entry:
    """A resident pattern: its handle, memory and state."""

    def __init__(self, handle, nbytes: int):
        self.handle = handle
        self.nbytes = nbytes
        self.busy = False
        self.last_used = 0.0


class Server:
    """patterns: name -> Problem (pattern, permutations, BTF/ND structure).

    make_handle(problem) -> handle and handle_bytes(handle) -> device bytes are
    injectable so that the scheduling can be exercised without a GPU.
    run_request(handle, request, slot) -> x performs one refactor+solve.
    """

    def __init__(self, patterns: Dict[str, object], slots: int = 4, mem_cap: float = 100e9,
                 make_handle: Optional[Callable] = None, handle_bytes: Optional[Callable] = None,
                 run_request: Optional[Callable] = None, precision: int = 0):
        self.patterns = patterns
        self.slots = max(1, int(slots))
        self.mem_cap = float(mem_cap)
        self.precision = int(precision)
        self._make_handle = make_handle or self._gpu_handle
        self._handle_bytes = handle_bytes or self._gpu_bytes
        self._run_request = run_request or self._gpu_request
        self._lock = threading.Condition()
        self._resident: Dict[str, _Entry] = {}
        self._size: Dict[str, int] = {}          # device bytes of each pattern's handle, once built
        self._streams: List[object] = []
        self.evictions = 0
        self.peak_bytes = 0

    # ---- GPU implementations (the library through its Python binding)
    def _gpu_handle(self, prob):
        from . import basker
        return basker.Handle.from_problem(prob, precision=self.precision)

    @staticmethod
    def _gpu_bytes(handle) -> int:
        return int(handle.info()["device_bytes"])

    def _gpu_request(self, handle, req: Request, slot: int) -> np.ndarray:
        return handle.refactor_solve_host(req.values, req.b, stream=self._streams[slot])

    # ---- memory admission
    def _held(self) -> int:
        return sum(e.nbytes for e in self._resident.values())

    def _evict_for(self, need: int) -> bool:
        """Free idle handles, least recently used first, until need more bytes fit."""
        idle = sorted((e.last_used, name) for name, e in self._resident.items() if not e.busy)
        for _, name in idle:
            if self._held() + need <= self.mem_cap:
                break
            e = self._resident.pop(name)
            self.evictions += 1
            free = getattr(e.handle, "free", None)
            if free:
                free()
        return self._held() + need <= self.mem_cap

    def _acquire(self, name: str):
        """The pattern's entry, marked busy (created, after admission, if needed).
        Called with the lock held; returns None if memory must be waited for."""
        e = self._resident.get(name)
        if e is not None:
            e.busy = True
            return e
        # a handle's size is known once it has been built: a known size is checked
        # before building; a new one is built, then room is made (a pattern larger
        # than the cap still runs when nothing else is resident)
        known = self._size.get(name)
        if known is not None and not self._evict_for(known) and self._resident:
            return None
        handle = self._make_handle(self.patterns[name])
        nbytes = self._handle_bytes(handle)
        self._size[name] = nbytes
        if not self._evict_for(nbytes) and self._resident:
            free = getattr(handle, "free", None)
            if free:
                free()
            return None
        e = _Entry(handle, nbytes)
        e.busy = True
        self._resident[name] = e
        self.peak_bytes = max(self.peak_bytes, self._held())
        return e

    # ---- the loop
    def run(self, requests: List[Request]) -> List[Result]:
        """Serve requests (arrival times relative to now); returns results by rid."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results: Dict[int, Result] = {}
        t0 = time.perf_counter()
        if self._run_request == self._gpu_request and not self._streams:
            import torch
            self._streams = [torch.cuda.Stream() for _ in range(self.slots)]

        def take(now: float):
            # the earliest arrived request whose pattern is free and admitted; a
            # pattern's later requests wait behind its earliest (order kept)
            blocked = set()
            for i, r in enumerate(pending):
                if r.arrival > now:
                    break
                if r.pattern in blocked:
                    continue
                blocked.add(r.pattern)
                e = self._resident.get(r.pattern)
                if e is not None and e.busy:
                    continue
                entry = self._acquire(r.pattern)
                if entry is not None:
                    return i, entry
            return None, None

        def worker(slot: int):
            while True:
                with self._lock:
                    while True:
                        if not pending:
                            return
                        now = time.perf_counter() - t0
                        i, entry = take(now)
                        if i is not None:
                            req = pending.pop(i)
                            break
                        nxt = pending[0].arrival - now if pending else 0.0
                        self._lock.wait(timeout=max(1e-4, min(nxt, 0.01)))
                start = time.perf_counter() - t0
                err = None
                try:
                    x = self._run_request(entry.handle, req, slot)
                except Exception as ex:       # reported per request
                    x, err = None, f"{type(ex).__name__}: {ex}"
                finish = time.perf_counter() - t0
                with self._lock:
                    entry.busy = False
                    entry.last_used = finish
                    results[req.rid] = Result(req.rid, req.pattern, x, req.arrival, start, finish, slot, err)
                    self._lock.notify_all()

        threads = [threading.Thread(target=worker, args=(k,), daemon=True) for k in range(self.slots)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]

    def close(self):
        with self._lock:
            for e in self._resident.values():
                free = getattr(e.handle, "free", None)
                if free:
                    free()
            self._resident.clear()


def poisson_arrivals(rng: np.random.Generator, count: int, rate: float) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate (requests per second)."""
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def latency_summary(results: List[Result]) -> dict:
    lat = np.array([r.latency for r in results if r.error is None])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    errs = sorted({r.error for r in results if r.error is not None})
    return {"requests": len(results), "errors": sum(r.error is not None for r in results),
            "error_kinds": errs[:3],
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "throughput": len(lat) / span if span > 0 else None}
