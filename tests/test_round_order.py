"""The claim order of a refactorization round (csrc/round_order.h), on the host.

A round's warps claim columns in this order and wait for the columns their
steps need.  The order must list every column of every active task once, keep
each task's columns ascending (a column's steps in its task come before it, so
no column waits for one not yet claimed), and interleave the tasks in
proportion to their lengths (so that no task's chain starts late).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1601_05725_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "round_order.h"
int main() {
    int k = 0;
    if (std::scanf("%d", &k) != 1) return 1;
    std::vector<std::pair<int32_t, int32_t>> r(k);
    for (auto &p : r) if (std::scanf("%d %d", &p.first, &p.second) != 2) return 1;
    std::vector<int32_t> cols;
    bk::bk_round_order(r, cols);
    std::printf("%zu\n", cols.size());
    for (int32_t c : cols) std::printf("%d\n", c);
    return 0;
}
"""


@pytest.fixture(scope="module")
def order_bin(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("round_order")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def run_order(exe, ranges):
    inp = f"{len(ranges)}\n" + "".join(f"{lo} {hi}\n" for lo, hi in ranges)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    n = int(out[0])
    return np.array([int(v) for v in out[1:1 + n]], dtype=np.int64)


CASES = [
    [(0, 10)],
    [(5, 6), (100, 101)],
    [(0, 3000), (6241, 6400), (12403, 18000), (20000, 20001)],
    [(37, 4000), (4100, 4101), (5000, 5700), (6000, 11000), (11000, 11500)],
    [(0, 0), (10, 20), (30, 30)],
]


@pytest.mark.parametrize("ranges", CASES)
def test_round_order_invariants(order_bin, ranges):
    cols = run_order(order_bin, ranges)
    want = np.concatenate([np.arange(lo, hi) for lo, hi in ranges]) if ranges else np.array([], np.int64)
    # every column once
    assert sorted(cols.tolist()) == sorted(want.tolist())
    pos = {c: i for i, c in enumerate(cols.tolist())}
    N = len(cols)
    for lo, hi in ranges:
        L = hi - lo
        if L <= 0:
            continue
        p = np.array([pos[c] for c in range(lo, hi)])
        # ascending within the task
        assert np.all(np.diff(p) > 0)
        # proportional interleave: after any prefix of the order, the task has had
        # its share of the claims.  A task's column i sits in bucket (2i + 1) N / 2L,
        # so up to bucket b it has b L / N columns within one; a prefix of the
        # order ends inside some bucket b and differs from b by at most the number
        # of tasks K, hence the bound 1 + K L / N.
        K = sum(1 for a, z in ranges if z > a)
        claimed = np.searchsorted(np.sort(p), np.arange(N + 1), side="left")
        share = np.arange(N + 1) * L / N
        assert np.all(np.abs(claimed - share) <= 1.0 + K * L / N + 1e-9)


def test_round_order_task_order_beats_serial(order_bin):
    # the last column of every task comes in the last stretch of the order (the
    # task-by-task order would claim the first task's end long before the others)
    ranges = [(0, 3000), (3000, 9000), (9000, 9300)]
    cols = run_order(order_bin, ranges).tolist()
    N = len(cols)
    for lo, hi in ranges:
        assert cols.index(hi - 1) >= N - N // (hi - lo) - len(ranges)
