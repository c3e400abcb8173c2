"""The bench's multi-rank logic on CPU (gloo, world size 2): the job's time is the
slowest rank's, the value is every rank's units over it, and the reference arm
runs on rank 0 alone.  The path itself has no exchange step (replicas only), so
no collective is in the data path; these are the bench's bookkeeping collectives.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 2.0 * rank, world, torch.device("cpu"))
        out[rank] = (t, bench.job_rate(10, world, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    # the slowest rank's time (3 s) everywhere; 2 ranks x 10 units over it
    assert res[0] == res[1] == (3.0, 20.0 / 3.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    assert bench.job_rate(40, 1, 4.0) == 10.0


@pytest.mark.slow
def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_block_parallel_oracle_partition_matches_the_whole():
    """The CPU baseline's block-parallel mode: the blocks of B split into groups,
    each group a problem of its own; the oracle on every group gives, bit for bit,
    the oracle's solution of the whole system restricted to the group's rows."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1601_05725_gb300 import inputs as I
    prob = I.block_diagonal_problem(5, nblocks=40, size_range=(3, 60))
    vals = [I.refactor_values(prob, k) for k in (1, 2)]
    rhs = [I.rhs_ones(prob, v) for v in vals]
    groups = bench._block_groups(prob, 3)
    assert sorted(b for g in groups for b in g) == list(range(prob.nblocks))
    whole = oracle.OracleLU(prob)
    assert whole.factor(vals[1]) == "OK"
    xw = whole.solve(rhs[1])                       # by A's columns
    bp = np.asarray(prob.block_ptr)
    for g, (sub, sv, sb) in zip(groups, bench._sub_problems(prob, groups, vals, rhs)):
        o = oracle.OracleLU(sub)
        assert o.factor(sv[1]) == "OK"
        xs = o.solve(sb[1])
        cols = np.concatenate([np.arange(bp[b], bp[b + 1]) for b in g])   # B columns, new order
        np.testing.assert_array_equal(xs, xw[prob.Q[cols]])
    t = bench._par_worker((sub, sv, sb, 0, 2))
    assert len(t) == 2 and min(t) > 0


def test_chain_depths_equal_brute_force_longest_paths():
    """The latency floor's link counts: the longest dependency chains of the
    oracle's factors, against a longest-path search written out over the DAGs
    (forward rows: L(i,k) != 0 puts row k before row i; columns: U(i,k) != 0 puts
    step i before column k)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1601_05725_gb300 import inputs as I
    prob = I.grid_problem(4, k=14, depth=2)
    o = oracle.OracleLU(prob)
    assert o.factor() == "OK"
    f = o.factors()
    dep = bench._chain_depths(prob, f.L, f.U)
    n = prob.n
    L, U = f.L.tocoo(), f.U.tocoo()

    def longest(edges):
        preds = [[] for _ in range(n)]
        for a, b in edges:
            preds[b].append(a)
        depth = [0] * n
        for v in range(n):                 # steps are a topological order
            depth[v] = 1 + max((depth[u] for u in preds[v]), default=0)
        return max(depth)
    assert dep["forward_rows"] == longest([(k, i) for i, k in zip(L.row, L.col)])
    assert dep["columns"] == longest([(i, k) for i, k in zip(U.row, U.col) if i != k])
    heights = bench._nd_tree(prob)
    assert list(heights) == [0, 0, 1, 0, 0, 1, 2]
    ptr = np.asarray(prob.nd_node_ptr)
    assert dep["separator_steps"] == int(ptr[3] - ptr[2] if ptr[3] - ptr[2] > ptr[6] - ptr[5] else ptr[6] - ptr[5]) + int(ptr[7] - ptr[6])
