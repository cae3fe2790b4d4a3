"""Multi-rank paths of bench.py on CPU (gloo, world size 2).

The hot path does not shard within one problem: N GPUs run N independent replicas (weak scaling)
and torch.distributed only carries the timing reductions.  These tests run those reductions and
the replica seeding in two spawned gloo ranks, and check that the reference arm does no work on
ranks other than 0.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    from svt_inputs import config_problem
    w, r, _, dist = bench._dist()
    mx = bench._max_over_ranks(dist, 1.5 + r, "cpu")
    sm = bench._sum_over_ranks(dist, 1.5 + r, "cpu")
    bench._barrier(dist)
    # replicas: rank k solves the problem of seed (--seed) + k
    p = config_problem("plain_fp64_200", 0 + r)
    q.put((r, w, mx, sm, p.rows.tobytes()[:4096], p.vals[:16].tolist()))
    dist.destroy_process_group()


def test_rank_reductions_and_replica_seeds_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out.sort()
    for r, w, mx, sm, _, _ in out:
        assert w == 2
        assert mx == 2.5          # max over ranks of 1.5 + rank
        assert sm == 4.0          # sum over ranks
    assert out[0][4] != out[1][4] or out[0][5] != out[1][5]   # independent problems


def test_reference_arm_ranks_other_than_zero_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, timeout=120, env=env, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
