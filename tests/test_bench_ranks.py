"""Replica runs of bench.py (one process per GPU, no data-path collective):
the job's time is the slowest rank's and its value counts every rank's work.
Two gloo ranks on the CPU exercise the same host logic."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    import bench
    td.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [3.0, 5.0][rank]
        slowest = bench.max_over_ranks(mine, "cpu")
        q.put((rank, slowest, bench.job_value(1e9, 4, world, slowest)))
    finally:
        td.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [5.0, 5.0]
    # 2 replicas x 4 steps x 1 GB in 5 s
    assert out[0][2] == pytest.approx(2 * 4 * 1e9 / 5.0 / 1e9)


def test_single_process_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.job_value(8e9, 2, 1, 4.0) == pytest.approx(4.0)
