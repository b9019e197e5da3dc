"""The multi-rank bench path on CPU: two gloo ranks (replicas, one process
per rank) agree on the slowest rank's time, and the reference arm runs on
rank 0 only."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        got = bench.max_over_ranks(1.5 + rank, world)
        # the reference arm: ranks other than 0 return without work or output
        class A:
            warmup, steps = 3, 1
        ref = bench.run_reference(A, None, rank, world) if rank != 0 else "skipped"
        out.put((rank, got, ref))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_rank_main, args=(world, port, q), nprocs=world, join=True, start_method="spawn")
    res = sorted(q.get(timeout=60) for _ in range(world))
    assert [r[1] for r in res] == [2.5, 2.5]
    assert res[1][2] is None


def test_max_over_ranks_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
