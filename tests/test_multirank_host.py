"""The multi-rank host logic of bench.py on CPU with two gloo ranks: every
rank runs its own replica, the job's times are the maxima over the ranks, and
only rank 0 prints (the reference arm's other ranks leave without work)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = bench.dist_env()
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.5], w)
        # the reference arm: rank 0 alone runs and prints; the others return at once
        buf = io.StringIO()
        if rank != 0:
            class A:
                warmup, steps = 1, 1
            with redirect_stdout(buf):
                bench.run_reference(A(), bench.WL.DEBLUR512)
        q.put((rank, (r, local, w), got, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_rank0_only():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, env, got, printed = q.get(timeout=120)
        out[rank] = (env, got, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        env, got, printed = out[rank]
        assert env == (rank, rank, world)
        assert got == [2.0, 10.0, 3.5]
        if rank != 0:
            assert printed == ""
