"""Multi-rank host logic on CPU (gloo, world size 2).  The path shards by
view with no data-path collective; the only cross-rank step is the bench's
whole-job reduction: the slowest rank's time and the sum of every rank's
samples.  Two spawned ranks with different figures must both get those."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, samples = bench.reduce_over_ranks(10.0 + 2.5 * rank, 1000 * (rank + 1), "cpu")
        out[rank] = (ms, samples)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res == {0: (12.5, 3000), 1: (12.5, 3000)}


def test_reduce_over_ranks_single_process_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.0, 42, "cpu") == (7.0, 42)
