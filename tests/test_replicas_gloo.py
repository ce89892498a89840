"""The multi-GPU mode of bench.py is independent replicas (the solver does
not shard): two ranks on the CPU with the gloo backend check the barrier, the
max over ranks of the timed region, the whole-job throughput, and that the
reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rep = bench.Replicas(dist, torch.device("cpu"))
        rep.barrier()
        slowest = rep.max(1.0 + rank)            # rank 1 is the slower one
        value = rep.throughput(100.0, slowest)   # 100 units per rank
        # the reference arm returns at once on ranks other than 0
        ref_none = True
        if rank != 0:
            class A:
                steps, warmup = 1, 0
            ref_none = bench.run_reference(A(), rank, world) is None
        out[rank] = (rep.rank, rep.world, slowest, value, ref_none)
        rep.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in (0, 1):
        r, w, slowest, value, ref_none = out[rank]
        assert (r, w) == (rank, 2)
        assert slowest == 2.0                 # max over ranks, seen by both
        assert value == pytest.approx(100.0)  # 2 ranks x 100 units / 2.0 s
        assert ref_none
