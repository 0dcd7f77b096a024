"""Host logic of multi-GPU runs, with two gloo ranks on the CPU.

bench.py runs N independent replicas (the update of one graph does not shard), so the
only cross-rank steps are the barriers around the timed region and the max-over-ranks
reduction of the timings.  These run here with world size 2
on the gloo backend.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    seed = bench.replica_seed(rank)
    dist.barrier()
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, float(seed)], "cpu")
    dist.barrier()
    out.put((rank, seed, got))
    dist.destroy_process_group()


def test_replicas_reduce_to_the_slowest_rank():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, g0), (r1, s1, g1) = res
    assert (r0, r1) == (0, 1)
    assert s0 != s1  # every replica works on its own graph
    assert g0 == g1 == [11.0, 5.0, float(max(s0, s1))]
