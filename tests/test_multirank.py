"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each, as torchrun launches them) reduce their timed seconds by max and their
histories by sum; seeds differ per rank; the reference arm's non-zero ranks
exit without work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, h = bench.reduce_over_ranks(1.5 + rank, 100.0 * (rank + 1), world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, h, bench.rank_seed(rank)))


def test_two_gloo_ranks_reduce_max_time_and_summed_histories():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(t, h) for _, t, h, _ in out] == [(2.5, 300.0), (2.5, 300.0)]
    assert out[0][3] != out[1][3]


def test_single_rank_passes_through():
    import bench
    assert bench.reduce_over_ranks(3.0, 7.0, 1, "cpu") == (3.0, 7.0)


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0
