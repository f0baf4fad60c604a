"""Host logic of the multi-rank bench on CPU with gloo, world size 2: each
rank owns a different camera, the slowest rank's time is what every rank
sees, and the whole-job throughput counts every rank's pixels."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, local, w = bench.dist_env()
    bench.barrier(w)
    slowest = bench.reduce_max(10.0 + 5.0 * r, w)
    out.put((r, bench.rank_seed(1, r), slowest))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_rank_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] != res[1][1]                 # distinct cameras per rank
    assert res[0][2] == res[1][2] == 15.0         # both see the slowest rank's time


def test_aggregate_counts_every_rank():
    one = bench.aggregate_mpx_per_s(1, 100, 1920 * 1080, 10.0)
    two = bench.aggregate_mpx_per_s(2, 100, 1920 * 1080, 10.0)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(100 * 1920 * 1080 / 0.01 / 1e6)
    assert bench.bytes_per_pixel(5, 0) == 327.125 and bench.bytes_per_pixel(3, 1) == 103.125
