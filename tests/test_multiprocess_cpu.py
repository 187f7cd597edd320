"""The multi-process (N > 1) path of bench.py on CPU: independent replicas, a barrier and
the max-over-ranks time, reduced over a world_size-2 gloo process group (no GPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        assert (ws, r, local) == (world, rank, rank)
        dist.barrier()
        # rank-dependent timed regions: the job time is the slowest rank's
        t = bench.max_over_ranks(dist, 0.25 + 0.5 * rank, device='cpu')
        rate = bench.aggregate_rate(ws, 1000.0, t)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate_gloo():
    world = 2
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, rate in got:
        assert t == pytest.approx(0.75)                  # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 1000.0 / 0.75)  # weak scaling: all ranks' units / job time


def test_single_process_path():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 1.5) == 1.5
    assert bench.aggregate_rate(1, 10.0, 2.0) == 5.0

