"""bench.py's multi-process plumbing (replicas, one process per GPU) on CPU with gloo:
barriers, max-over-ranks timing and the whole-job throughput aggregate."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), MPT_BENCH_BACKEND="gloo")
    import bench
    w, r, local = bench.dist_setup()
    bench.dist_barrier(w)
    # rank r moved 10 GB in (1 + r) seconds: the job moved 10 GB per rank over the slowest time
    value, slowest = bench.aggregate(w, 10e9, 1.0 + r)
    q.put((r, w, local, value, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_aggregate_uses_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, world, local, value, slowest) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == pytest.approx(2.0)
        assert value == pytest.approx(2 * 10e9 / 2.0 / 1e9)


def test_single_process_needs_no_process_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.aggregate(1, 4e9, 2.0) == (2.0, 2.0)
