"""The multi-rank path of bench.py on CPU (gloo, world size 2, 127.0.0.1):
the single-instance problem does not shard, so N GPUs run N replicas; the
timing takes the slowest rank's time on every rank and the reported value is
the whole job's (world x per-rank outputs / that time).  The reference arm
runs on rank 0 alone."""
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


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [10.0, 12.5][rank]
    ms = bench._max_over_ranks(local_ms, dist, torch.device("cpu"))
    value = bench._whole_job_value(world, 1000, 4, ms)

    class A:
        workload = "d20_int64"
        steps = 1
        warmup = 0
    ref = bench._reference_arm(A, rank, world) if rank != 0 else None
    q.put((rank, ms, value, ref))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, ref in sorted(out):
        assert ms == 12.5                       # the slowest rank, on every rank
        assert value == pytest.approx(2 * 1000 * 4 / 12.5e-3)
        if rank != 0:
            assert ref == 0                     # reference arm: rank 0 alone works


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(7.0, None, None) == 7.0
    assert bench._whole_job_value(1, 3 ** 20, 30, 1000.0) == pytest.approx(3 ** 20 * 30)
