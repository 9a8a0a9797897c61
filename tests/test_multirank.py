"""Host logic of the N > 1 benchmark path (replicas: one independent
instance per rank, no collective on the data path) with world_size-2
gloo process groups on the CPU: the max-over-ranks timing, the whole-job
throughput and the per-rank replica seeds."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]
        ms_max = bench.max_over_ranks(ms, "cpu")
        q.put((rank, ms_max, bench.job_gflops(1e9, world, ms_max),
               bench.replica_seed(2, rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_seeds():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # both ranks see the slower rank's time; value counts both ranks' work
    assert [o[1] for o in out] == [5.0, 5.0]
    assert all(abs(o[2] - 2 * 1e9 / 5e-3 / 1e9) < 1e-9 for o in out)
    assert out[0][3] != out[1][3]


def test_single_process_without_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5, "cpu") == 4.5
    assert bench.job_gflops(2e9, 1, 2.0) == 1000.0
