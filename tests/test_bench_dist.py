"""Multi-rank path of bench.py on CPU: two gloo ranks, barrier, max over
ranks, and the whole-job throughput formula (weak scaling, one independent
problem per rank, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    elapsed = 1.0 + rank          # rank 1 is the slowest
    m = bench.max_over_ranks(elapsed, w)
    q.put((rank, m, bench.aggregate(w, 5, m)))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, m, v in res:
        assert m == 2.0                       # max over ranks
        assert v == pytest.approx(world * 5 / 2.0)


def test_aggregate_single_rank():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(1, 4, 2.0) == 2.0
    assert bench.algorithmic_flops(16384, 4096) == 2 * 16384 * 16383 * 4096
