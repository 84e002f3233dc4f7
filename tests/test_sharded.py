"""Column-sharded back-transformation (paper_1811_01277_gb300.sharded) on
CPU ranks (gloo, world size 2): the shard map covers every column once in
whole 128-column items, the reflectors reach every rank by broadcast, and
the concatenation of the ranks' blocks equals the single-rank result.

The per-rank compute here is the oracle (a stand-in that needs no GPU,
passed in by the test; the product path calls the library), so this checks
the host-side partitioning, broadcast and gather exactly."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")


def test_column_shard_covers_every_column_once():
    from paper_1811_01277_gb300.sharded import column_shard
    for nev in (0, 1, 127, 128, 129, 1000, 4096, 4097):
        for world in (1, 2, 3, 4, 8):
            parts = [column_shard(nev, world, r) for r in range(world)]
            cols = [c for c0, k in parts for c in range(c0, c0 + k)]
            assert cols == list(range(nev))
            for c0, k in parts:
                if k:      # a non-empty block starts on an item and holds whole items, bar the last
                    assert c0 % 128 == 0 and (k % 128 == 0 or c0 + k == nev)
            units = [-(-k // 128) for _, k in parts]
            assert max(units) - min(units) <= 1          # items spread as evenly as possible
    with pytest.raises(ValueError):
        column_shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, b, nev, q):
    import torch.distributed as dist
    from paper_1811_01277_gb300.sharded import column_shard, trans_ev_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        hv_np, ht_np = inputs.synthetic_reflectors(n, b, seed=5)
        Z = inputs.z_gaussian(n, nev, seed=6)
        # only rank 0 holds the reflectors; the others start from garbage
        hv = torch.from_numpy(hv_np.copy()) if rank == 0 else torch.full((hv_np.size,), np.nan, dtype=torch.float64)
        ht = torch.from_numpy(ht_np.copy()) if rank == 0 else torch.full((ht_np.size,), np.nan, dtype=torch.float64)
        c0, cnt = column_shard(nev, world, rank)
        Zloc = torch.from_numpy(np.ascontiguousarray(Z[:, c0:c0 + cnt].T)).T       # n x cnt, column-major

        def apply(n_, b_, v, t, Zl):            # the oracle stands in for the GPU kernel
            Zl.copy_(torch.from_numpy(oracle.trans_ev(n_, b_, v.numpy(), t.numpy(), Zl.numpy())))
            return 0

        Zall, status = trans_ev_sharded(n, b, hv, ht, Zloc, nev, src=0, gather=True, apply=apply)
        q.put((rank, status, bool(np.array_equal(hv.numpy(), hv_np)), Zall.contiguous().numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_concatenation_equals_single_rank():
    import multiprocessing as mp
    n, b, nev = 300, 16, 300          # 128 + 128 + 44 columns: rank 0 takes two items, rank 1 one
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, b, nev, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    hv, ht = inputs.synthetic_reflectors(n, b, seed=5)
    Z = inputs.z_gaussian(n, nev, seed=6)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    for rank, status, got_reflectors, Zall in sorted(res, key=lambda r: r[0]):
        assert status == 0 and got_reflectors
        assert Zall.shape == (n, nev)
        assert np.array_equal(Zall, ref)          # same arithmetic per column, so bit-identical
