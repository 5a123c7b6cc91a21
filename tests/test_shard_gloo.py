"""The multi-rank path on CPU: two gloo ranks, one process each.

Cells are independent, so ranks share no data: a batch split into contiguous ranges
and integrated rank by rank (here by the FP64 oracle, the GPU being absent) must give
the single-process result cell for cell; the timing reduction takes the slowest rank;
weak scaling gives every rank its own batch.
"""
import os
import socket

import numpy as np
import pytest

from paper_2504_04941_gb300 import inputs as I
from paper_2504_04941_gb300 import shard

WORLD = 2
NCELLS = 37          # odd: the ranges differ in size
DT_SCALE = 1e-2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        wl = I.workload(2, NCELLS)
        lo, hi = shard.contiguous_range(NCELLS, rank, world)
        r = oracle.OracleNetwork(wl.network).integrate(wl.cells.subset(range(lo, hi)), wl.tol.dt * DT_SCALE,
                                                       oracle.options(wl.tol), 1)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, {k: np.asarray(v) for k, v in r.items()}))
        slowest = shard.max_over_ranks(0.25 * (rank + 1))
        total = shard.sum_over_ranks(hi - lo)
        own = I.workload(2, 4, seed=shard.rank_seed(2, rank)).cells.T
        allT = [None] * world
        dist.all_gather_object(allT, own)
        queue.put((rank, parts, slowest, total, allT))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def gathered(oracle_mod):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(WORLD):
        rank, *rest = q.get(timeout=600)
        out[rank] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_contiguous_ranges_tile_the_batch():
    for n in (0, 1, 5, 37, 65536):
        for world in (1, 2, 3, 8):
            ranges = [shard.contiguous_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.contiguous_range(10, 2, 2)


def test_two_ranks_reproduce_the_single_process_result(gathered, oracle_mod):
    parts = gathered[0][0]
    assert gathered[1][0][0][:2] == parts[0][:2]          # both ranks saw the same gather
    wl = I.workload(2, NCELLS)
    ref = oracle_mod.OracleNetwork(wl.network).integrate(wl.cells, wl.tol.dt * DT_SCALE,
                                                         oracle_mod.options(wl.tol), 1)
    for k in ("y", "T", "status", "nsub", "nnewton"):
        got = np.concatenate([np.asarray(p[2][k]) for p in parts], axis=-1)
        assert np.array_equal(got, np.asarray(ref[k])), k


def test_reductions_and_weak_scaling_batches(gathered):
    for rank in range(WORLD):
        _, slowest, total, allT = gathered[rank]
        assert slowest == 0.25 * WORLD                   # max over ranks, seen by every rank
        assert total == NCELLS
        assert not np.array_equal(allT[0], allT[1])      # each rank draws its own batch
    assert np.array_equal(gathered[0][3][1], I.workload(2, 4, seed=shard.rank_seed(2, 1)).cells.T)
    assert shard.weak_throughput(65536, 2, 3, 1.5) == 2 * 65536 * 3 / 1.5
