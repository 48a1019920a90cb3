"""Multi-rank layout on CPU: two gloo ranks (no GPU, no data-path collective)."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_05100_b300 import dist as rdist


def test_shard_ranges_cover_events_disjointly():
    for nev in (0, 1, 7, 1 << 20, 1000003):
        for world in (1, 2, 3, 8):
            rs = [rdist.shard_range(nev, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == nev
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        rdist.shard_range(10, 2, 2)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = rdist.env()
    elapsed = 1.0 + rank            # rank 1 is the slow one
    mx = rdist.max_over_ranks(elapsed)
    seed = rdist.rank_seed(3, r)
    lo, hi = rdist.shard_range(101, r, w)
    dist.barrier()
    q.put((r, w, mx, seed, lo, hi, rdist.job_throughput(1000.0, w, mx)))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling_value():
    world = 2
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 2.0 for r in res)               # max over ranks seen by both
    assert [r[3] for r in res] == [3, 4]               # each rank its own batch
    assert res[0][4:6] == (0, 51) and res[1][4:6] == (51, 101)
    assert all(r[6] == 1000.0 for r in res)            # 2 ranks x 1000 units / 2 s


def test_single_process_defaults():
    assert rdist.max_over_ranks(3.5) == 3.5
    assert rdist.job_throughput(10.0, 1, 2.0) == 5.0
