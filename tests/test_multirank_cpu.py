"""Multi-rank layout on CPU: two gloo ranks (no GPU).  The one data exchange is the
cross-section state of a sample split over the ranks."""
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


def _local_state(w, wn):
    """A rank's cross-section state computed on the host (stands in for the GPU
    accumulation, whose own parity is tested on the GPU): per point (n, mean, M2,
    sum, sum of w'/w), then (n, n with w != 0, sum w)."""
    import numpy as np
    k = wn.shape[1]
    st = np.empty(5 * k + 3)
    nz = w != 0.0
    for j in range(k):
        x = wn[:, j]
        st[5 * j:5 * j + 5] = (x.size, x.mean(), ((x - x.mean()) ** 2).sum(), x.sum(), (x[nz] / w[nz]).sum())
    st[5 * k:] = (w.size, nz.sum(), w.sum())
    return st


def _xsec_worker(rank, world, port, q):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from rexlib import ensure_built
    rex = ensure_built()
    g = np.random.default_rng(5)
    w = g.uniform(0.2, 3.0, 1000)
    w[::97] = 0.0
    wn = w[:, None] * g.lognormal(0.0, 0.3, (1000, 4))
    lo, hi = rdist.shard_range(1000, rank, world)
    st = rdist.allgather_merge_xsec_state(_local_state(w[lo:hi], wn[lo:hi]), 4, rex.xsec_merge_states)
    q.put((rank, st.tolist()))
    dist.destroy_process_group()


def test_cross_section_state_exchange_over_two_gloo_ranks():
    """Each rank holds half of a sample; after the exchange both ranks hold the same
    state, and it gives the oracle's sigma' and dsigma' of the whole sample."""
    import numpy as np
    from oracle import xsec as oracle_xsec
    world = 2
    port = 30500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_xsec_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = np.array(res[0][1]), np.array(res[1][1])
    assert np.array_equal(a, b)
    # sigma' and dsigma' from the merged state, by the formulas of Sec. 3.1.2
    g = np.random.default_rng(5)
    w = g.uniform(0.2, 3.0, 1000)
    w[::97] = 0.0
    wn = w[:, None] * g.lognormal(0.0, 0.3, (1000, 4))
    k = 4
    n, nr, sw = a[5 * k:]
    m = a[:5 * k].reshape(k, 5)
    sig = 2.0 / sw * m[:, 3]
    dsig = 0.1 * m[:, 4] / nr + 2.0 * np.sqrt(m[:, 2] / m[:, 0])
    rs, rds, _ = oracle_xsec.reweighted_xsec(w, wn, 2.0, 0.1)
    assert np.allclose(sig, rs, rtol=1e-13) and np.allclose(dsig, rds, rtol=1e-12)
    assert n == 1000
