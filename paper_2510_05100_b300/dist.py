"""Multi-GPU layout for reweighting: event shards per rank.

Events are independent and parameter points are shared, so N GPUs either
reweight N independent batches (weak scaling, what the benchmark runs) or split
one batch into N contiguous event ranges (strong scaling).  The weights need no
collective.  The one exchange on the path is the reweighted cross sections
(Sec. 3.1.2) of a sample spread over the ranks: every rank gathers the others'
accumulated statistics (5k + 3 doubles) and merges them in rank order, so that
every rank ends with the same bits.  Besides that, only timing bookkeeping: a
barrier and a max-reduce of the elapsed time.  Works with any torch.distributed
backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations


def env() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (defaults: 1, 0, 0)."""
    import os
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's own batch in weak scaling."""
    return base_seed + rank


def shard_range(nev: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) event range of ``rank`` when one batch is split over ``world`` ranks."""
    if world < 1 or not 0 <= rank < world or nev < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(nev, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (x itself if not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
    return units_per_rank * world / max_seconds


def allgather_merge_xsec_state(state, k: int, merge, device=None):
    """Gather every rank's cross-section state (numpy, 5k + 3 doubles) and merge them
    in rank order with ``merge(a, b, k)``; the same result on every rank.  With no
    process group (or one rank) returns the state unchanged."""
    import numpy as np
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return np.asarray(state, dtype=np.float64)
    t = torch.as_tensor(np.ascontiguousarray(state, dtype=np.float64), device=device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    out = parts[0].cpu().numpy()
    for p in parts[1:]:
        out = merge(out, p.cpu().numpy(), k)
    return out
