"""Host-side logic of multi-GPU runs.

The plan step's units are independent (samples, scenes, closed-loop runs),
so a multi-GPU run is one process per GPU, each planning its own problems
(weak scaling): rank r plans the scene of seed (seed + r).  No data crosses
ranks; the only collectives are a barrier around the timed region and the
maximum of the ranks' times.  A sample-sharded plan step (samples split in
contiguous index ranges) would add one exchange: the minimum of the ranks'
packed (class, cost, index) keys, given here by `min_key`.
"""
import os

import torch


def dist_env():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed, rank):
    return int(seed) + int(rank)


def shard(n, world, rank):
    """Contiguous index range [n0, n0 + count) of rank among world."""
    base, extra = divmod(int(n), int(world))
    n0 = rank * base + min(rank, extra)
    return n0, base + (1 if rank < extra else 0)


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity in a
    single process)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank, world, max_seconds):
    """Units all ranks processed per second of the slowest rank."""
    return float(units_per_rank) * int(world) / float(max_seconds)


def _to_signed(key_u64):
    # order-preserving map of [0, 2^64) onto the signed 64-bit range
    return int(key_u64) - (1 << 63)


def _from_signed(v):
    return int(v) + (1 << 63)


def min_key(key_u64, device=None):
    """Minimum over ranks of an unsigned 64-bit packed key ((dead << 63) |
    (cost bits or T - first_hit) << 32 | sample index)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(key_u64)
    t = torch.tensor([_to_signed(key_u64)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return _from_signed(int(t.item()))
