"""Host-side work partition for several GPUs (one process per GPU).

Particles are independent on the tracking path (no collective element), so
the path shards without any exchange during tracking.  Two partitions are
offered: contiguous slices of one ensemble (strong scaling) and one lattice
error seed per rank (weak scaling, the benchmark's mode).  The only
collective is the final reduction of two scalars for the throughput report.
"""
from __future__ import annotations


def shard_range(n: int, world: int, rank: int):
    """Contiguous slice [lo, hi) of n particles for `rank` of `world`; the
    first n % world ranks get one particle more."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def rank_seed(base_seed: int, rank: int) -> int:
    """Lattice-error seed of a rank in weak-scaling mode."""
    return base_seed + rank


def reduce_throughput(units: float, elapsed_ms: float, device=None):
    """Job throughput over all ranks: sum of units / max of elapsed times.
    Returns (job_units, job_elapsed_ms); a no-op without an initialised
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(elapsed_ms)
    t = torch.tensor([float(units), float(elapsed_ms)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    s = t.clone()
    m = t.clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(s[0]), float(m[1])
