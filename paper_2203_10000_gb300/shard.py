"""Multi-GPU use of the labeling path: one process per GPU.

Points are independent units (Sec. 2.1.3: the solid-angle test of a point
needs only the surfaces), so a point set shards into contiguous ranges with no
exchange during labeling; every rank holds a full copy of the surfaces.  The
only collectives are outside the data path: gathering the labels of a sharded
point set and taking the slowest rank's time.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple:
    """Contiguous [start, stop) of rank `rank` among `world` near-equal shards."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def gather_labels(local, n: int, group=None):
    """All-gather the int32 labels of every rank's shard into the full array
    (same device as `local`); every rank receives the result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [shard_range(n, r, world) for r in range(world)]
    longest = max(b - a for a, b in sizes)
    pad = torch.full((longest,), -2, dtype=torch.int32, device=local.device)
    pad[: local.numel()] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: b - a] for p, (a, b) in zip(parts, sizes)])


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
