"""Multi-GPU use of the labeling path: one process per GPU.

Points are independent units (Sec. 2.1.3: the solid-angle test of a point
needs only the surfaces), so a point set shards into ranges with no exchange
during labeling; every rank holds a full copy of the surfaces.  The only
collectives are outside the data path: gathering the labels of a sharded
point set and taking the slowest rank's time.

Work per point is far from uniform: a point deep inside one compartment is
decided by a representative or by culling, while a point near a surface is
summed over the triangles near it.  `equal_work_ranges` therefore orders the
points along a Z-order (Morton) curve of the surfaces' union box, cuts the
ordered points into tiles of consecutive points, estimates each tile's work
as the triangle count of the compartments whose bounding box its own box
meets, and splits the cumulative estimate into `world` near-equal contiguous
ranges.  This is host logic only (geometry of boxes); the labeling itself
runs in the library on each rank's GPU.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple:
    """Contiguous [start, stop) of rank `rank` among `world` near-equal shards
    by count."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def _spread3(v: np.ndarray) -> np.ndarray:
    """Bits of v (< 2^10) moved to every third position."""
    v = v.astype(np.uint32) & 0x3FF
    v = (v | (v << 16)) & 0x030000FF
    v = (v | (v << 8)) & 0x0300F00F
    v = (v | (v << 4)) & 0x030C30C3
    v = (v | (v << 2)) & 0x09249249
    return v


def morton_order(points: np.ndarray, lo, hi, bits: int = 10) -> np.ndarray:
    """Indices of `points` ordered along the Z-order curve of the box
    [lo, hi] at `bits` bits per axis (stable within a cell).  Points outside
    the box or with a non-finite coordinate come last, in input order."""
    p = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ext = np.where(hi > lo, hi - lo, 1.0)
    with np.errstate(invalid="ignore"):
        inside = np.all(np.isfinite(p), axis=1) & np.all(p >= lo, axis=1) & np.all(p <= hi, axis=1)
        q = np.clip(np.floor((np.nan_to_num(p) - lo) / ext * (1 << bits)), 0, (1 << bits) - 1)
    q = q.astype(np.uint32)
    key = _spread3(q[:, 0]) | (_spread3(q[:, 1]) << 1) | (_spread3(q[:, 2]) << 2)
    key = np.where(inside, key, np.uint32(0xFFFFFFFF))
    return np.argsort(key, kind="stable")


def tile_work(points_ordered: np.ndarray, comp_lo: np.ndarray, comp_hi: np.ndarray,
              comp_tris: np.ndarray, tile: int = 64, base: float = 64.0) -> np.ndarray:
    """Estimated work of every tile of `tile` consecutive ordered points: the
    sum of the triangle counts of the compartments whose bounding box meets
    the tile's box, plus `base` per tile (the per-point passes)."""
    p = np.asarray(points_ordered, dtype=np.float64).reshape(-1, 3)
    n = p.shape[0]
    if n == 0:
        return np.zeros(0)
    starts = np.arange(0, n, tile)
    fin = np.all(np.isfinite(p), axis=1)
    pl = np.where(fin[:, None], p, np.inf)
    ph = np.where(fin[:, None], p, -np.inf)
    tlo = np.minimum.reduceat(pl, starts, axis=0)
    thi = np.maximum.reduceat(ph, starts, axis=0)
    lo = np.asarray(comp_lo, dtype=np.float64).reshape(-1, 3)
    hi = np.asarray(comp_hi, dtype=np.float64).reshape(-1, 3)
    t = np.asarray(comp_tris, dtype=np.float64).reshape(-1)
    work = np.full(starts.size, float(base))
    for c in range(lo.shape[0]):
        meets = np.all(thi >= lo[c], axis=1) & np.all(tlo <= hi[c], axis=1)
        work += meets * t[c]
    return work


def equal_work_ranges(points: np.ndarray, surfaces, world: int, tile: int = 64):
    """Split a point set into `world` contiguous ranges of its Morton order
    with near-equal estimated work.

    surfaces: objects with .verts (V, 3) and .tris (T, 3).  Returns
    (order, cuts, work): rank r labels points[order[cuts[r]:cuts[r + 1]]];
    cuts fall on tile boundaries; work[r] is the rank's estimate."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lo = np.array([np.min(s.verts, axis=0) for s in surfaces], dtype=np.float64)
    hi = np.array([np.max(s.verts, axis=0) for s in surfaces], dtype=np.float64)
    nt = np.array([s.tris.shape[0] for s in surfaces], dtype=np.float64)
    order = morton_order(points, lo.min(axis=0), hi.max(axis=0))
    n = order.size
    w = tile_work(np.asarray(points)[order], lo, hi, nt, tile)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        k = int(np.searchsorted(cum, total * r / world))   # first tile boundary at or past the share
        cuts.append(min(n, max(cuts[-1], k * tile)))
    cuts.append(n)
    cuts = np.asarray(cuts, dtype=np.int64)
    ranks = [cum[min(len(w), (cuts[r + 1] + tile - 1) // tile)] - cum[cuts[r] // tile] for r in range(world)]
    return order, cuts, np.asarray(ranks)


def gather_sharded(local, order: np.ndarray, cuts: np.ndarray, group=None):
    """All-gather the int32 labels of every rank's range (rank r holds the
    labels of points[order[cuts[r]:cuts[r + 1]]]) into the labels of the
    whole point set in its original order (a torch tensor on local's
    device); every rank receives the result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [int(cuts[r + 1] - cuts[r]) for r in range(world)]
    longest = max(sizes) if sizes else 0
    pad = torch.full((max(1, longest),), -2, dtype=torch.int32, device=local.device)
    pad[: local.numel()] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    full = torch.empty(int(cuts[-1]), dtype=torch.int32, device=local.device)
    idx = torch.from_numpy(np.ascontiguousarray(order, dtype=np.int64)).to(local.device)
    full[idx] = torch.cat([p[:s] for p, s in zip(parts, sizes)])
    return full


def gather_labels(local, n: int, group=None):
    """All-gather the int32 labels of every rank's count-based shard
    (shard_range) into the full array; every rank receives the result."""
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
