"""The N > 1 host path on CPU.

One point set is split into contiguous equal-work ranges of its Morton order
(estimated work of a tile of consecutive ordered points: the triangle counts
of the compartments whose bounding box its box meets); two gloo ranks label
their ranges (with the oracle, on the CPU), gather the labels into the
original order and reduce the time.  The gathered labels must equal a
single-process labeling, and the ranks' estimated work must be near-equal."""
import os
import socket

import numpy as np
import pytest

import zef_synth as zs
from paper_2203_10000_gb300.shard import (equal_work_ranges, morton_order, shard_range, tile_work)


def test_shard_ranges_partition():
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c and b - a >= d - c >= b - a - 1


def test_morton_order_is_a_permutation_with_outside_points_last():
    rng = np.random.default_rng(1)
    p = rng.uniform(-2, 2, size=(40000, 3)).astype(np.float32)
    p[17] = np.nan
    order = morton_order(p, (-1, -1, -1), (1, 1, 1))
    assert np.array_equal(np.sort(order), np.arange(p.shape[0]))
    inside = np.all(np.abs(p) <= 1, axis=1)
    k = int(inside.sum())
    assert inside[order[:k]].all() and not inside[order[k:]].any()
    # consecutive points along the curve are close: the mean step is far
    # below that of the (random) input order
    q = p[order[:k]].astype(np.float64)
    r = p[inside].astype(np.float64)
    step = np.linalg.norm(np.diff(q, axis=0), axis=1).mean()
    assert step < 0.25 * np.linalg.norm(np.diff(r, axis=0), axis=1).mean()


def test_equal_work_ranges_balance_the_estimate():
    """Three-layer head, points of a coarse lattice: the work is concentrated
    where the surfaces are, so equal counts are not equal work; the split
    must cover every point once and give each rank about 1 / world of the
    estimated work (within one tile's work)."""
    w = zs.config1()
    pts = w.points[::37]
    for world in (2, 3, 4):
        order, cuts, est = equal_work_ranges(pts, w.surfaces, world, tile=64)
        assert cuts[0] == 0 and cuts[-1] == pts.shape[0] and np.all(np.diff(cuts) >= 0)
        assert np.array_equal(np.sort(order), np.arange(pts.shape[0]))
        assert np.all(cuts[1:-1] % 64 == 0)
        lo = np.array([s.verts.min(0) for s in w.surfaces])
        hi = np.array([s.verts.max(0) for s in w.surfaces])
        tiles = tile_work(pts[order], lo, hi, np.array([s.tris.shape[0] for s in w.surfaces]), 64)
        assert abs(est.sum() - tiles.sum()) < 1e-6 * tiles.sum()
        assert est.max() - est.min() <= 2 * tiles.max()
    # the count split of the same order is unbalanced in work
    order, cuts, est = equal_work_ranges(pts, w.surfaces, 4, tile=64)
    counts = np.diff(cuts)
    assert counts.max() > 1.1 * counts.min()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    import zef_synth as zs
    from paper_2203_10000_gb300.shard import equal_work_ranges, gather_sharded, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload()
        order, cuts, est = equal_work_ranges(w.points, w.surfaces, world, tile=64)
        mine = w.points[order[cuts[rank]:cuts[rank + 1]]]
        lab, _ = oracle.label_points(mine, w.surfaces, w.priority, threads=1)
        full = gather_sharded(torch.from_numpy(lab), order, cuts)
        slowest = max_over_ranks(10.0 * (rank + 1))
        if rank == 0:
            np.save(out, full.numpy())
            np.save(out + ".est.npy", est)
            with open(out + ".t", "w") as f:
                f.write(str(slowest))
    finally:
        dist.destroy_process_group()


def _workload():
    """Two nested spheres and an intersecting third, points of a coarse
    lattice around them (small enough for the oracle on one core)."""
    def sphere(r, f, cid, c=(0.0, 0.0, 0.0)):
        u, t = zs.geodesic_sphere(f)
        return zs.Surface(cid, f"s{cid}", (u * r + np.asarray(c)).astype(np.float32), t.astype(np.int32))
    surfs = [sphere(0.5, 4, 1), sphere(1.0, 6, 2), sphere(0.4, 4, 3, (0.9, 0.0, 0.0))]
    g = np.linspace(-1.3, 1.3, 23)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)
    return zs.Workload("three spheres", surfs, [3, 1, 2], pts)


def test_two_gloo_ranks_gather_equals_single_process(tmp_path, oracle_mod):
    import torch.multiprocessing as mp

    out = str(tmp_path / "labels.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w = _workload()
    want, _ = oracle_mod.label_points(w.points, w.surfaces, w.priority)
    assert np.array_equal(got, want)
    assert set(np.unique(want)) == {0, 1, 2, 3}
    est = np.load(out + ".est.npy")
    assert abs(est[0] - est[1]) <= 0.1 * est.sum()
    assert float(open(out + ".t").read()) == 20.0
