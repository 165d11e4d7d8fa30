"""The N > 1 host path on CPU: two gloo ranks shard a point set, label their
shards (with the oracle, on the CPU), gather the labels and reduce the time.
The gathered labels must equal a single-process labeling."""
import os
import socket

import numpy as np
import pytest

from paper_2203_10000_gb300.shard import shard_range


def test_shard_ranges_partition():
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c and b - a >= d - c >= b - a - 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    import zef_synth as zs
    from paper_2203_10000_gb300.shard import gather_labels, max_over_ranks, shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = zs.config0()
        pts = w.points[::7]
        a, b = shard_range(len(pts), rank, world)
        lab, _ = oracle.label_points(pts[a:b], w.surfaces, w.priority, threads=1)
        full = gather_labels(torch.from_numpy(lab), len(pts))
        slowest = max_over_ranks(10.0 * (rank + 1))
        if rank == 0:
            np.save(out, full.numpy())
            with open(out + ".t", "w") as f:
                f.write(str(slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_equals_single_process(tmp_path, oracle_mod):
    import torch.multiprocessing as mp

    import zef_synth as zs
    out = str(tmp_path / "labels.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    w = zs.config0()
    pts = w.points[::7]
    want, _ = oracle_mod.label_points(pts, w.surfaces, w.priority)
    assert np.array_equal(got, want)
    assert float(open(out + ".t").read()) == 20.0
