"""zef_label_points_async: batches in host memory labelled with their copies
on their own streams (two staging slots in turn) give the labels of the
synchronous call, which is itself held to the FP64 oracle; here the batches
are also checked against the oracle directly on the small head."""
import numpy as np
import pytest

import zef_synth as zs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zef():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10000_gb300 import build
    build.build()
    from paper_2203_10000_gb300 import zef as z
    return z


def make_ctx(zef, w):
    ctx = zef.Context(0)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(w.priority)
    return ctx


def batches(pts, sizes):
    out, o = [], 0
    for k in sizes:
        out.append(np.ascontiguousarray(pts[o:o + k]))
        o += k
    return out


def test_pinned_batches_equal_oracle(zef, oracle_mod):
    """Growing, shrinking and ragged batch sizes (each slot reallocates while
    the other is in flight); pinned inputs and outputs."""
    w = zs.config0()
    ctx = make_ctx(zef, w)
    sizes = [1000, 7001, 20000, 333, 8530]
    parts = batches(w.points, sizes)
    ins = [torch.from_numpy(p).pin_memory() for p in parts]
    outs = [torch.full((p.shape[0],), -7, dtype=torch.int32).pin_memory() for p in parts]
    for a, b in zip(ins, outs):
        ctx.label_points_async(a, b)
    ctx.synchronize()
    got = np.concatenate([o.numpy() for o in outs])
    olab, _ = oracle_mod.label_points(w.points[:sum(sizes)], w.surfaces, w.priority)
    assert np.array_equal(got, olab), np.nonzero(got != olab)[0][:20]


def test_pageable_and_device_mixes_equal_sync(zef):
    """Pageable numpy buffers, device points with host labels, host points
    with device labels, all-device: the synchronous call's labels."""
    w = zs.config1(npts_limit=400_000)
    ctx = make_ctx(zef, w)
    ref = ctx.label_points(torch.from_numpy(w.points).cuda(), stats=False)[0].cpu().numpy()
    parts = batches(w.points, [100_000, 150_000, 150_000])
    offs = np.cumsum([0] + [p.shape[0] for p in parts])
    got = [np.full(p.shape[0], -7, np.int32) for p in parts]
    ctx.label_points_async(parts[0], got[0])                         # pageable both ways
    d1 = torch.from_numpy(parts[1]).cuda()
    ctx.label_points_async(d1, got[1])                               # device in, host out
    l2 = torch.full((parts[2].shape[0],), -7, dtype=torch.int32, device="cuda")
    ctx.label_points_async(torch.from_numpy(parts[2]).pin_memory(), l2)   # host in, device out
    ctx.synchronize()
    got[2] = l2.cpu().numpy()
    for k in range(3):
        assert np.array_equal(got[k], ref[offs[k]:offs[k + 1]]), k
    d_all = torch.from_numpy(w.points).cuda()
    l_all = torch.empty(w.points.shape[0], dtype=torch.int32, device="cuda")
    ctx.label_points_async(d_all, l_all)                             # all device: no copies
    ctx.synchronize()
    assert np.array_equal(l_all.cpu().numpy(), ref)


def test_pipeline_interleaved_with_sync_calls_and_reused_output(zef):
    """A synchronous call between asynchronous ones, and one host output
    buffer written by consecutive calls (the last call's labels remain)."""
    w = zs.config1(npts_limit=300_000)
    ctx = make_ctx(zef, w)
    ref = ctx.label_points(torch.from_numpy(w.points).cuda(), stats=False)[0].cpu().numpy()
    a = torch.from_numpy(np.ascontiguousarray(w.points[:150_000])).pin_memory()
    b = torch.from_numpy(np.ascontiguousarray(w.points[150_000:])).pin_memory()
    out = torch.full((150_000,), -7, dtype=torch.int32).pin_memory()
    other = torch.full((150_000,), -7, dtype=torch.int32).pin_memory()
    for _ in range(3):
        ctx.label_points_async(a, out)
        mid = ctx.label_points(w.points[:1000], stats=False)[0]    # synchronous, host buffers
        assert np.array_equal(mid, ref[:1000])
        ctx.label_points_async(b, other)
        ctx.label_points_async(b, out)
    ctx.synchronize()
    assert np.array_equal(out.numpy(), ref[150_000:])
    assert np.array_equal(other.numpy(), ref[150_000:])
