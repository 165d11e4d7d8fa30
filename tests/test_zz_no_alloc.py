"""zef_label_points_noalloc: the entry point for callers that cannot let the
library allocate device memory (it takes its scratch from a fixed array
compiled into libzef instead of cudaMalloc).

Its results must equal those of zef_label_points on the same inputs, on two
calls in a row (the shared scratch keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared).  The
cases cover the sizing edges of the fixed array: exactly
ZEF_NOALLOC_MAX_POINTS points over several compartments, the plain FP64
kernel (whose (tile, compartment) flags and items live in the array), the
strip kernel forms, and a call without Omega.  The first calls run on a fresh
context, before zef_label_points ever ran on it, and free device memory must
not change across them.  This file is collected last so that a failure here
does not hide any other test.
"""
import ctypes

import numpy as np
import pytest

import zef_synth as zs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
OMEGA_TOL = 1e-5


@pytest.fixture(scope="module")
def zef():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10000_gb300 import build
    build.build()
    from paper_2203_10000_gb300 import zef as z
    return z


def _ctx(zef, w):
    ctx = zef.Context(0)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(w.priority)
    return ctx


def _call_noalloc(zef, ctx, pts, labels, omega, opts=None):
    st = zef.LabelStats()
    o = opts if opts is not None else zef.make_opts()
    rc = zef.lib().zef_label_points_noalloc(ctx.handle, pts.data_ptr(), pts.shape[0], labels.data_ptr(),
                                            omega.data_ptr() if omega is not None else None,
                                            ctypes.byref(o), ctypes.byref(st))
    return rc, st


def _head_sample(n):
    """n points of the three-layer head's 2 mm lattice: the centred window of
    the lattice order (every compartment's box is crossed there)."""
    w = zs.config1()
    c = w.points.shape[0] // 2
    w.points = np.ascontiguousarray(w.points[c - n // 2: c - n // 2 + n])
    return w


def test_noalloc_matches_label_points_two_calls(zef):
    w = zs.config0()
    ctx = _ctx(zef, w)
    pts = torch.from_numpy(w.points).cuda()
    n = pts.shape[0]
    assert n <= zef.NOALLOC_MAX_POINTS
    # the allocation-free calls first, on a fresh context (no work buffers of
    # zef_label_points exist yet): free device memory must not move between
    # them (the first call may load the library's device code)
    outs = []
    labs = [torch.full((n,), -7, dtype=torch.int32, device="cuda") for _ in range(2)]
    oms = [torch.full((1, n), float("nan"), dtype=torch.float32, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for rep in range(2):
        rc, st = _call_noalloc(zef, ctx, pts, labs[rep], oms[rep])
        assert rc == zef.ZEF_OK, zef.lib().zef_last_error(ctx.handle)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert st.points == n and st.pairs_evaluated > 0 and st.kernel_launches > 0
        outs.append((labs[rep].cpu().numpy(), oms[rep].cpu().numpy()))
    assert free[0] == free[1], f"free device memory changed by {free[0] - free[1]} bytes"
    # then the reference on a second context
    ctx2 = _ctx(zef, w)
    ref_lab, ref_om, _ = ctx2.label_points(pts, want_omega=True)
    torch.cuda.synchronize()
    ref_lab = ref_lab.cpu().numpy()
    ref_om = ref_om.cpu().numpy().astype(np.float64)
    for rep, (lab, om) in enumerate(outs):
        assert np.array_equal(lab, ref_lab), f"labels differ on call {rep + 1}"
        err = np.abs(om.astype(np.float64) - ref_om).max()
        assert err <= OMEGA_TOL, f"Omega differs by {err} on call {rep + 1}"
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("case", ["max_points", "fp64_plain", "strip_kernel", "no_omega"])
def test_noalloc_sizing_edges_match_label_points(zef, oracle_mod, case):
    """Multi-compartment head at the largest call size (and the FP64 tiles,
    the strip form, the call without Omega), two calls in a row against
    zef_label_points; a seeded sample also against the FP64 oracle."""
    n = {"max_points": zef.NOALLOC_MAX_POINTS, "fp64_plain": 8192, "strip_kernel": 16384,
         "no_omega": zef.NOALLOC_MAX_POINTS}[case]
    opts = {"fp64_plain": zef.make_opts(precision=zef.ZEF_FP64_PLAIN),
            "strip_kernel": zef.make_opts(kernel=1)}.get(case, zef.make_opts())
    w = _head_sample(n)
    C = len(w.surfaces)
    ctx = _ctx(zef, w)
    pts = torch.from_numpy(w.points).cuda()
    want_omega = case != "no_omega"
    ref_lab, ref_om, _ = ctx.label_points(pts, want_omega=want_omega, opts=opts)
    torch.cuda.synchronize()
    ref_lab = ref_lab.cpu().numpy()
    for rep in range(2):
        lab = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        om = torch.full((C, n), float("nan"), dtype=torch.float32, device="cuda") if want_omega else None
        rc, st = _call_noalloc(zef, ctx, pts, lab, om, opts)
        assert rc == zef.ZEF_OK, zef.lib().zef_last_error(ctx.handle)
        torch.cuda.synchronize()
        lab = lab.cpu().numpy()
        assert np.array_equal(lab, ref_lab), f"labels differ on call {rep + 1}"
        if want_omega:
            err = np.abs(om.cpu().numpy().astype(np.float64) - ref_om.cpu().numpy().astype(np.float64)).max()
            assert err <= OMEGA_TOL, f"Omega differs by {err} on call {rep + 1}"
        assert st.points == n and st.tiles > 0
    idx = zs.sample_rows(w.points, 400, seed=7)
    olab, _ = oracle_mod.label_points(w.points[idx], w.surfaces, w.priority)
    assert np.array_equal(lab[idx], olab)
    assert np.unique(olab).size >= 3       # the sample reaches several compartments
    ctx.close()


def test_noalloc_rejects_oversize_and_host_pointers(zef):
    w = zs.config0()
    ctx = zef.Context(0)
    s = w.surfaces[0]
    ctx.add_compartment(s.id, s.verts, s.tris)
    big = torch.zeros((zef.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    lab = torch.empty(big.shape[0], dtype=torch.int32, device="cuda")
    rc, _ = _call_noalloc(zef, ctx, big, lab, None)
    assert rc == zef.ZEF_ERR_INVALID_ARG
    host = torch.zeros((16, 3), dtype=torch.float32)
    hlab = torch.empty(16, dtype=torch.int32)
    rc, _ = _call_noalloc(zef, ctx, host, hlab, None)
    assert rc == zef.ZEF_ERR_INVALID_ARG
    ctx.close()
