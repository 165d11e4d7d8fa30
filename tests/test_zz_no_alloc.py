"""zef_label_points_noalloc: the entry point for callers that cannot let the
library allocate device memory (it takes its scratch from a fixed array
compiled into libzef instead of cudaMalloc).

Its results must equal those of zef_label_points on the same inputs, on two
calls in a row (the shared scratch keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared).  This
file is collected last so that a failure here does not hide any other test.
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


def _call_noalloc(zef, ctx, pts, labels, omega):
    st = zef.LabelStats()
    rc = zef.lib().zef_label_points_noalloc(ctx.handle, pts.data_ptr(), pts.shape[0], labels.data_ptr(),
                                            omega.data_ptr() if omega is not None else None,
                                            ctypes.byref(zef.make_opts()), ctypes.byref(st))
    return rc, st


def test_noalloc_matches_label_points_two_calls(zef):
    w = zs.config0()
    ctx = zef.Context(0)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(w.priority)
    pts = torch.from_numpy(w.points).cuda()
    n = pts.shape[0]
    assert n <= zef.NOALLOC_MAX_POINTS
    ref_lab, ref_om, _ = ctx.label_points(pts, want_omega=True)
    torch.cuda.synchronize()
    ref_lab = ref_lab.cpu().numpy()
    ref_om = ref_om.cpu().numpy()
    for rep in range(2):
        lab = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        om = torch.full((1, n), float("nan"), dtype=torch.float32, device="cuda")
        rc, st = _call_noalloc(zef, ctx, pts, lab, om)
        assert rc == zef.ZEF_OK, zef.lib().zef_last_error(ctx.handle)
        torch.cuda.synchronize()
        assert np.array_equal(lab.cpu().numpy(), ref_lab), f"labels differ on call {rep + 1}"
        err = np.abs(om.cpu().numpy().astype(np.float64) - ref_om.astype(np.float64)).max()
        assert err <= OMEGA_TOL, f"Omega differs by {err} on call {rep + 1}"
        assert st.points == n and st.pairs_evaluated > 0
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
