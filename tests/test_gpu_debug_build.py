"""The debug build of the library (ZEF_DEBUG_BOUNDS): its kernels check every
index they compute before they use it -- cap-tree nodes and segment ranges of
the walks, sorted positions of the scatter and of the classification, work
items, uncertain pairs, the permutation of the resolve -- and a failed check
records ZEF_ERR_BOUNDS instead of touching memory.  On the workloads below
no check may fail, and the labels must equal the release build's.  The debug
library runs in a child process (the binding loads the build that
ZEF_LIBRARY names)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import zef_synth as zs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import zef_synth as zs
from paper_2203_10000_gb300 import zef
assert zef.LIB_PATH.endswith("_build_debug/libzef.so"), zef.LIB_PATH
for cfg, n, out in [(0, 0, sys.argv[2]), (1, 200_000, sys.argv[3]), (4, 300_000, sys.argv[4])]:
    w = zs.make_config(cfg)
    if n:
        c = w.points.shape[0] // 2
        w.points = np.ascontiguousarray(w.points[c - n // 2: c - n // 2 + n])
    ctx = zef.Context(0)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(w.priority)
    pts = torch.from_numpy(w.points).cuda()
    lab, _, st = ctx.label_points(pts)
    ctx.synchronize()                       # raises on ZEF_ERR_BOUNDS
    lab2, om, _ = ctx.label_points(pts, want_omega=True, opts=zef.make_opts(coherence=False))
    ctx.synchronize()
    assert torch.equal(lab, lab2)
    np.save(out, lab.cpu().numpy())
    ctx.close()
print("debug build ok")
'''


def test_debug_build_checks_pass_and_labels_match(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10000_gb300 import build
    lib = build.build(debug=True)
    build.build()
    from paper_2203_10000_gb300 import zef
    outs = [str(tmp_path / f"lab{k}.npy") for k in range(3)]
    env = dict(os.environ, ZEF_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, *outs], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build ok" in r.stdout
    for cfg, n, out in [(0, 0, outs[0]), (1, 200_000, outs[1]), (4, 300_000, outs[2])]:
        w = zs.make_config(cfg)
        if n:
            c = w.points.shape[0] // 2
            w.points = np.ascontiguousarray(w.points[c - n // 2: c - n // 2 + n])
        ctx = zef.Context(0)
        for s in w.surfaces:
            ctx.add_compartment(s.id, s.verts, s.tris)
        ctx.set_priority(w.priority)
        lab, _, _ = ctx.label_points(torch.from_numpy(w.points).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(np.load(out), lab.cpu().numpy()), f"debug and release labels differ (config {cfg})"
        ctx.close()
