"""CPU-only tests of the C-ABI library: it loads, exports every declared
symbol, and its host logic (surface validation, orientation, triangle strips,
priority checks) behaves as documented.  No kernel runs here."""
import os
import re

import numpy as np
import pytest

import zef_synth as zs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zef():
    from paper_2203_10000_gb300 import build
    build.build()
    from paper_2203_10000_gb300 import zef as z
    return z


def _declared_symbols():
    syms = set()
    for h in ("zef.h", "zef_debug.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        syms |= set(re.findall(r"\b(zef_[a-z_]+)\s*\(", txt))
    return sorted(syms)


def test_library_exports_every_declared_symbol(zef):
    syms = _declared_symbols()
    assert "zef_label_points" in syms and "zef_refine_and_relabel" in syms
    assert "zef_compartment_priority" in syms
    for s in syms:
        assert hasattr(zef.lib(), s), s
    assert zef.version() == 1000


def _host_ctx(zef):
    return zef.Context(device=-1)


def test_host_only_context_registers_and_refuses_labeling(zef):
    ctx = _host_ctx(zef)
    s = zs.config0().surfaces[0]
    ctx.add_compartment(1, s.verts, s.tris)
    assert ctx.info() == (1, 1280)
    with pytest.raises(zef.ZefError) as e:
        ctx.label_points(np.zeros((4, 3), np.float32))
    assert e.value.status == zef.ZEF_ERR_NOT_READY
    with pytest.raises(zef.ZefError) as e:
        ctx.label_points_async(np.zeros((4, 3), np.float32), np.zeros(4, np.int32))
    assert e.value.status == zef.ZEF_ERR_NOT_READY
    assert ctx._inflight == []
    ctx.synchronize()   # nothing in flight on a host-only context


def test_async_labeling_argument_checks(zef):
    ctx = _host_ctx(zef)
    pts = np.zeros((4, 3), np.float32)
    with pytest.raises(ValueError):
        ctx.label_points_async(pts, np.zeros(3, np.int32))        # wrong label count
    with pytest.raises(ValueError):
        ctx.label_points_async(pts, np.zeros(4, np.int64))        # wrong label type
    with pytest.raises(ValueError):
        ctx.label_points_async(pts.astype(np.float64), np.zeros(4, np.int32))  # would need a temporary
    s = zs.config0().surfaces[0]
    ctx.add_compartment(1, s.verts, s.tris)
    with pytest.raises(zef.ZefError) as e:   # checks of the library itself
        ctx.label_points_async(pts, np.zeros(4, np.int32), opts=zef.make_opts(kernel=7))
    assert e.value.status in (zef.ZEF_ERR_INVALID_ARG, zef.ZEF_ERR_NOT_READY)


def test_open_surface_rejected(zef):
    ctx = _host_ctx(zef)
    s = zs.config0().surfaces[0]
    with pytest.raises(zef.ZefError) as e:
        ctx.add_compartment(1, s.verts, s.tris[:-1])
    assert e.value.status == zef.ZEF_ERR_SURFACE_NOT_CLOSED


def test_inconsistent_orientation_rejected(zef):
    ctx = _host_ctx(zef)
    s = zs.config0().surfaces[0]
    t = s.tris.copy()
    t[5] = t[5, [0, 2, 1]]
    with pytest.raises(zef.ZefError) as e:
        ctx.add_compartment(1, s.verts, t)
    assert e.value.status == zef.ZEF_ERR_SURFACE_NOT_CLOSED


def test_inward_surface_needs_auto_orient(zef):
    ctx = _host_ctx(zef)
    s = zs.config0().surfaces[0]
    inward = s.tris[:, [0, 2, 1]]
    with pytest.raises(zef.ZefError) as e:
        ctx.add_compartment(1, s.verts, inward)
    assert e.value.status == zef.ZEF_ERR_SURFACE_ORIENTATION
    ctx.add_compartment(2, s.verts, inward, auto_orient=True)
    ent = ctx.strip_entries(0)
    _check_strips(ent, s.verts, s.tris)


def test_argument_errors(zef):
    ctx = _host_ctx(zef)
    s = zs.config0().surfaces[0]
    for cid in (0, -3):
        with pytest.raises(zef.ZefError) as e:
            ctx.add_compartment(cid, s.verts, s.tris)
        assert e.value.status == zef.ZEF_ERR_INVALID_ARG
    bad = s.tris.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(zef.ZefError):
        ctx.add_compartment(1, s.verts, bad)
    nanv = s.verts.copy()
    nanv[3, 1] = np.nan
    with pytest.raises(zef.ZefError):
        ctx.add_compartment(1, nanv, s.tris)
    ctx.add_compartment(1, s.verts, s.tris)
    with pytest.raises(zef.ZefError):
        ctx.add_compartment(1, s.verts, s.tris)   # duplicate id


def test_priority_must_be_permutation(zef):
    ctx = _host_ctx(zef)
    s = zs.config0().surfaces[0]
    ctx.add_compartment(4, s.verts, s.tris)
    ctx.add_compartment(7, (s.verts * 2).astype(np.float32), s.tris)
    ctx.set_priority([7, 4])
    for bad in ([7], [4, 4], [4, 5], [7, 4, 1]):
        with pytest.raises(zef.ZefError) as e:
            ctx.set_priority(bad)
        assert e.value.status == zef.ZEF_ERR_INVALID_ARG


def _check_strips(ent, verts, tris):
    """The strip stream must reproduce every surface triangle exactly once
    with its orientation (as a cyclic vertex sequence) and its normal."""
    v = verts.astype(np.float32)
    key = {tuple(map(float, p)): i for i, p in enumerate(v)}
    assert ent.shape[0] % 16 == 0
    want = {}
    for t in tris:
        i = int(np.argmin(t))
        want[tuple(np.roll(t, -i))] = t
    got = set()
    idx = [key[tuple(map(float, e[:3]))] for e in ent]
    for k in range(2, len(ent)):
        if ent[k, 3] == 0.0:
            # a non-triangle window repeats a vertex (so D >= 0 and N = 0
            # exactly: an identity factor), with zero normal and kappa
            assert ent[k, 7] == 0.0 and np.all(ent[k, 4:7] == 0)
            assert len({idx[k - 2], idx[k - 1], idx[k]}) < 3, k
            continue
        # weight +1: the window order keeps the triangle's orientation; -1: reverses it
        assert ent[k, 3] in (1.0, -1.0)
        a, b, c = idx[k - 2], idx[k - 1], idx[k]
        tri = (a, b, c) if ent[k, 3] == 1.0 else (a, c, b)
        i = int(np.argmin(tri))
        r = tuple(np.roll(tri, -i))
        hit = r if r in want else None
        assert hit is not None, (a, b, c)
        assert hit not in got
        got.add(hit)
        t = want[hit]
        p = v[t].astype(np.float64)
        n = np.cross(p[1] - p[0], p[2] - p[0])
        np.testing.assert_allclose(ent[k, 4:7], n, rtol=1e-6, atol=1e-12 * np.abs(n).max())
        assert ent[k, 7] == pytest.approx(np.linalg.norm(n) / 8192.0, rel=1e-6)
    assert len(got) == len(tris)
    assert ent[0, 3] == 0.0 and ent[1, 3] == 0.0


@pytest.mark.parametrize("which", ["sphere", "torus", "ellipsoid"])
def test_strip_stream_reproduces_triangles(zef, which):
    if which == "sphere":
        s = zs.config0().surfaces[0]
        v, t = s.verts, s.tris
    elif which == "torus":
        v, t = zs.torus(10.0, 3.0, 40, 18, seed=1, amp=0.5)
    else:
        v, t = zs.perturbed_ellipsoid(12, (9.0, 7.0, 5.0), amp=1.0, seed=3)
    ctx = _host_ctx(zef)
    ctx.add_compartment(1, v, t)
    ent = ctx.strip_entries(0)
    _check_strips(ent, v, t)
    n_ent, n_strips = ctx.strip_stats(0)
    assert n_ent == ent.shape[0]
    # strips must pay off: far fewer than one restart per triangle
    assert n_strips < len(t) / 4


def test_strip_efficiency_head_surfaces(zef):
    w = zs.config1(npts_limit=0)
    ctx = _host_ctx(zef)
    for s in w.surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    for i, s in enumerate(w.surfaces):
        n_ent, n_strips = ctx.strip_stats(i)
        # entries = T + 2 strips + padding; overhead under 10 %
        assert n_ent < 1.10 * s.ntris, (s.name, n_ent, s.ntris, n_strips)


def _seg_triangles(e):
    """Triangles (m, 3, 3) of a strip segment (entries (k, 8)), each with its
    own orientation: entry j with weight +-1 closes the window (x[j-2],
    x[j-1], x[j]), reversed when the weight is -1."""
    x = e[:, :3].astype(np.float64)
    out = []
    for j in range(e.shape[0]):
        if abs(e[j, 3]) == 1.0:
            a, b = (j - 2, j - 1) if e[j, 3] > 0 else (j - 1, j - 2)
            out.append(np.stack([x[a], x[b], x[j]]))
    return np.array(out).reshape(-1, 3, 3)


def _tri_omega(oracle_mod, p, tri):
    v = tri.reshape(-1, 3)
    t = np.arange(v.shape[0], dtype=np.int32).reshape(-1, 3)
    return oracle_mod.solid_angle(p, v, t) if t.size else np.zeros(p.shape[0])


def _strip_omega(p, e):
    """Omega of a strip segment evaluated window by window in FP64, as the
    kernel does: a reset entry (weight 2) restarts the window at its vertex,
    every entry's window (a, b, c) adds 2 atan2(N, D) with N = n . (c - p)."""
    om = np.zeros(p.shape[0])
    x = e[:, :3].astype(np.float64)
    n = e[:, 4:7].astype(np.float64)
    for q, pt in enumerate(p):
        a = b = None
        for j in range(e.shape[0]):
            c = x[j] - pt
            if e[j, 3] == 2.0:
                a = b = c
            N = n[j] @ c
            ra, rb, rc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(c)
            D = ra * rb * rc + (a @ b) * rc + (a @ c) * rb + (b @ c) * ra
            om[q] += 2.0 * np.arctan2(N, D)
            a, b = b, c
    return om


@pytest.mark.parametrize("which", ["sphere", "torus", "ellipsoid", "pinched"])
def test_cap_tree_identity(zef, oracle_mod, which):
    """Every node of the library's cap tree: outside the node's box its
    cap's solid angle equals that of its leaves' triangles (FP64 oracle),
    the leaf strips hold every triangle once with its orientation, every
    window that is not a triangle repeats a vertex with a zero normal, and
    the root (the closed surface) has no cap."""
    if which == "sphere":
        s = zs.config0().surfaces[0]
        v, t = s.verts, s.tris
    elif which == "torus":
        v, t = zs.torus(10.0, 3.0, 40, 18, seed=1, amp=0.5)
    elif which == "ellipsoid":
        v, t = zs.perturbed_ellipsoid(16, (9.0, 7.0, 5.0), amp=1.0, seed=3)
    else:
        # two spheres sharing one vertex: patch boundaries through it twice
        u, t0 = zs.geodesic_sphere(4)
        va = u * 9.0
        k = int(np.argmax(va[:, 0]))
        tb = t0[:, [0, 2, 1]] + va.shape[0]
        tb = np.where(tb == k + va.shape[0], k, tb)
        v = np.concatenate([va, 2.0 * va[k] - va]).astype(np.float32)
        t = np.concatenate([t0, tb]).astype(np.int32)
    ctx = _host_ctx(zef)
    ctx.add_compartment(1, v, t)
    boxes, links, ent = ctx.cap_tree(0)
    assert links[0, 5] == 0 and links[0, 7] == 0                 # root: closed, no cap
    leaf = links[:, 0] < 0
    # pre-order: left child next, skip past the subtree (leaves: the next node)
    assert links[0, 8] == len(boxes)
    for k in range(len(boxes)):
        if leaf[k]:
            assert links[k, 8] == k + 1
        else:
            assert links[k, 0] == k + 1 and links[k, 8] == links[links[k, 1], 8]
            assert links[links[k, 0], 8] == links[k, 1]
    assert links[leaf, 6].sum() == t.shape[0] and links[leaf, 6].max() <= 64

    def seg(k, cap):
        b, c = (links[k, 4], links[k, 5]) if cap else (links[k, 2], links[k, 3])
        return ent[b:b + c]

    # segment format: reset first, whole groups of four, identity windows
    for k in range(len(boxes)):
        for cap in ([False, True] if leaf[k] else [True]):
            e = seg(k, cap)
            if e.shape[0] == 0:
                continue
            assert e.shape[0] % 4 == 0 and e[0, 3] == 2.0 and not np.any(e[1:, 3] == 2.0)
            for j in range(e.shape[0]):
                if abs(e[j, 3]) == 1.0:
                    continue
                assert np.all(e[j, 4:8] == 0)
                if j >= 1:
                    w = [e[max(j - 2, 0), :3], e[j - 1, :3], e[j, :3]]
                    assert any(np.array_equal(w[u], w[w2]) for u in range(3) for w2 in range(u + 1, 3))
            tri = _seg_triangles(e)
            assert tri.shape[0] == (links[k, 7] if cap else links[k, 6])
            nn = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
            tw = e[np.abs(e[:, 3]) == 1.0]
            np.testing.assert_allclose(tw[:, 4:7], nn, rtol=1e-5, atol=1e-6 * max(np.abs(nn).max(), 1e-30))
            np.testing.assert_allclose(tw[:, 7], np.linalg.norm(nn, axis=1) / 8192.0, rtol=1e-5)
    # the leaves hold every oriented triangle once
    index = {}
    for i in np.unique(t):  # referenced vertices (the pinched case holds an unused duplicate)
        index.setdefault(tuple(v[i].astype(np.float32).tolist()), int(i))
    got = []
    for k in np.nonzero(leaf)[0]:
        for tr in _seg_triangles(seg(k, False)):
            ids = [index[tuple(np.float32(q).tolist())] for q in tr]
            r = int(np.argmin(ids))
            got.append(tuple(ids[r:] + ids[:r]))
    want = []
    for f in t.tolist():
        r = int(np.argmin(f))
        want.append(tuple(f[r:] + f[:r]))
    assert sorted(got) == sorted(want)
    # entries per triangle (strip overhead): caps are single zigzag strips
    assert links[leaf, 3].sum() <= 2.0 * t.shape[0]
    assert links[:, 5].sum() <= 1.2 * links[:, 7].sum() + 8 * len(boxes)

    rng = np.random.default_rng(7)
    checked = 0

    def leaf_tris(k):
        if leaf[k]:
            return [_seg_triangles(seg(k, False))]
        return leaf_tris(links[k, 0]) + leaf_tris(links[k, 1])

    for k in rng.choice(len(boxes), size=min(40, len(boxes)), replace=False):
        lo, hi = boxes[k, :3].astype(np.float64), boxes[k, 3:].astype(np.float64)
        if links[k, 5] == 0:
            continue
        ext = hi - lo
        # points just outside the box on every side, and farther away
        pts = np.concatenate([lo + rng.uniform(0, 1, (8, 3)) * ext + np.eye(3)[rng.integers(0, 3, 8)] * ext * 1.01,
                              lo - rng.uniform(0.01, 3.0, (8, 3)) * ext.max()])
        outside = np.any((pts < lo) | (pts > hi), axis=1)
        pts = pts[outside]
        a = _tri_omega(oracle_mod, pts, np.concatenate(leaf_tris(k)))
        b = _tri_omega(oracle_mod, pts, _seg_triangles(seg(k, True)))
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-9)
        if checked < 4:
            # the window-by-window evaluation of the strips; N uses the stored
            # float32 normals (relative rounding 2^-24 per component), hence
            # the wider tolerance against the exact triple products
            np.testing.assert_allclose(_strip_omega(pts[:3], seg(k, True)), b[:3], rtol=0, atol=1e-6)
            if leaf[k]:
                np.testing.assert_allclose(_strip_omega(pts[:3], seg(k, False)), a[:3], rtol=0, atol=1e-6)
        checked += 1
    assert checked >= 10
