"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against a closed form, an independent formula
(L'Huilier's theorem, signed ray crossings), a geometric invariant or brute
force, so that a dropped term, a wrong sign or index or a transposed operand in
oracle.c fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import zef_synth as zs

HERE = os.path.dirname(os.path.abspath(__file__))
FOUR_PI = 4.0 * math.pi


# ---------------------------------------------------------------- helpers
def lhuilier(p, a, b, c):
    """Solid angle of triangle (a, b, c) seen from p by L'Huilier's theorem on
    the spherical excess, signed by the orientation of (a - p, b - p, c - p)."""
    u = [x - p for x in (a, b, c)]
    u = [x / np.linalg.norm(x) for x in u]

    def ang(x, y):
        return math.atan2(np.linalg.norm(np.cross(x, y)), float(np.dot(x, y)))

    A, B, C = ang(u[1], u[2]), ang(u[0], u[2]), ang(u[0], u[1])
    s = 0.5 * (A + B + C)
    t = math.tan(s / 2) * math.tan((s - A) / 2) * math.tan((s - B) / 2) * math.tan((s - C) / 2)
    E = 4.0 * math.atan(math.sqrt(max(t, 0.0)))
    sign = np.sign(np.dot(u[0], np.cross(u[1], u[2])))
    return sign * E


def ray_winding(points, verts, tris, direction=(0.5773502691896258 + 1e-3 * math.pi,
                                                0.5773502691896258 - 1e-3 * math.e,
                                                0.5773502691896258)):
    """Signed count of crossings of the ray p + s d (s > 0) with the oriented
    triangles (Moller-Trumbore).  For a closed outward surface this is the
    winding number: 1 inside, 0 outside."""
    d = np.asarray(direction, dtype=np.float64)
    d /= np.linalg.norm(d)
    v = verts.astype(np.float64)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    e1, e2 = b - a, c - a
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    nrm = np.cross(e1, e2)
    orient = -np.sign(np.einsum("ij,j->i", nrm, d))   # +1 if the ray leaves through the face
    out = np.zeros(len(points), dtype=np.int64)
    P = np.asarray(points, dtype=np.float64)
    for s in range(0, len(P), 256):
        p = P[s:s + 256]
        tv = p[:, None, :] - a[None, :, :]
        uu = np.einsum("pij,ij->pi", tv, pv) / det
        qv = np.cross(tv, e1[None])
        vv = np.einsum("j,pij->pi", d, qv) / det
        tt = np.einsum("pij,ij->pi", qv, e2) / det
        hit = (uu >= 0) & (vv >= 0) & (uu + vv <= 1) & (tt > 0)
        out[s:s + 256] = -(hit * orient[None, :]).sum(1)
    return out


def load_golden():
    with open(os.path.join(HERE, "golden", "closed_forms.json")) as f:
        return json.load(f)["cases"]


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_closed_forms(oracle_mod, case):
    terms = oracle_mod.triangle_terms(case["point"], case["verts"], case["tris"])
    assert abs(terms.sum() - case["expected_total"]) < 1e-12
    if "expected_each" in case:
        np.testing.assert_allclose(terms, case["expected_each"], rtol=0, atol=1e-12)


def test_lhuilier_random_triangles(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(300):
        tri = rng.uniform(-1, 1, size=(3, 3))
        p = rng.uniform(-2, 2, size=3)
        if min(np.linalg.norm(tri - p, axis=1)) < 0.05:
            continue
        got = oracle_mod.triangle_terms(p, tri, [[0, 1, 2]])[0]
        want = lhuilier(p, *tri)
        assert abs(got - want) < 1e-9, (got, want)


def test_far_small_triangle(oracle_mod):
    # Omega ~ area * cos(theta) / r^2 with relative error O((h / r)^2)
    rng = np.random.default_rng(3)
    for r in (10.0, 100.0, 1000.0):
        h = 1.0
        tri = np.array([[0, 0, 0], [h, 0, 0], [0, h, 0]], dtype=np.float64)
        cen = tri.mean(0)
        dirv = rng.standard_normal(3)
        dirv /= np.linalg.norm(dirv)
        p = cen + r * dirv
        area = 0.5 * h * h
        cos_t = np.dot(np.array([0, 0, 1.0]), cen - p) / r   # normal +z, R = centroid - p
        approx = area * cos_t / r ** 2
        got = oracle_mod.triangle_terms(p, tri, [[0, 1, 2]])[0]
        assert abs(got - approx) <= 2.0 * (h / r) ** 2 * abs(area / r ** 2) + 1e-15


def test_unit_sphere_inside_outside(oracle_mod):
    w = zs.config0()
    s = w.surfaces[0]
    v = s.verts.astype(np.float64)
    a, b, c = v[s.tris[:, 0]], v[s.tris[:, 1]], v[s.tris[:, 2]]
    n = np.cross(b - a, c - a)
    inr = np.min(np.abs(np.einsum("ij,ij->i", n, a)) / np.linalg.norm(n, axis=1))
    outr = np.max(np.linalg.norm(v, axis=1))
    r = np.linalg.norm(w.points.astype(np.float64), axis=1)
    om = oracle_mod.solid_angle(w.points, s.verts, s.tris)
    ins = r < inr
    out = r > outr
    assert ins.sum() > 1000 and out.sum() > 10000
    np.testing.assert_allclose(om[ins], FOUR_PI, atol=1e-11)
    np.testing.assert_allclose(om[out], 0.0, atol=1e-11)


def test_winding_invariant_head_surfaces(oracle_mod):
    w = zs.config1(npts_limit=0)
    pts = zs.lattice_centroids(100, 2.0, (-100.0, -100.0, -100.0))
    pts = pts[zs.sample_rows(pts, 4000, seed=5)]
    for s in w.surfaces:
        om = oracle_mod.solid_angle(pts, s.verts, s.tris)
        k = np.round(om / FOUR_PI)
        assert np.all(np.abs(om - FOUR_PI * k) < 1e-9)
        assert set(np.unique(k)) <= {0.0, 1.0}
        assert (k == 1).sum() > 100


def test_orientation_flip_negates(oracle_mod):
    s = zs.config0().surfaces[0]
    pts = np.random.default_rng(1).uniform(-1.4, 1.4, size=(500, 3))
    a = oracle_mod.solid_angle(pts, s.verts, s.tris)
    b = oracle_mod.solid_angle(pts, s.verts, s.tris[:, [0, 2, 1]])
    np.testing.assert_allclose(b, -a, rtol=0, atol=1e-12)


def test_translation_invariance(oracle_mod):
    s = zs.config0().surfaces[0]
    pts = np.random.default_rng(2).uniform(-1.4, 1.4, size=(300, 3))
    shift = np.array([3.25, -7.5, 11.125])
    a = oracle_mod.solid_angle(pts, s.verts, s.tris)
    b = oracle_mod.solid_angle(pts + shift, s.verts.astype(np.float64) + shift, s.tris)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-11)


def test_triangle_order_only_changes_rounding(oracle_mod):
    s = zs.config0().surfaces[0]
    pts = np.random.default_rng(4).uniform(-1.4, 1.4, size=(300, 3))
    perm = np.random.default_rng(5).permutation(s.tris.shape[0])
    a = oracle_mod.solid_angle(pts, s.verts, s.tris)
    b = oracle_mod.solid_angle(pts, s.verts, s.tris[perm])
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("shape", ["sphere", "torus", "ellipsoid"])
def test_ray_parity_brute_force(oracle_mod, shape):
    rng = np.random.default_rng(11)
    if shape == "sphere":
        s = zs.config0().surfaces[0]
        v, t = s.verts, s.tris
        pts = zs.config0().points[::3]
    elif shape == "torus":
        v, t = zs.torus(10.0, 3.0, 48, 24, seed=1, amp=0.8)
        pts = rng.uniform(-14, 14, size=(6000, 3)).astype(np.float32)
    else:
        v, t = zs.perturbed_ellipsoid(10, (9.0, 7.0, 5.0), amp=1.0, seed=9)
        pts = rng.uniform(-10, 10, size=(6000, 3)).astype(np.float32)
    om = oracle_mod.solid_angle(pts, v, t)
    wind = ray_winding(pts, v, t)
    k = np.round(om / FOUR_PI).astype(np.int64)
    assert np.array_equal(k, wind)
    assert np.array_equal(oracle_mod.inside(om), wind == 1)
    assert 0 < (wind == 1).sum() < len(pts)


# ---------------------------------------------------------------- priority
def _sphere(radius, freq, cid):
    u, t = zs.geodesic_sphere(freq)
    v = (u * radius).astype(np.float32)
    return zs.Surface(cid, f"r{radius}", v, t.astype(np.int32))


def test_priority_nested_ary_spheres(oracle_mod):
    # Ary geometry radii 87 / 92 / 100 (Sec. 2.4); innermost first
    surfs = [_sphere(87.0, 12, 3), _sphere(92.0, 12, 2), _sphere(100.0, 12, 1)]
    rng = np.random.default_rng(8)
    dirs = rng.standard_normal((3000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = rng.uniform(0, 110, size=3000)
    pts = (dirs * radii[:, None]).astype(np.float32)
    lab, om = oracle_mod.label_points(pts, surfs, [3, 2, 1])
    r = np.linalg.norm(pts.astype(np.float64), axis=1)

    def inr(s):
        v = s.verts.astype(np.float64)
        a, b, c = v[s.tris[:, 0]], v[s.tris[:, 1]], v[s.tris[:, 2]]
        n = np.cross(b - a, c - a)
        return np.min(np.abs(np.einsum("ij,ij->i", n, a)) / np.linalg.norm(n, axis=1))

    bounds = [(inr(s), float(np.max(np.linalg.norm(s.verts.astype(np.float64), axis=1))))
              for s in surfs]
    analytic = np.full(len(pts), -9)
    analytic[r > bounds[2][1]] = 0
    analytic[(r < bounds[2][0]) & (r > bounds[1][1])] = 1
    analytic[(r < bounds[1][0]) & (r > bounds[0][1])] = 2
    analytic[r < bounds[0][0]] = 3
    known = analytic != -9
    assert known.sum() > 2500
    assert np.array_equal(lab[known], analytic[known])
    # points in the faceting shells: ray parity decides
    amb = ~known
    want = np.zeros(len(pts), dtype=np.int32)
    for cid, s in zip([3, 2, 1], surfs):
        w = ray_winding(pts[amb], s.verts, s.tris)
        sub = want[amb]
        sub[(sub == 0) & (w == 1)] = cid
        want[amb] = sub
    assert np.array_equal(lab[amb], want[amb])


@pytest.mark.parametrize("order", [[1, 2], [2, 1]])
def test_priority_intersecting_spheres(oracle_mod, order):
    a = _sphere(10.0, 10, 1)
    b = _sphere(10.0, 10, 2)
    b.verts = (b.verts.astype(np.float64) + np.array([12.0, 0, 0])).astype(np.float32)
    rng = np.random.default_rng(3)
    lens = np.column_stack([rng.uniform(4.0, 8.0, 500), rng.uniform(-2, 2, 500),
                            rng.uniform(-2, 2, 500)]).astype(np.float32)
    only_a = np.column_stack([rng.uniform(-8, -2, 300), rng.uniform(-2, 2, 300),
                              rng.uniform(-2, 2, 300)]).astype(np.float32)
    outside = np.column_stack([rng.uniform(30, 40, 300), rng.uniform(-2, 2, 300),
                               rng.uniform(-2, 2, 300)]).astype(np.float32)
    lab, _ = oracle_mod.label_points(np.concatenate([lens, only_a, outside]), [a, b], order)
    assert np.all(lab[:500] == order[0])
    assert np.all(lab[500:800] == 1)
    assert np.all(lab[800:] == 0)


def test_nonfinite_points_get_minus_one(oracle_mod):
    s = zs.config0().surfaces[0]
    pts = np.array([[0, 0, 0], [np.nan, 0, 0], [0, np.inf, 0], [5, 5, 5]], dtype=np.float32)
    lab, om = oracle_mod.label_points(pts, [s], [1])
    assert lab.tolist() == [1, -1, -1, 0]


# ---------------------------------------------------------------- refinement
def _vol(nodes, t):
    a, b, c, d = (nodes[t[i]].astype(np.float64) for i in range(4))
    return float(np.dot(b - a, np.cross(c - a, d - a))) / 6.0


def test_refine_single_tet_one_to_eight():
    from oracle import refine
    nodes = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0], [0, 0, 4], [9, 9, 9]], dtype=np.float32)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    # node 0 differs from the rest: only tet 0 straddles a label boundary
    new_nodes, out, flagged, _ = refine.refine_level(nodes, tets, np.array([1, 2, 2, 2, 2]))
    assert flagged.tolist() == [0]
    assert new_nodes.shape == (6, 3)
    assert out.shape == (2 + 7, 4)
    allnodes = np.concatenate([nodes, new_nodes])
    pv = _vol(nodes, tets[0])
    kids = [out[0]] + [out[2 + i] for i in range(7)]
    vols = [_vol(allnodes, k) for k in kids]
    np.testing.assert_allclose(vols, pv / 8.0, rtol=1e-12)
    assert np.array_equal(out[1], tets[1])
    # every child vertex is a corner or an edge midpoint of the parent
    mids = {tuple(((nodes[i].astype(float) + nodes[j]) / 2)) for i in range(4) for j in range(i + 1, 4)}
    for k in kids:
        for q in k:
            pt = tuple(allnodes[q].astype(float))
            assert q < 4 or pt in mids


def test_refine_plane_split_flag_count(oracle_mod):
    from oracle import refine
    c = 0.37
    L = 50.0
    box_v = np.array([[-L, -L, -L], [c, -L, -L], [c, L, -L], [-L, L, -L],
                      [-L, -L, L], [c, -L, L], [c, L, L], [-L, L, L]], dtype=np.float32)
    box_t = np.array([[0, 3, 2], [0, 2, 1], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                      [2, 3, 7], [2, 7, 6], [1, 2, 6], [1, 6, 5], [0, 4, 7], [0, 7, 3]],
                     dtype=np.int32)
    surf = zs.Surface(1, "box", box_v, box_t)
    nodes, tets = zs.lattice_5tet(6, 1.0, (-3.0, -3.0, -3.0))
    n2, t2, lab, per = refine.refine_and_relabel(nodes, tets, [surf], [1], levels=2)
    # brute force of level 1 from coordinates alone
    x = nodes[:, 0].astype(np.float64)[tets]
    want = int(((x.min(1) < c) & (x.max(1) > c)).sum())
    assert per[0]["flagged"] == want
    assert np.array_equal(lab, np.where(n2[:, 0] < c, 1, 0))
    # conservation of volume
    vol0 = sum(_vol(nodes, t) for t in tets)
    vol2 = sum(_vol(n2, t) for t in t2)
    assert abs(vol0 - vol2) < 1e-9 * vol0
    assert min(_vol(n2, t) for t in t2) > 0
    # level 2 flags exactly the level-1 children that still straddle the plane
    assert per[1]["flagged"] > 0


def test_refine_incremental_labels_equal_full_relabel(oracle_mod):
    from oracle import refine
    s = zs.config0().surfaces[0]
    nodes, tets = zs.lattice_5tet(5, 0.6, (-1.5, -1.5, -1.5))
    n2, t2, lab, per = refine.refine_and_relabel(nodes, tets, [s], [1], levels=2)
    full, _ = oracle_mod.label_points(n2, [s], [1])
    assert np.array_equal(lab, full)
    assert per[0]["new_nodes"] > 0


# ---------------------------------------------------------------- element labels
def _box_elements_case():
    """Three boxes (nested, nested, intersecting) over a 5-tet lattice whose
    nodes sit on integer + 0.5 coordinates and box faces on integers, so no
    node is on a face and insideness is exact by coordinates."""
    boxes = {  # id: (lo, hi, subdivisions)
        1: ((-4.0, -4.0, -4.0), (4.0, 4.0, 4.0), 2),   # outer
        2: ((-2.0, -2.0, -2.0), (2.0, 2.0, 3.0), 1),   # inside 1
        3: ((1.0, -1.0, -1.0), (6.0, 1.0, 2.0), 3),    # crosses 1 and 2
    }
    surfaces = [zs.Surface(i, f"box{i}", *zs.box_surface(lo, hi, m))
                for i, (lo, hi, m) in boxes.items()]
    nodes, tets = zs.lattice_5tet(11, 1.0, (-5.5, -5.5, -5.5))
    return boxes, surfaces, nodes, tets


def _box_brute_force(boxes, priority, nodes, tets):
    x = nodes.astype(np.float64)
    lab = np.zeros(tets.shape[0], dtype=np.int32)
    done = np.zeros(tets.shape[0], dtype=bool)
    for cid in priority:
        lo, hi, _ = boxes[cid]
        inside_node = np.all((x > lo) & (x < hi), axis=1)
        hit = ~done & inside_node[tets].all(axis=1)
        lab[hit] = cid
        done |= hit
    return lab


@pytest.mark.parametrize("priority", [[3, 2, 1], [2, 3, 1], [1, 2, 3]])
def test_element_four_node_rule_boxes(oracle_mod, priority):
    boxes, surfaces, nodes, tets = _box_elements_case()
    elem, node_lab = oracle_mod.label_elements(nodes, tets, surfaces, priority)
    want = _box_brute_force(boxes, priority, nodes, tets)
    assert np.array_equal(elem, want)
    # straddling tets exist and the rule is not "any node inside"
    first = node_lab[tets]
    mixed = (first != first[:, :1]).any(axis=1)
    assert mixed.sum() > 100
    assert np.any(elem[mixed] != first[mixed].max(axis=1))
    # a tet whose nodes share one label needs all four inside that box
    same = ~mixed & (first[:, 0] > 0)
    assert np.array_equal(elem[same], first[same, 0])


def test_element_rule_nonfinite_node(oracle_mod):
    boxes, surfaces, nodes, tets = _box_elements_case()
    nodes = nodes.copy()
    nodes[0] = np.nan
    elem, node_lab = oracle_mod.label_elements(nodes, tets, surfaces, [1, 2, 3])
    has0 = (tets == 0).any(axis=1)
    assert node_lab[0] == -1 and np.all(elem[has0] == -1) and np.all(elem[~has0] >= 0)
    with pytest.raises(ValueError):
        oracle_mod.label_elements(nodes, tets[:4] + 10 ** 6, surfaces, [1, 2, 3])


def test_box_surface_winding(oracle_mod):
    v, t = zs.box_surface((-1.0, -2.0, -3.0), (1.0, 2.0, 3.0), 3)
    assert t.shape == (12 * 9, 3)
    om = oracle_mod.solid_angle(np.array([[0.1, 0.2, 0.3], [5.0, 0, 0]]), v, t)
    assert abs(om[0] - 4 * math.pi) < 1e-12 and abs(om[1]) < 1e-12


# ---------------------------------------------------------------- recursive re-labeling
def _box_labels(nodes, lo, hi, cid):
    x = nodes.astype(np.float64)
    return np.where(np.all((x > lo) & (x < hi), axis=1), cid, 0).astype(np.int32)


@pytest.mark.parametrize("grow", [True, False])
def test_relabel_boundary_moving_box(oracle_mod, grow):
    """Labels of box B0 repaired against box B1 (faces 2-3 lattice steps
    apart): the boundary front reaches every node whose label changed, so the
    result equals the exact coordinate labels of B1, after several passes."""
    from oracle import relabel
    nodes, tets = zs.lattice_5tet(14, 1.0, (-7.5, -7.5, -7.5))
    small = ((-3.0, -2.0, -4.0), (3.0, 2.0, 1.0))
    big = ((-5.0, -5.0, -6.0), (6.0, 4.0, 4.0))
    b0, b1 = (small, big) if grow else (big, small)
    lab0 = _box_labels(nodes, *b0, 1)
    surf = zs.Surface(1, "box", *zs.box_surface(*b1, 2))
    lab, per, conv = relabel.relabel_boundary(nodes, tets, lab0, [surf], [1], 20)
    want = _box_labels(nodes, *b1, 1)
    assert conv
    assert np.array_equal(lab, want)
    assert len(per) >= 3 and per[-1][1] == 0
    assert sum(c for _, c in per) == int((lab0 != want).sum())
    # each node is evaluated at most once
    assert sum(e for e, _ in per) <= nodes.shape[0]


def test_relabel_boundary_fixed_point_and_pass_limit(oracle_mod):
    from oracle import relabel
    nodes, tets = zs.lattice_5tet(12, 1.0, (-6.5, -6.5, -6.5))
    box = ((-3.0, -3.0, -3.0), (3.0, 2.0, 4.0))
    surf = zs.Surface(1, "box", *zs.box_surface(*box, 1))
    exact = _box_labels(nodes, *box, 1)
    lab, per, conv = relabel.relabel_boundary(nodes, tets, exact, [surf], [1], 10)
    assert conv and len(per) == 1 and per[0][0] > 0 and per[0][1] == 0
    assert np.array_equal(lab, exact)
    # a pass limit of one on a moved surface stops before convergence
    lab0 = _box_labels(nodes, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), 1)
    lab, per, conv = relabel.relabel_boundary(nodes, tets, lab0, [surf], [1], 1)
    assert not conv and len(per) == 1 and per[0][1] > 0


def test_relabel_boundary_sphere_equals_full_relabel(oracle_mod):
    from oracle import relabel
    nodes, tets = zs.lattice_5tet(16, 0.5, (-4.0, -4.0, -4.0))
    s0, s1 = _sphere(2.0, 6, 1), _sphere(3.2, 6, 1)
    lab0, _ = oracle_mod.label_points(nodes, [s0], [1])
    lab, per, conv = relabel.relabel_boundary(nodes, tets, lab0, [s1], [1], 20)
    full, _ = oracle_mod.label_points(nodes, [s1], [1])
    assert conv and np.array_equal(lab, full) and len(per) >= 3


# ---------------------------------------------------------------- conforming refinement
def _faces_conform(nodes, tets, lo, hi):
    """Every face is shared by exactly two tets except faces on the domain
    box, which belong to one: no hanging node anywhere."""
    from collections import Counter
    faces = Counter()
    for t in tets:
        a, b, c, d = (int(x) for x in t)
        for f in ((a, b, c), (a, b, d), (a, c, d), (b, c, d)):
            faces[tuple(sorted(f))] += 1
    x = nodes.astype(np.float64)
    for f, k in faces.items():
        if k == 2:
            continue
        if k != 1:
            return False
        p = x[list(f)]
        on_box = any(np.all(p[:, ax] == lo[ax]) or np.all(p[:, ax] == hi[ax]) for ax in range(3))
        if not on_box:
            return False
    return True


def test_conforming_single_red_tet_needs_no_promotion():
    """One red tet in a conforming mesh: every neighbour shares one of its
    edges or one of its faces, both green patterns, so nothing is promoted;
    the result conforms and keeps the volume."""
    from oracle import refine
    nodes, tets = zs.lattice_5tet(3, 1.0, (0.0, 0.0, 0.0))
    labels = np.zeros(nodes.shape[0], np.int32)
    centre = 5 * 13 + 4           # the central tet of the middle cell
    labels[tets[centre][0]] = 1   # one node differs: every tet holding it flags
    flagged = refine.flag_tets(tets, labels)
    red = refine.closure(tets, flagged)
    assert red.sum() >= flagged.sum()
    n1, t1, fl, st = refine.refine_level(nodes, tets, labels, conforming=True)
    allnodes = np.concatenate([nodes, n1])
    assert _faces_conform(allnodes, t1, (0, 0, 0), (3, 3, 3))
    v0 = sum(_vol(nodes, t) for t in tets)
    v1 = [_vol(allnodes, t) for t in t1]
    assert min(v1) > 0 and abs(sum(v1) - v0) < 1e-9 * v0
    # the pattern classes, and a single red tet promotes nothing
    assert refine.green_pattern(0b000001) == ("edge", 0, 1)
    assert refine.green_pattern(0b100001) == "red"          # opposite edges 01, 23
    assert refine.green_pattern(0b001011) == ("face", 0, 1, 2)
    assert refine.green_pattern(0b000111) == "red"          # three edges at vertex 0
    assert refine.green_pattern(0b000011) == ("two", 0, 1, 2)
    red_one = np.zeros(tets.shape[0], bool)
    red_one[centre] = True
    assert refine.closure(tets, red_one).sum() == 1


@pytest.mark.parametrize("levels", [1, 2])
def test_conforming_refinement_of_a_sphere(oracle_mod, levels):
    from oracle import refine
    s = zs.config0().surfaces[0]
    nodes, tets = zs.lattice_5tet(5, 0.6, (-1.5, -1.5, -1.5))
    n2, t2, lab, per = refine.refine_and_relabel(nodes, tets, [s], [1], levels=levels, conforming=True)
    assert _faces_conform(n2, t2, (-1.5, -1.5, -1.5), (1.5, 1.5, 1.5))
    v0 = sum(_vol(nodes, t) for t in tets)
    v2 = [_vol(n2, t) for t in t2]
    assert min(v2) > 0 and abs(sum(v2) - v0) < 1e-9 * v0
    assert all(p["green"] > 0 for p in per)
    # the incremental labels equal a full re-labeling of the final nodes
    full, _ = oracle_mod.label_points(n2, [s], [1])
    assert np.array_equal(lab, full)
    # closure property of the last level: every tet that is not red has an
    # empty or green pattern; every promoted tet has a red pattern from the
    # other red tets alone
    n1, t1, l1, _ = refine.refine_and_relabel(nodes, tets, [s], [1], levels=levels - 1, conforming=True)
    fl = refine.flag_tets(t1, l1)
    red = refine.closure(t1, fl)
    keys = [refine._edge_keys(t) for t in t1]
    split = set(k for i in np.nonzero(red)[0] for k in keys[i])
    for i in range(t1.shape[0]):
        if red[i] and fl[i]:
            continue
        if red[i]:
            others = set(k for j in np.nonzero(red)[0] if j != i for k in keys[j])
            mask = sum(1 << e for e in range(6) if keys[i][e] in others)
            assert refine.green_pattern(mask) == "red"
        else:
            mask = sum(1 << e for e in range(6) if keys[i][e] in split)
            assert refine.green_pattern(mask) != "red"
    # without closure the same level leaves hanging nodes
    n3, t3, _, _ = refine.refine_and_relabel(nodes, tets, [s], [1], levels=levels)
    assert not _faces_conform(n3, t3, (-1.5, -1.5, -1.5), (1.5, 1.5, 1.5))


# ---------------------------------------------------------------- post-processing (Sec. 2.2)
def _edge_sets_brute(tets, n):
    adj = [set() for _ in range(n)]
    for t in tets:
        for a in t:
            for b in t:
                if a != b:
                    adj[int(a)].add(int(b))
    return adj


def test_taubin_step_matches_spectral_factors():
    """One Taubin iteration equals (I - mu M)(I + lambda M) x with
    M = (D + I)^-1 (A - D) from a brute-force adjacency, i.e. every
    eigenvector of M with eigenvalue -k is scaled by (1 - lambda k)(1 + mu k)."""
    from oracle import postprocess as pp
    nodes, tets = zs.lattice_5tet(3, 1.0, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(3)
    x = nodes.astype(np.float64) + rng.normal(0, 0.2, nodes.shape)
    n = x.shape[0]
    adj = _edge_sets_brute(tets, n)
    A = np.zeros((n, n))
    for i, s in enumerate(adj):
        A[i, list(s)] = 1.0
    D = np.diag(A.sum(1))
    M = np.linalg.solve(D + np.eye(n), A - D)
    lam, mu = 0.4, 0.4
    out, it = pp.taubin_smooth(x, tets, lam, mu, xi=10.0, max_iters=1)
    assert it == 1
    want = (np.eye(n) - mu * M) @ ((np.eye(n) + lam * M) @ x)
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)
    w, V = np.linalg.eig(M)
    k = -w.real
    assert np.all(k > -1e-12) and np.all(k < 2.0 + 1e-12)
    c = np.linalg.solve(V, x)                      # modal coordinates
    c2 = np.linalg.solve(V, out)
    factor = ((1 - lam * k) * (1 + mu * k))[:, None]
    np.testing.assert_allclose(c2.real, (factor * c).real, atol=1e-9)


def test_taubin_fixed_nodes_translation_and_stop():
    from oracle import postprocess as pp
    nodes, tets = zs.lattice_5tet(4, 1.0, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(4)
    x = nodes.astype(np.float64) + rng.normal(0, 0.1, nodes.shape)
    fixed = np.any((nodes == 0) | (nodes == 4), axis=1)
    a, ia = pp.taubin_smooth(x, tets, 0.4, 0.4, 0.0, 5, fixed)
    b, ib = pp.taubin_smooth(x + [10.0, -3.0, 7.0], tets, 0.4, 0.4, 0.0, 5, fixed)
    assert ia == ib == 5
    np.testing.assert_allclose(b - [10.0, -3.0, 7.0], a, atol=1e-12)
    assert np.array_equal(a[fixed], x[fixed])
    _, i1 = pp.taubin_smooth(x, tets, 0.4, 0.4, 0.9, 50, fixed)
    assert i1 == 1


def test_inflation_towards_box_faces():
    """Nodes inside a box move along their crossing edges by zeta times the
    distance to the face they cross (exact for axis-aligned planes)."""
    from oracle import postprocess as pp
    nodes, tets = zs.lattice_5tet(6, 1.0, (-3.0, -3.0, -3.0))
    lo, hi = np.array([-1.7, -1.4, -2.3]), np.array([1.6, 1.3, 0.8])
    surf = zs.Surface(1, "box", *zs.box_surface(lo, hi, 1))
    zeta = 0.05
    out, moved = pp.inflate(nodes, tets, surf, zeta)
    x = nodes.astype(np.float64)
    inside = np.all((x > lo) & (x < hi), axis=1)
    edges = pp.unique_edges(tets)
    disp = np.zeros_like(x)
    cnt = np.zeros(len(x))
    for a, b in edges:
        if inside[a] == inside[b]:
            continue
        i, j = (a, b) if inside[a] else (b, a)
        d = x[j] - x[i]
        # first box face crossed along the edge, by coordinates
        ts = []
        for ax in range(3):
            if d[ax] > 0:
                ts.append((hi[ax] - x[i, ax]) / d[ax])
            elif d[ax] < 0:
                ts.append((lo[ax] - x[i, ax]) / d[ax])
        t = min(t for t in ts if t >= 0)
        disp[i] += zeta * t * d
        cnt[i] += 1
    m = cnt > 0
    want = x.copy()
    want[m] += disp[m] / cnt[m, None]
    assert moved == int(m.sum()) > 10
    np.testing.assert_allclose(out, want, atol=1e-12)


# ------------------------------------------------------------------ boundary-surface smoothing (Sec. 2.2.1)
def _block_labels(nodes, tets, lo, hi):
    """Element label 1 for the tets of the lattice cells inside [lo, hi)
    (cell corners on the integer lattice), else 0."""
    c = nodes[tets].astype(np.float64).mean(axis=1)
    cell = np.floor(c)
    return np.all((cell >= lo) & (cell < hi), axis=1).astype(np.int32)


def _faces_brute(tets, labels):
    """Tissue-boundary faces by a dictionary over every tet face."""
    seen = {}
    for t, lab in zip(tets, labels):
        t = [int(v) for v in t]
        for f in ((t[0], t[1], t[2]), (t[0], t[1], t[3]), (t[0], t[2], t[3]), (t[1], t[2], t[3])):
            seen.setdefault(tuple(sorted(f)), []).append(int(lab))
    return sorted(f for f, ls in seen.items() if len(ls) == 2 and ls[0] != ls[1])


def test_boundary_faces_of_a_labeled_block():
    """A block of a x b x c lattice cells labeled 1 in a lattice labeled 0:
    every cell face of the block's surface is split into two triangles by
    the five-tet subdivision, so there are 4 (ab + bc + ca) boundary faces,
    each on one of the block's six planes."""
    from oracle import postprocess as pp
    nodes, tets = zs.lattice_5tet(6, 1.0, (0.0, 0.0, 0.0))
    lo, hi = np.array([1, 2, 1]), np.array([4, 5, 3])
    lab = _block_labels(nodes, tets, lo, hi)
    faces = pp.boundary_faces(tets, lab)
    a, b, c = hi - lo
    assert faces.shape[0] == 4 * (a * b + b * c + c * a)
    assert [tuple(f) for f in faces.tolist()] == _faces_brute(tets, lab)
    x = nodes[faces].astype(np.float64)          # (F, 3 nodes, 3)
    on_plane = np.zeros(faces.shape[0], bool)
    for ax in range(3):
        for v in (lo[ax], hi[ax]):
            on_plane |= np.all(x[:, :, ax] == v, axis=1)
    assert on_plane.all()
    # no boundary where every label is equal
    assert pp.boundary_faces(tets, np.zeros(len(tets), np.int32)).shape[0] == 0


def test_surface_taubin_step_equals_dense_form():
    """One iteration over the boundary graph equals
    (I - mu M)(I + lambda M) x on the boundary nodes, M = (D + I)^-1 (A - D)
    with A the adjacency of the brute-force boundary faces' edges; the other
    nodes keep their positions exactly."""
    from oracle import postprocess as pp
    nodes, tets = zs.lattice_5tet(5, 1.0, (0.0, 0.0, 0.0))
    lab = _block_labels(nodes, tets, np.array([1, 1, 1]), np.array([4, 3, 4]))
    rng = np.random.default_rng(11)
    x = nodes.astype(np.float64) + rng.normal(0, 0.15, nodes.shape)
    faces = _faces_brute(tets, lab)
    n = x.shape[0]
    A = np.zeros((n, n))
    for f in faces:
        for i in f:
            for j in f:
                if i != j:
                    A[i, j] = 1.0
    on = A.sum(1) > 0
    D = np.diag(A.sum(1))
    M = np.linalg.solve(D + np.eye(n), A - D)
    lam, mu = 0.4, 0.4
    out, it, nf = pp.taubin_smooth_surface(x, tets, lab, lam, mu, xi=10.0, max_iters=1)
    assert it == 1 and nf == len(faces)
    want = (np.eye(n) - mu * M) @ ((np.eye(n) + lam * M) @ x)
    np.testing.assert_allclose(out[on], want[on], rtol=0, atol=1e-12)
    assert np.array_equal(out[~on], x[~on])


def test_surface_taubin_keeps_face_planes_and_stops():
    """On the unperturbed lattice a node inside a face of the block, two
    lattice steps or more from the face's edges, has its boundary neighbours
    and theirs in that face's plane through one iteration (forward and
    backward step), so its normal coordinate stays exactly; the block's
    corners move (the boundary shrinks where it bends); translation commutes
    with the smoothing; a large xi stops after one iteration."""
    from oracle import postprocess as pp
    nodes, tets = zs.lattice_5tet(8, 1.0, (0.0, 0.0, 0.0))
    lo, hi = np.array([1, 1, 1]), np.array([7, 7, 6])
    lab = _block_labels(nodes, tets, lo, hi)
    x = nodes.astype(np.float64)
    out, it, _ = pp.taubin_smooth_surface(x, tets, lab, 0.4, 0.4, 0.0, 1)
    assert it == 1
    for ax in range(3):
        others = [k for k in range(3) if k != ax]
        for v in (lo[ax], hi[ax]):
            inner = (x[:, ax] == v) & np.all((x[:, others] >= lo[others] + 2) & (x[:, others] <= hi[others] - 2),
                                             axis=1)
            assert inner.any()
            assert np.array_equal(out[inner, ax], x[inner, ax])
    corner = np.all((x == lo) | (x == hi), axis=1)
    assert corner.sum() == 8 and np.all(np.linalg.norm(out[corner] - x[corner], axis=1) > 1e-3)
    off = ~np.isin(np.arange(len(x)), pp.boundary_faces(tets, lab).ravel())
    assert np.array_equal(out[off], x[off])
    moved, _, _ = pp.taubin_smooth_surface(x + [3.0, -2.0, 5.0], tets, lab, 0.4, 0.4, 0.0, 1)
    np.testing.assert_allclose(moved - [3.0, -2.0, 5.0], out, atol=1e-12)
    _, i1, _ = pp.taubin_smooth_surface(x, tets, lab, 0.4, 0.4, 0.9, 50)
    assert i1 == 1
