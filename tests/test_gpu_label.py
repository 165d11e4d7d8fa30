"""GPU parity of zef_label_points against the FP64 oracle (through the C ABI).

Bars: labels bit-exact; Omega within 1e-5 sr of the oracle for every
(point, compartment) pair (pairs outside the compartment's bounding box are
exactly 0 on the GPU); pairs re-evaluated in FP64 match to 1e-6 (the float32
output rounding).  Points on a surface, where the decision itself is
ill-posed, are asserted absent from the seeded inputs.
"""
import math

import numpy as np
import pytest

import zef_synth as zs

pytestmark = pytest.mark.gpu

FOUR_PI = 4.0 * math.pi
OMEGA_TOL = 1e-5

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zef():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10000_gb300 import build
    build.build()
    from paper_2203_10000_gb300 import zef as z
    return z


def make_ctx(zef, surfaces, priority):
    ctx = zef.Context(0)
    for s in surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(priority)
    return ctx


def gpu_label(ctx, pts, **kw):
    p = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).cuda()
    opts = kw.pop("opts", None)
    lab, om, st = ctx.label_points(p, want_omega=True, opts=opts)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), om.cpu().numpy(), st


def assert_parity(lab, om, olab, oom, tol=OMEGA_TOL):
    assert np.array_equal(lab, olab), np.nonzero(lab != olab)[0][:20]
    fin = np.isfinite(oom)
    assert np.all(np.isfinite(om[fin]))
    err = np.abs(om.astype(np.float64)[fin] - oom[fin])
    assert err.max() <= tol, err.max()


def off_surface(oom):
    """No query point may sit within 1e-9 of the threshold (on a surface)."""
    fin = np.isfinite(oom)
    assert np.all(np.abs(oom[fin] - 2 * math.pi) > 1e-9)


# ------------------------------------------------------------------ failure detection
def test_bounded_wait_expires_and_context_survives(zef, oracle_mod):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    assert ctx.wait_probe(50_000_000) == zef.ZEF_ERR_TIMEOUT
    lab, om, st = gpu_label(ctx, w.points[:2048])
    olab, oom = oracle_mod.label_points(w.points[:2048], w.surfaces, w.priority)
    assert_parity(lab, om, olab, oom)


# ------------------------------------------------------------------ FP32 atan2
def test_fp32_atan2_within_atan2f_bound(zef):
    """The label kernel's own atan2 against FP64 atan2, with CUDA's atan2f
    (torch.atan2 on the device) measured on the same float32 inputs: both
    within atan2f's documented maximum error of 3 ulp.  Inputs: log-uniform
    magnitudes over 2^-40..2^40 of both signs, half of them with |y|/|x|
    near 1 (the octant boundary), plus the axes."""
    rng = np.random.default_rng(5)
    n = 1 << 22
    y = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-40, 40, n)
    x = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-40, 40, n)
    m = n // 2
    x[:m] = rng.choice([-1.0, 1.0], m) * np.abs(y[:m]) * (1 + rng.uniform(-0.25, 0.25, m))
    axes_y = [0.0, 0.0, -0.0, -0.0, 1.0, -1.0, 3.0, -3.0, 2.0 ** -40, 1.0]
    axes_x = [1.0, -1.0, 1.0, -1.0, 0.0, 0.0, 3.0, -3.0, 1.0, 2.0 ** -40]
    y = np.concatenate([y, axes_y]).astype(np.float32)
    x = np.concatenate([x, axes_x]).astype(np.float32)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    ty, tx = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    ctx = zef.Context(0)
    ours = ctx.half_angle(ty, tx, torch.empty_like(ty)).cpu().numpy().astype(np.float64)
    cuda = torch.atan2(ty, tx).cpu().numpy().astype(np.float64)
    e_ours = np.abs(ours - ref) / ulp
    e_cuda = np.abs(cuda - ref) / ulp
    print(f"max ulp: kernel atan2 {e_ours.max():.3f}, atan2f {e_cuda.max():.3f}")
    assert e_cuda.max() <= 3.0
    assert e_ours.max() <= 3.0, (e_ours.max(), y[np.argmax(e_ours)], x[np.argmax(e_ours)])
    assert np.array_equal(np.signbit(ours[-10:]), np.signbit(ref[-10:]))
    # a zero pair has no angle: NaN, which the label kernel re-evaluates in FP64
    z = torch.zeros(4, device="cuda")
    assert torch.isnan(ctx.half_angle(z, z.clone(), torch.empty_like(z))).all()


def test_fma_microbenchmark_is_sane(zef):
    """Measured FMA rates: FP32 within reach of 152 SMs x 128 lanes x 2 flop
    at up to 2.07 GHz (80.5 TFLOP/s), FP64 far below FP32 on this part."""
    ctx = zef.Context(0)
    f32, f64 = ctx.fma_rate(False), ctx.fma_rate(True)
    print(f"FMA TFLOP/s: fp32 {f32:.2f}, fp64 {f64:.3f}")
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.3 * nominal < f32 < 1.05 * nominal
    assert 0 < f64 < 0.5 * f32


# ------------------------------------------------------------------ small case
def test_config0_parity(zef, oracle_mod):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab, om, st = gpu_label(ctx, w.points)
    olab, oom = oracle_mod.label_points(w.points, w.surfaces, w.priority)
    off_surface(oom)
    assert_parity(lab, om, olab, oom)
    assert st["pairs_evaluated"] <= st["pairs_nominal"]
    tile = 32 * st["points_per_thread"]   # one warp's tile
    # tiles cover the points inside the surfaces' union box (the others are
    # outside every compartment: winding number 0, no tile)
    v = np.concatenate([s.verts for s in w.surfaces])
    inside = np.all((w.points >= v.min(0)) & (w.points <= v.max(0)), axis=1)
    assert 0 < inside.sum() < len(w.points)
    assert st["work_items"] >= 1 and st["tiles"] == (int(inside.sum()) + tile - 1) // tile
    assert st["kernel_launches"] > 0


def test_config0_host_pointers_match_device(zef):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab_d, om_d, _ = gpu_label(ctx, w.points)
    lab_h, om_h, st = ctx.label_points(w.points, want_omega=True)
    assert isinstance(lab_h, np.ndarray)
    assert np.array_equal(lab_h, lab_d)
    assert np.array_equal(om_h, om_d)


def test_host_buffers_match_device_large(zef, oracle_mod):
    """Host arrays (pageable and pinned, lattice order and shuffled) of over
    2^20 points give the device-pointer labels, which a sample checks
    against the oracle."""
    w = zs.config1(npts_limit=0)
    g = zs.lattice_centroids(60, 10.0 / 3.0, (-100.0, -100.0, -100.0))   # 1,080,000 centroids
    assert g.shape[0] > (1 << 20)
    ctx = make_ctx(zef, w.surfaces, w.priority)
    dev = ctx.label_points(torch.from_numpy(g).cuda(), stats=False)[0].cpu().numpy()
    host = np.empty(g.shape[0], np.int32)
    ctx.label_points(g, labels=host, stats=False)
    assert np.array_equal(host, dev)
    pin = torch.from_numpy(g).pin_memory()
    lab_pin = torch.empty(g.shape[0], dtype=torch.int32).pin_memory()
    ctx.label_points(pin, labels=lab_pin, stats=False)
    assert np.array_equal(lab_pin.numpy(), dev)
    perm = np.random.default_rng(12).permutation(g.shape[0])
    sh = np.ascontiguousarray(g[perm])
    host_sh = np.empty(g.shape[0], np.int32)
    ctx.label_points(sh, labels=host_sh, stats=False)
    assert np.array_equal(host_sh, dev[perm])
    idx = zs.sample_rows(g, 2000, seed=13)
    olab, _ = oracle_mod.label_points(g[idx], w.surfaces, w.priority)
    assert np.array_equal(dev[idx], olab)


@pytest.mark.parametrize("shape", [(256, 4), (256, 2), (128, 2), (128, 4)])
def test_launch_shapes_ragged_tail(zef, oracle_mod, shape):
    w = zs.config0()
    pts = w.points[: len(w.points) - 37]            # several tiles plus a ragged tail
    ctx = make_ctx(zef, w.surfaces, w.priority)
    olab, oom = oracle_mod.label_points(pts, w.surfaces, w.priority)
    for coherence in (True, False):
        opts = zef.make_opts(block_threads=shape[0], points_per_thread=shape[1], coherence=coherence)
        lab, om, st = gpu_label(ctx, pts, opts=opts)
        assert_parity(lab, om, olab, oom)
        assert st["block_threads"] == shape[0] and st["points_per_thread"] == shape[1]
    # evaluated point by point, a point's arithmetic does not depend on the tile shape
    lab2, om2, _ = gpu_label(ctx, pts, opts=zef.make_opts(block_threads=256, points_per_thread=4, coherence=False))
    assert np.array_equal(om, om2) and np.array_equal(lab, lab2)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_kernel_forms_match_oracle(zef, oracle_mod, kernel):
    """Cap trees (0, the default: far patches replaced by their caps), strips
    with grouped complex products (1), strips with one atan2 per triangle (2)."""
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab, om, st = gpu_label(ctx, w.points, opts=zef.make_opts(kernel=kernel))
    olab, oom = oracle_mod.label_points(w.points, w.surfaces, w.priority)
    assert_parity(lab, om, olab, oom)
    surfs = [_sphere(87.0, 12, 3), _sphere(92.0, 12, 2), _sphere(100.0, 12, 1)]
    pts = np.random.default_rng(21).uniform(-110, 110, size=(30000, 3)).astype(np.float32)
    ctx = make_ctx(zef, surfs, [3, 2, 1])
    lab, om, st = gpu_label(ctx, pts, opts=zef.make_opts(kernel=kernel))
    olab, oom = oracle_mod.label_points(pts, surfs, [3, 2, 1])
    assert_parity(lab, om, olab, oom)


def test_point_walk_matches_shared_lists(zef, oracle_mod):
    """Kernel form 0 with every point walking the cap tree for itself (the
    point as a zero-size box) instead of sharing its tile's list: the same
    arithmetic over the point's own leaves and caps, so the labels equal the
    shared-list evaluation and the oracle."""
    w = zs.config1(npts_limit=0)
    g = zs.lattice_centroids(40, 5.0, (-100.0, -100.0, -100.0))   # 320,000 centroids
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab_s, om_s, st_s = gpu_label(ctx, g, opts=zef.make_opts(coherence=False))
    lab_p, om_p, st_p = gpu_label(ctx, g, opts=zef.make_opts(coherence=False, point_walk=True))
    assert st_p["lane_walk_items"] > 0.5 * st_p["tiles"]
    assert np.array_equal(lab_s, lab_p)
    assert np.abs(om_s.astype(np.float64) - om_p).max() <= 2 * OMEGA_TOL
    idx = zs.sample_rows(g, 3000, seed=9)
    olab, oom = oracle_mod.label_points(g[idx], w.surfaces, w.priority)
    assert_parity(lab_p[idx], om_p[:, idx], olab, oom)
    # the flag is validated
    o = zef.make_opts()
    o.flags = 8  # not a label flag
    with pytest.raises(zef.ZefError):
        ctx.label_points(torch.from_numpy(g[:100]).cuda(), opts=o)


def test_autotuned_shape_matches_fixed_shape(zef, oracle_mod):
    """With no shape given the library times its candidate shapes on a
    sample of the call's points and caches the winner; the per-point
    arithmetic does not depend on the shape, so Omega is bit-identical."""
    w = zs.config1(npts_limit=0)
    g = zs.lattice_centroids(40, 5.0, (-100.0, -100.0, -100.0))   # 320,000 centroids
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab_a, om_a, st_a = gpu_label(ctx, g)
    lab_b, om_b, st_b = gpu_label(ctx, g)          # second call: cached choice
    assert (st_a["block_threads"], st_a["points_per_thread"]) in {(256, 4), (256, 2), (128, 4), (128, 2)}
    assert (st_b["block_threads"], st_b["points_per_thread"]) == (st_a["block_threads"],
                                                                  st_a["points_per_thread"])
    lab_f, om_f, _ = gpu_label(ctx, g, opts=zef.make_opts(block_threads=256, points_per_thread=4))
    assert np.array_equal(lab_a, lab_f)
    assert np.abs(om_a.astype(np.float64) - om_f).max() <= 2 * OMEGA_TOL
    idx = zs.sample_rows(g, 3000, seed=6)
    olab, oom = oracle_mod.label_points(g[idx], w.surfaces, w.priority)
    assert_parity(lab_a[idx], om_a[:, idx], olab, oom)


def test_tile_coherence_matches_oracle_and_point_by_point(zef, oracle_mod):
    """Tiles the surface does not cross take the winding number of one
    representative: Omega = 4 pi k exactly there, the labels equal the
    point-by-point evaluation and the oracle."""
    w = zs.config1(npts_limit=0)
    g = zs.lattice_centroids(50, 4.0, (-100.0, -100.0, -100.0))   # 625,000 centroids
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab_c, om_c, st_c = gpu_label(ctx, g, opts=zef.make_opts(coherence=True))
    lab_p, om_p, st_p = gpu_label(ctx, g, opts=zef.make_opts(coherence=False))
    assert np.array_equal(lab_c, lab_p)
    assert np.abs(om_c.astype(np.float64) - om_p).max() <= 2 * OMEGA_TOL
    assert st_c["coherent_pairs"] > 0.3 * len(g) and st_p["coherent_pairs"] == 0
    assert st_c["pairs_evaluated"] < 0.8 * st_p["pairs_evaluated"]
    # every finite Omega is 4 pi k exactly or close to it
    k = np.round(om_c / FOUR_PI)
    assert np.abs(om_c - FOUR_PI * k).max() <= OMEGA_TOL
    idx = zs.sample_rows(g, 4000, seed=8)
    olab, oom = oracle_mod.label_points(g[idx], w.surfaces, w.priority)
    assert_parity(lab_c[idx], om_c[:, idx], olab, oom)


def test_hull_culling_exact_zero_outside(zef, oracle_mod):
    """Points inside a compartment's bounding box but outside its convex hull
    (the box corners of a sphere) get Omega exactly 0 and are labelled 0."""
    s = _sphere(10.0, 16, 1)
    rng = np.random.default_rng(12)
    d = rng.uniform(-1, 1, size=(20000, 3))
    d = d[np.linalg.norm(d, axis=1) > 0.9 * np.sqrt(3)]          # toward the corners
    pts = np.concatenate([(d * 10.0).astype(np.float32),
                          rng.uniform(-9.5, 9.5, size=(4000, 3)).astype(np.float32)])
    ctx = make_ctx(zef, [s], [1])
    lab, om, st = gpu_label(ctx, pts)
    olab, oom = oracle_mod.label_points(pts, [s], [1])
    assert_parity(lab, om, olab, oom)
    corner = np.arange(len(d))
    assert np.all(om[0, corner] == 0.0) and np.all(lab[corner] == 0)


def test_empty_and_tiny_inputs(zef, oracle_mod):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    p = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    lab, om, st = ctx.label_points(p, want_omega=True)
    assert lab.numel() == 0
    for n in (1, 2, 31, 33):
        pts = w.points[:n]
        lab, om, _ = gpu_label(ctx, pts)
        olab, oom = oracle_mod.label_points(pts, w.surfaces, w.priority)
        assert_parity(lab, om, olab, oom)


def _pinched_spheres(freq, radius, cid):
    """Two geodesic spheres that share one vertex (the second is the first
    reflected through its vertex of largest x, orientation restored): a
    closed, oriented surface whose patches have boundary loops through the
    shared vertex twice."""
    u, t = zs.geodesic_sphere(freq)
    va = u * radius
    k = int(np.argmax(va[:, 0]))
    P = va[k]
    vb = 2.0 * P - va
    nb = va.shape[0]
    tb = t[:, [0, 2, 1]] + nb
    tb = np.where(tb == k + nb, k, tb)
    v = np.concatenate([va, vb]).astype(np.float32)
    return zs.Surface(cid, "pinched", v, np.concatenate([t, tb]).astype(np.int32))


@pytest.mark.parametrize("kernel,walk", [(0, False), (0, True), (1, False)])
def test_small_and_pinched_surfaces(zef, oracle_mod, kernel, walk):
    """Surfaces of a single cap-tree leaf (a tetrahedron, a 12-triangle box:
    no caps at all), of a few leaves (a 108-triangle box), and a pinched one
    (two spheres sharing a vertex) against the oracle."""
    tet_v = np.array([[0, 0, 0], [10, 0, 0], [0, 10, 0], [0, 0, 10]], np.float32) + np.float32(-30.0)
    tet_t = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    surfs = [zs.Surface(4, "tet", tet_v, tet_t),
             zs.Surface(3, "box1", *zs.box_surface((5.0, -20.0, -20.0), (17.0, -8.0, -9.0), 1)),
             zs.Surface(2, "box3", *zs.box_surface((-12.0, 6.0, 4.0), (3.0, 19.0, 16.0), 3)),
             _pinched_spheres(3, 9.0, 1)]
    prio = [4, 3, 2, 1]
    rng = np.random.default_rng(31)
    pts = rng.uniform(-32.0, 32.0, size=(40000, 3)).astype(np.float32)
    pts = np.concatenate([pts, surfs[3].verts[rng.integers(0, len(surfs[3].verts), 2000)] *
                          np.float32(0.97)]).astype(np.float32)
    ctx = make_ctx(zef, surfs, prio)
    lab, om, st = gpu_label(ctx, pts, opts=zef.make_opts(kernel=kernel, point_walk=walk))
    olab, oom = oracle_mod.label_points(pts, surfs, prio)
    off_surface(oom)
    assert_parity(lab, om, olab, oom)
    assert np.count_nonzero(lab == 1) > 1000 and np.count_nonzero(lab == 4) > 10


def test_nonfinite_points(zef, oracle_mod):
    """Non-finite points get label -1 and NaN solid angles, points outside
    the surfaces' union box label 0 and Omega 0 (both decided by the key
    pass, outside the sorted order), with and without Omega, from device and
    from host buffers."""
    w = zs.config0()
    pts = w.points[:3000].copy()
    pts[5] = [np.nan, 0, 0]
    pts[77] = [0, np.inf, 0]
    pts[2999] = [0, 0, -np.inf]
    outside = [10, 11, 2998]
    pts[10] = [50, 0, 0]
    pts[11] = [0, -40, 3]
    pts[2998] = [1e30, 1e30, 1e30]
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab, om, st = gpu_label(ctx, pts)
    olab, oom = oracle_mod.label_points(pts, w.surfaces, w.priority)
    assert np.array_equal(lab, olab)
    assert st["nonfinite_points"] == 3
    assert lab[5] == -1 and lab[77] == -1 and lab[2999] == -1
    assert np.all(np.isnan(om[:, [5, 77, 2999]]))
    assert np.all(lab[outside] == 0) and np.all(om[:, outside] == 0)
    fin = np.isfinite(oom)
    assert np.abs(om.astype(np.float64)[fin] - oom[fin]).max() <= OMEGA_TOL
    # labels alone (priority early exit), device and host buffers
    p = torch.from_numpy(pts).cuda()
    lab_d, _, _ = ctx.label_points(p)
    torch.cuda.synchronize()
    lab_h, _, _ = ctx.label_points(pts)
    assert np.array_equal(lab_d.cpu().numpy(), olab) and np.array_equal(lab_h, olab)


def test_deterministic(zef):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    a = gpu_label(ctx, w.points)
    b = gpu_label(ctx, w.points)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_fp64_plain_kernel(zef, oracle_mod):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    pts = w.points[zs.sample_rows(w.points, 8000, seed=4)]
    lab, om, st = gpu_label(ctx, pts, opts=zef.make_opts(precision=zef.ZEF_FP64_PLAIN))
    olab, oom = oracle_mod.label_points(pts, w.surfaces, w.priority)
    assert_parity(lab, om, olab, oom, tol=1e-6)
    assert st["pairs_rescued"] == 0 and st["pairs_evaluated"] > 0


def test_everything_rescued_when_margin_covers_all(zef, oracle_mod):
    # margin > 2 pi marks every evaluated pair uncertain: the FP64
    # re-evaluation alone must then reproduce the oracle
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    pts = w.points[zs.sample_rows(w.points, 4000, seed=5)]
    lab, om, st = gpu_label(ctx, pts, opts=zef.make_opts(margin=7.0))
    olab, oom = oracle_mod.label_points(pts, w.surfaces, w.priority)
    assert_parity(lab, om, olab, oom, tol=1e-6)
    assert st["uncertain_pairs"] > 0 and st["pairs_rescued"] > 0


def test_points_hugging_the_surface_are_rescued(zef, oracle_mod):
    # points a hair inside / outside triangle centroids: the FP32 sign of N
    # is unreliable there, the conditioning test must send them to FP64
    s = zs.config0().surfaces[0]
    v = s.verts.astype(np.float64)
    cen = v[s.tris].mean(1)
    nrm = np.cross(v[s.tris[:, 1]] - v[s.tris[:, 0]], v[s.tris[:, 2]] - v[s.tris[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    pts = []
    for d in (-3e-6, -1e-6, 1e-6, 3e-6):
        pts.append(cen + d * nrm)
    pts = np.concatenate(pts).astype(np.float32)
    ctx = make_ctx(zef, [s], [1])
    lab, om, st = gpu_label(ctx, pts)
    olab, oom = oracle_mod.label_points(pts, [s], [1])
    keep = np.abs(oom[0] - 2 * math.pi) > 1e-9
    assert keep.sum() > len(pts) // 2
    assert np.array_equal(lab[keep], olab[keep])
    assert st["uncertain_pairs"] > 0


def test_fp32_only_mode_runs(zef, oracle_mod):
    w = zs.config0()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab, om, st = gpu_label(ctx, w.points, opts=zef.make_opts(precision=zef.ZEF_FP32_ONLY))
    olab, oom = oracle_mod.label_points(w.points, w.surfaces, w.priority)
    assert st["pairs_rescued"] == 0
    assert np.mean(lab == olab) > 0.999


# ------------------------------------------------------------------ priority
def _sphere(radius, freq, cid, shift=(0.0, 0.0, 0.0)):
    u, t = zs.geodesic_sphere(freq)
    v = (u * radius + np.asarray(shift)).astype(np.float32)
    return zs.Surface(cid, f"r{radius}", v, t.astype(np.int32))


@pytest.mark.parametrize("order", [[3, 2, 1], [1, 2, 3], [2, 3, 1]])
def test_priority_nested_spheres(zef, oracle_mod, order):
    surfs = [_sphere(87.0, 12, 3), _sphere(92.0, 12, 2), _sphere(100.0, 12, 1)]
    rng = np.random.default_rng(8)
    pts = rng.uniform(-110, 110, size=(20000, 3)).astype(np.float32)
    ctx = make_ctx(zef, surfs, order)
    lab, om, _ = gpu_label(ctx, pts)
    olab, oom = oracle_mod.label_points(pts, surfs, order)
    assert_parity(lab, om, olab, oom)


def test_priority_intersecting_spheres(zef, oracle_mod):
    surfs = [_sphere(10.0, 10, 1), _sphere(10.0, 10, 2, shift=(12.0, 0, 0))]
    rng = np.random.default_rng(3)
    pts = rng.uniform(-12, 24, size=(20000, 3)).astype(np.float32)
    for order in ([1, 2], [2, 1]):
        ctx = make_ctx(zef, surfs, order)
        lab, om, _ = gpu_label(ctx, pts)
        olab, oom = oracle_mod.label_points(pts, surfs, order)
        assert_parity(lab, om, olab, oom)
        lens = (np.linalg.norm(pts.astype(np.float64), axis=1) < 9.0) & \
               (np.linalg.norm(pts.astype(np.float64) - [12, 0, 0], axis=1) < 9.0)
        assert lens.sum() > 10 and np.all(lab[lens] == order[0])


# ------------------------------------------------------------------ full-size head workload
@pytest.mark.parametrize("kernel", [0, 1])
def test_config1_full_size_sampled(zef, oracle_mod, kernel):
    """All 5,000,000 centroids of the 2 mm lattice against the three-layer
    head; a seeded sample is checked against the oracle element by element and
    every Omega against the closed-surface invariant."""
    w = zs.config1()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    lab, om, st = gpu_label(ctx, w.points, opts=zef.make_opts(kernel=kernel))
    assert st["points"] == 5_000_000
    # invariant at full size: every Omega is 0 or 4 pi to within 1e-5
    d = np.minimum(np.abs(om), np.abs(om - FOUR_PI))
    assert d.max() <= OMEGA_TOL
    # labels consistent with Omega and priority (rows in priority order)
    inside = om > 2 * math.pi
    first = np.where(inside.any(0), np.argmax(inside, axis=0), -1)
    ids = np.array(w.priority)
    want = np.where(first >= 0, ids[np.maximum(first, 0)], 0)
    assert np.array_equal(lab, want)
    # element-by-element against the oracle on a seeded sample
    idx = zs.sample_rows(w.points, 6000, seed=11)
    olab, oom = oracle_mod.label_points(w.points[idx], w.surfaces, w.priority)
    off_surface(oom)
    assert_parity(lab[idx], om[:, idx], olab, oom)
    assert 0 < st["pairs_evaluated"] < st["pairs_nominal"]
    assert st["uncertain_pairs"] < 0.001 * st["points"]
    if kernel == 0:  # tiles across a jump of the Morton order walk per point
        assert st["lane_walk_items"] >= 1
