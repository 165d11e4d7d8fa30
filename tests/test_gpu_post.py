"""GPU post-processing (Sec. 2.2) against the FP64 oracle through the C ABI:
Taubin smoothing of the volume (zef_taubin_smooth) and of the tissue
boundaries (zef_taubin_smooth_surface), and inflation (zef_inflate).

Tolerances: positions are float32; the smoothing sums every node's
neighbours in float32 (a few dozen terms of lattice-sized differences, error
a few ulps of the coordinates per step), so after k iterations of two steps
the nodes agree with the FP64 oracle to 2k x 2^-20 x max|x| (written below as
SMOOTH_TOL); an inflation move is zeta times an edge parameter computed in
float32 (relative error ~2^-20) times the edge, so it agrees to 1e-6 x the
largest coordinate."""
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


def smooth_tol(iters, x):
    return 2 * iters * 2.0 ** -20 * float(np.abs(x).max())


def _perturbed_lattice(n, h, seed, amp):
    nodes, tets = zs.lattice_5tet(n, h, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(seed)
    x = (nodes + rng.uniform(-amp, amp, nodes.shape)).astype(np.float32)
    fixed = np.any((nodes == 0) | (nodes == n * h), axis=1)
    x[fixed] = nodes[fixed]
    return x, tets, fixed


@pytest.mark.parametrize("where", ["device", "host"])
def test_taubin_matches_oracle(zef, where):
    from oracle import postprocess as pp
    x, tets, fixed = _perturbed_lattice(12, 1.0, 5, 0.3)
    ctx = zef.Context(0)
    if where == "device":
        xt = torch.from_numpy(x.copy()).cuda()
        it = ctx.taubin_smooth(xt, torch.from_numpy(tets).cuda(), 0.4, 0.4, 0.0, 10,
                               fixed=torch.from_numpy(fixed.astype(np.uint8)).cuda())
        out = xt.cpu().numpy()
    else:
        out = x.copy()
        it = ctx.taubin_smooth(out, tets, 0.4, 0.4, 0.0, 10, fixed=fixed)
    want, oit = pp.taubin_smooth(x, tets, 0.4, 0.4, 0.0, 10, fixed)
    assert it == oit == 10
    assert np.abs(out - want).max() <= smooth_tol(10, x)
    assert np.array_equal(out[fixed], x[fixed])
    # the smoothing did something: the perturbation shrank
    grid, _ = zs.lattice_5tet(12, 1.0, (0.0, 0.0, 0.0))
    assert np.abs(out - grid).mean() < 0.8 * np.abs(x - grid).mean()


def test_taubin_stop_rule_and_repeat(zef):
    from oracle import postprocess as pp
    x, tets, fixed = _perturbed_lattice(8, 1.0, 6, 0.3)
    ctx = zef.Context(0)
    out = x.copy()
    assert ctx.taubin_smooth(out, tets, 0.4, 0.4, 0.9, 50, fixed=fixed) == 1
    want, oit = pp.taubin_smooth(x, tets, 0.4, 0.4, 0.9, 50, fixed)
    assert oit == 1 and np.abs(out - want).max() <= smooth_tol(1, x)
    # deterministic: a second run gives the same bits
    a, b = x.copy(), x.copy()
    ctx.taubin_smooth(a, tets, 0.4, 0.4, 0.0, 7)
    ctx.taubin_smooth(b, tets, 0.4, 0.4, 0.0, 7)
    assert np.array_equal(a, b)
    with pytest.raises(zef.ZefError):
        ctx.taubin_smooth(x.copy(), tets, 1.5, 0.4, 0.0, 5)
    bad = tets.copy()
    bad[2, 1] = x.shape[0]
    with pytest.raises(zef.ZefError) as e:
        ctx.taubin_smooth(x.copy(), bad, 0.4, 0.4, 0.0, 5)
    assert e.value.status == zef.ZEF_ERR_INVALID_ARG


def test_taubin_head_mesh(zef):
    """The 4 mm head lattice of the refinement workload (132,651 nodes,
    625,000 tets), nodes jittered by 1 mm, 5 iterations."""
    from oracle import postprocess as pp
    w = zs.config3()
    rng = np.random.default_rng(8)
    x = (w.nodes + rng.uniform(-1.0, 1.0, w.nodes.shape)).astype(np.float32)
    ctx = zef.Context(0)
    xt = torch.from_numpy(x.copy()).cuda()
    it = ctx.taubin_smooth(xt, torch.from_numpy(w.tets).cuda(), 0.4, 0.4, 0.0, 5)
    want, oit = pp.taubin_smooth(x, w.tets, 0.4, 0.4, 0.0, 5)
    assert it == oit == 5
    assert np.abs(xt.cpu().numpy() - want).max() <= smooth_tol(5, x)


# ------------------------------------------------------------------ tissue-boundary smoothing
def _block_case(n, lo, hi, seed, amp):
    """Lattice of n^3 cells with element label 2 on the cells inside
    [lo, hi), 1 elsewhere, nodes jittered (the outer boundary kept)."""
    nodes, tets = zs.lattice_5tet(n, 1.0, (0.0, 0.0, 0.0))
    cell = np.floor(nodes[tets].astype(np.float64).mean(axis=1))
    lab = np.where(np.all((cell >= lo) & (cell < hi), axis=1), 2, 1).astype(np.int32)
    rng = np.random.default_rng(seed)
    x = (nodes + rng.uniform(-amp, amp, nodes.shape)).astype(np.float32)
    return x, tets, lab


@pytest.mark.parametrize("where", ["device", "host"])
def test_taubin_surface_matches_oracle(zef, where):
    """A labeled block inside a jittered lattice: boundary faces, iterations
    and positions against the oracle; nodes off the boundary keep their bits."""
    from oracle import postprocess as pp
    x, tets, lab = _block_case(10, np.array([2, 3, 2]), np.array([8, 7, 6]), 9, 0.25)
    ctx = zef.Context(0)
    if where == "device":
        xt = torch.from_numpy(x.copy()).cuda()
        it, nf = ctx.taubin_smooth_surface(xt, torch.from_numpy(tets).cuda(), torch.from_numpy(lab).cuda(),
                                           0.4, 0.4, 0.0, 8)
        out = xt.cpu().numpy()
    else:
        out = x.copy()
        it, nf = ctx.taubin_smooth_surface(out, tets, lab, 0.4, 0.4, 0.0, 8)
    want, oit, onf = pp.taubin_smooth_surface(x, tets, lab, 0.4, 0.4, 0.0, 8)
    assert it == oit == 8
    assert nf == onf == 4 * (6 * 4 + 4 * 4 + 4 * 6)
    assert np.abs(out - want).max() <= smooth_tol(8, x)
    on = np.zeros(len(x), bool)
    on[pp.boundary_faces(tets, lab).ravel()] = True
    assert np.array_equal(out[~on], x[~on])
    assert np.abs(out[on] - x[on]).max() > 1e-3


def test_taubin_surface_head_mesh_and_stop_rule(zef, oracle_mod):
    """Element labels of the 4 mm head lattice (four-nodes rule, through the
    library) define the tissue boundaries; smoothing with the paper's
    xi = 0.1 stops where the oracle does; a labeling without boundaries
    moves nothing."""
    from oracle import postprocess as pp
    w = zs.config3()
    ctx = zef.Context(0)
    for s_ in w.surfaces:
        ctx.add_compartment(s_.id, s_.verts, s_.tris)
    ctx.set_priority(w.priority)
    elem, _, _ = ctx.label_elements(torch.from_numpy(w.nodes).cuda(), torch.from_numpy(w.tets).cuda())
    lab = elem.cpu().numpy()
    olab, _ = oracle_mod.label_elements(w.nodes, w.tets, w.surfaces, w.priority)
    assert np.array_equal(lab, olab)
    rng = np.random.default_rng(12)
    x = (w.nodes + rng.uniform(-1.0, 1.0, w.nodes.shape)).astype(np.float32)
    for xi, cap in ((0.0, 4), (0.1, 100)):
        xt = torch.from_numpy(x.copy()).cuda()
        it, nf = ctx.taubin_smooth_surface(xt, torch.from_numpy(w.tets).cuda(), torch.from_numpy(lab).cuda(),
                                           0.4, 0.4, xi, cap)
        want, oit, onf = pp.taubin_smooth_surface(x, w.tets, lab, 0.4, 0.4, xi, cap)
        assert it == oit and nf == onf > 1000
        assert np.abs(xt.cpu().numpy() - want).max() <= smooth_tol(it, x)
    same = np.zeros(len(w.tets), np.int32)
    y = x.copy()
    assert ctx.taubin_smooth_surface(y, w.tets, same) == (0, 0)
    assert np.array_equal(y, x)


def _inflate_case(zef, surface, nodes, tets, zeta=0.05, where="device"):
    import oracle
    from oracle import postprocess as pp
    ctx = zef.Context(0)
    ctx.add_compartment(surface.id, surface.verts, surface.tris)
    if where == "device":
        xt = torch.from_numpy(nodes.copy()).cuda()
        moved = ctx.inflate(xt, torch.from_numpy(tets).cuda(), surface.id, zeta)
        out = xt.cpu().numpy()
    else:
        out = nodes.copy()
        moved = ctx.inflate(out, tets, surface.id, zeta)
    want, omoved = pp.inflate(nodes, tets, surface, zeta)
    om = oracle.solid_angle(nodes, surface.verts, surface.tris)
    assert np.all(np.abs(om - 2 * np.pi) > 1e-9)        # no node on the surface
    assert moved == omoved > 0
    assert np.abs(out - want).max() <= 1e-6 * float(np.abs(nodes).max())
    unmoved = np.all(want == nodes.astype(np.float64), axis=1)
    assert np.array_equal(out[unmoved], nodes[unmoved])
    return moved


@pytest.mark.parametrize("where", ["device", "host"])
def test_inflate_box(zef, where):
    nodes, tets = zs.lattice_5tet(6, 1.0, (-3.0, -3.0, -3.0))
    surf = zs.Surface(1, "box", *zs.box_surface((-1.7, -1.4, -2.3), (1.6, 1.3, 0.8), 2))
    _inflate_case(zef, surf, nodes, tets, where=where)


def test_inflate_sphere_and_scalp(zef):
    # a generic lattice for the sphere; the head lattice has axis edges that
    # pass exactly through surface vertices (crossings at a shared vertex)
    s = zs.config0().surfaces[0]
    nodes, tets = zs.lattice_5tet(12, 0.25, (-1.4871, -1.5123, -1.4937))
    assert _inflate_case(zef, s, nodes, tets) > 100
    scalp = [t for t in zs.config1(npts_limit=0).surfaces if t.name == "scalp"][0]
    nodes, tets = zs.lattice_5tet(20, 10.0, (-100.0, -100.0, -100.0))
    assert _inflate_case(zef, scalp, nodes, tets) > 100
