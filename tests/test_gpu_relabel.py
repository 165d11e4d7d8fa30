"""GPU recursive re-labeling at the tissue boundaries (zef_relabel_boundary,
Sec. 2.1.3 item 2 and Fig. 3) against the oracle's pass-by-pass recursion,
through the C ABI: labels bit-exact and the same (evaluated, changed) counts
in every pass."""
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


def _ctx(zef, surfaces, priority):
    ctx = zef.Context(0)
    for s in surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(priority)
    return ctx


def _box_labels(nodes, lo, hi, cid):
    x = nodes.astype(np.float64)
    return np.where(np.all((x > lo) & (x < hi), axis=1), cid, 0).astype(np.int32)


def _run(ctx, nodes, tets, lab0, passes, where):
    if where == "device":
        lab = torch.from_numpy(lab0.copy()).cuda()
        per, conv = ctx.relabel_boundary(torch.from_numpy(nodes).cuda(), torch.from_numpy(tets).cuda(), lab,
                                         passes)
        return lab.cpu().numpy(), per, conv
    lab = lab0.copy()
    per, conv = ctx.relabel_boundary(nodes, tets, lab, passes)
    return lab, per, conv


@pytest.mark.parametrize("grow", [True, False])
@pytest.mark.parametrize("where", ["device", "host"])
def test_relabel_moving_box(zef, oracle_mod, grow, where):
    from oracle import relabel
    nodes, tets = zs.lattice_5tet(14, 1.0, (-7.5, -7.5, -7.5))
    small = ((-3.0, -2.0, -4.0), (3.0, 2.0, 1.0))
    big = ((-5.0, -5.0, -6.0), (6.0, 4.0, 4.0))
    b0, b1 = (small, big) if grow else (big, small)
    lab0 = _box_labels(nodes, *b0, 1)
    surf = zs.Surface(1, "box", *zs.box_surface(*b1, 2))
    ctx = _ctx(zef, [surf], [1])
    lab, per, conv = _run(ctx, nodes, tets, lab0, 20, where)
    olab, oper, oconv = relabel.relabel_boundary(nodes, tets, lab0, [surf], [1], 20)
    assert np.array_equal(lab, olab)
    assert per == oper and conv == oconv and conv
    assert np.array_equal(lab, _box_labels(nodes, *b1, 1))
    # the pass limit stops the recursion early, identically on both sides
    lab1, per1, conv1 = _run(ctx, nodes, tets, lab0, 2, where)
    olab1, oper1, oconv1 = relabel.relabel_boundary(nodes, tets, lab0, [surf], [1], 2)
    assert np.array_equal(lab1, olab1) and per1 == oper1 and not conv1 and not oconv1
    # the cached graph gives the same result on a second call
    lab2, per2, _ = _run(ctx, nodes, tets, lab0, 20, where)
    assert np.array_equal(lab2, olab) and per2 == oper


def test_relabel_head_moved_nodes(zef, oracle_mod):
    """Three-layer head, 6 mm five-tet lattice (42,875 nodes): labels of the
    regular nodes, then every node moved by up to 0.4 of a lattice step
    (seeded), as smoothing would; the boundary recursion repairs the labels
    pass by pass like the oracle's."""
    from oracle import relabel
    w = zs.config1(npts_limit=0)
    nodes, tets = zs.lattice_5tet(34, 6.0, (-102.0, -102.0, -102.0))
    lab0, _ = oracle_mod.label_points(nodes, w.surfaces, w.priority)
    rng = np.random.default_rng(31)
    moved = (nodes + rng.uniform(-2.4, 2.4, nodes.shape)).astype(np.float32)
    ctx = _ctx(zef, w.surfaces, w.priority)
    lab, per, conv = _run(ctx, moved, tets, lab0, 64, "device")
    olab, oper, oconv = relabel.relabel_boundary(moved, tets, lab0, w.surfaces, w.priority, 64)
    assert per == oper and conv == oconv and conv
    assert np.array_equal(lab, olab)
    assert sum(c for _, c in per) > 100


def test_relabel_errors_keep_context(zef, oracle_mod):
    nodes, tets = zs.lattice_5tet(6, 1.0, (-3.5, -3.5, -3.5))
    surf = zs.Surface(1, "box", *zs.box_surface((-2.0, -2.0, -2.0), (2.0, 1.0, 2.0), 1))
    ctx = _ctx(zef, [surf], [1])
    lab0 = np.zeros(nodes.shape[0], np.int32)
    lab0[:10] = 1
    for bad_passes in (0, 2000):
        with pytest.raises(zef.ZefError) as e:
            ctx.relabel_boundary(nodes, tets, lab0.copy(), bad_passes)
        assert e.value.status == zef.ZEF_ERR_INVALID_ARG
    t2 = tets.copy()
    t2[3, 1] = -1
    with pytest.raises(zef.ZefError) as e:
        ctx.relabel_boundary(nodes, t2, lab0.copy(), 8)
    assert e.value.status == zef.ZEF_ERR_INVALID_ARG
    # mixed host / device arrays
    with pytest.raises(zef.ZefError) as e:
        ctx.relabel_boundary(torch.from_numpy(nodes).cuda(), tets, lab0.copy(), 8)
    assert e.value.status == zef.ZEF_ERR_INVALID_ARG
    from oracle import relabel
    lab = lab0.copy()
    per, conv = ctx.relabel_boundary(nodes, tets, lab, 8)
    olab, oper, oconv = relabel.relabel_boundary(nodes, tets, lab0, [surf], [1], 8)
    assert np.array_equal(lab, olab) and per == oper and conv == oconv
