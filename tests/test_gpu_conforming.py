"""GPU conforming refinement (zef_refine_and_relabel with
ZEF_REFINE_CONFORMING: Sec. 2.1.2 volume refinement plus the one-to-three
edge closure of Fig. 2 c-e) against the oracle: node coordinates, tet arrays,
labels and per-level counts equal, the mesh conforming."""
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


def make_ctx(zef, surfaces, priority):
    ctx = zef.Context(0)
    for s in surfaces:
        ctx.add_compartment(s.id, s.verts, s.tris)
    ctx.set_priority(priority)
    return ctx


def gpu_refine(ctx, nodes, tets, levels, node_cap, tet_cap, device=True):
    N0, M0 = nodes.shape[0], tets.shape[0]
    nd = np.zeros((node_cap, 3), np.float32)
    nd[:N0] = nodes
    td = np.zeros((tet_cap, 4), np.int32)
    td[:M0] = tets
    ld = np.zeros(node_cap, np.int32)
    if device:
        nd_t, td_t, ld_t = (torch.from_numpy(a).cuda() for a in (nd, td, ld))
        n1, m1, per = ctx.refine_and_relabel(nd_t, td_t, ld_t, N0, M0, levels, conforming=True)
        torch.cuda.synchronize()
        return nd_t.cpu().numpy()[:n1], td_t.cpu().numpy()[:m1], ld_t.cpu().numpy()[:n1], per
    n1, m1, per = ctx.refine_and_relabel(nd, td, ld, N0, M0, levels, conforming=True)
    return nd[:n1], td[:m1], ld[:n1], per


def conforms(nodes, tets, lo, hi):
    faces = np.sort(np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]],
                                    tets[:, [1, 2, 3]]]), axis=1)
    uniq, count = np.unique(faces, axis=0, return_counts=True)
    if count.max() > 2:
        return False
    single = uniq[count == 1]
    p = nodes.astype(np.float64)[single]          # (F, 3 vertices, 3)
    on_box = np.zeros(single.shape[0], bool)
    for ax in range(3):
        on_box |= np.all(p[:, :, ax] == lo[ax], axis=1) | np.all(p[:, :, ax] == hi[ax], axis=1)
    return bool(on_box.all())


def volumes(nodes, tets):
    p = nodes.astype(np.float64)[tets]
    return np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0])) / 6.0


def check_levels(per, oper):
    assert [p["flagged_tets"] for p in per] == [p["flagged"] for p in oper]
    assert [p["promoted_tets"] for p in per] == [p["promoted"] for p in oper]
    assert [p["green_tets"] for p in per] == [p["green"] for p in oper]
    assert [p["new_nodes"] for p in per] == [p["new_nodes"] for p in oper]
    assert [p["tets"] for p in per] == [p["tets"] for p in oper]


@pytest.mark.parametrize("device", [True, False])
def test_conforming_sphere_exact(zef, device):
    from oracle import refine
    w = zs.config0()
    nodes, tets = zs.lattice_5tet(6, 0.5, (-1.5, -1.5, -1.5))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    n1, t1, l1, per = gpu_refine(ctx, nodes, tets, 3, 300_000, 2_000_000, device=device)
    on, ot, ol, oper = refine.refine_and_relabel(nodes, tets, w.surfaces, w.priority, 3, conforming=True)
    check_levels(per, oper)
    assert np.array_equal(n1, on)
    assert np.array_equal(t1, ot)
    assert np.array_equal(l1, ol)
    assert conforms(n1, t1, (-1.5, -1.5, -1.5), (1.5, 1.5, 1.5))
    v0 = volumes(nodes, tets).sum()
    v1 = volumes(n1, t1)
    assert v1.min() > 0 and abs(v1.sum() - v0) < 1e-9 * v0
    assert all(p["green_tets"] > 0 for p in per)


def test_conforming_head_exact(zef):
    """Three-layer head on the 20 mm five-tet lattice, two conforming levels."""
    from oracle import refine
    w = zs.config1(npts_limit=0)
    nodes, tets = zs.lattice_5tet(10, 20.0, (-100.0, -100.0, -100.0))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    n1, t1, l1, per = gpu_refine(ctx, nodes, tets, 2, 400_000, 3_000_000)
    on, ot, ol, oper = refine.refine_and_relabel(nodes, tets, w.surfaces, w.priority, 2, conforming=True)
    check_levels(per, oper)
    assert np.array_equal(n1, on)
    assert np.array_equal(t1, ot)
    assert np.array_equal(l1, ol)
    assert conforms(n1, t1, (-100.0, -100.0, -100.0), (100.0, 100.0, 100.0))
    assert sum(p["promoted_tets"] for p in per) > 0


def test_conforming_capacity_error_keeps_context(zef):
    w = zs.config0()
    nodes, tets = zs.lattice_5tet(6, 0.5, (-1.5, -1.5, -1.5))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    # room for the red children but not for the green ones
    from oracle import refine
    _, ot, _, oper = refine.refine_and_relabel(nodes, tets, w.surfaces, w.priority, 1, conforming=True)
    red = oper[0]["flagged"] + oper[0]["promoted"]
    with pytest.raises(zef.ZefError) as e:
        gpu_refine(ctx, nodes, tets, 1, 100_000, tets.shape[0] + 7 * red + 1)
    assert e.value.status == zef.ZEF_ERR_CAPACITY
    # the context still refines afterwards
    n1, t1, l1, per = gpu_refine(ctx, nodes, tets, 1, 100_000, 400_000)
    assert t1.shape[0] == ot.shape[0]
