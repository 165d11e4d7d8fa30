"""GPU parity of zef_refine_and_relabel (Sec. 2.1.2, Sec. 2.1.3 item 2).

The oracle (oracle/refine.py) numbers new nodes by first appearance and
appends children in flagged order, the same rule the CUDA path implements, so
node coordinates, tet arrays and labels must match exactly.  The full config-3
workload is checked by properties that hold at any size plus a sampled
oracle comparison of node labels.
"""
import math

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


def gpu_refine(zef, ctx, nodes, tets, levels, node_cap, tet_cap, device=True, labels=None):
    N0, M0 = nodes.shape[0], tets.shape[0]
    nd = np.zeros((node_cap, 3), np.float32)
    nd[:N0] = nodes
    td = np.zeros((tet_cap, 4), np.int32)
    td[:M0] = tets
    ld = np.zeros(node_cap, np.int32)
    if labels is not None:
        ld[:N0] = labels
    if device:
        nd_t, td_t, ld_t = (torch.from_numpy(a).cuda() for a in (nd, td, ld))
        n1, m1, per = ctx.refine_and_relabel(nd_t, td_t, ld_t, N0, M0, levels, labels_valid=labels is not None)
        torch.cuda.synchronize()
        return nd_t.cpu().numpy()[:n1], td_t.cpu().numpy()[:m1], ld_t.cpu().numpy()[:n1], per
    n1, m1, per = ctx.refine_and_relabel(nd, td, ld, N0, M0, levels, labels_valid=labels is not None)
    return nd[:n1], td[:m1], ld[:n1], per


def tet_volumes(nodes, tets):
    p = nodes.astype(np.float64)[tets]
    return np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0])) / 6.0


@pytest.mark.parametrize("device", [True, False])
def test_refine_sphere_exact(zef, device):
    from oracle import refine
    w = zs.config0()
    nodes, tets = zs.lattice_5tet(6, 0.5, (-1.5, -1.5, -1.5))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    n1, t1, l1, per = gpu_refine(zef, ctx, nodes, tets, 3, 200_000, 1_000_000, device=device)
    on, ot, ol, oper = refine.refine_and_relabel(nodes, tets, w.surfaces, w.priority, 3)
    assert [p["flagged_tets"] for p in per] == [p["flagged"] for p in oper]
    assert [p["new_nodes"] for p in per] == [p["new_nodes"] for p in oper]
    assert np.array_equal(n1, on)
    assert np.array_equal(t1, ot)
    assert np.array_equal(l1, ol)
    assert per[0]["flagged_tets"] > 0


def test_refine_head_coarse_exact(zef):
    """config-3 surfaces (11 compartments) on a 10 mm lattice, 2 levels."""
    from oracle import refine
    w = zs.config3()
    nodes, tets = zs.lattice_5tet(20, 10.0, (-100.0, -100.0, -100.0))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    n1, t1, l1, per = gpu_refine(zef, ctx, nodes, tets, 2, 400_000, 2_000_000)
    on, ot, ol, oper = refine.refine_and_relabel(nodes, tets, w.surfaces, w.priority, 2)
    assert [p["flagged_tets"] for p in per] == [p["flagged"] for p in oper]
    assert np.array_equal(n1, on)
    assert np.array_equal(t1, ot)
    assert np.array_equal(l1, ol)


def test_refine_config3_full(zef, oracle_mod):
    """The full config-3 workload: 51^3 nodes, 3 levels, labels_valid = 0."""
    w = zs.config3()
    ctx = make_ctx(zef, w.surfaces, w.priority)
    n1, t1, l1, per = gpu_refine(zef, ctx, w.nodes, w.tets, 3, 6_000_000, 16_000_000)
    N0, M0 = w.nodes.shape[0], w.tets.shape[0]
    # counts chain
    n, m = N0, M0
    for p in per:
        assert p["nodes"] == n + p["new_nodes"] and p["tets"] == m + 7 * p["flagged_tets"]
        assert 0 < p["new_nodes"] <= 6 * p["flagged_tets"]
        n, m = p["nodes"], p["tets"]
    assert n1.shape[0] == n and t1.shape[0] == m
    # no duplicate nodes (edge midpoints deduplicated), old nodes untouched
    assert np.unique(n1, axis=0).shape[0] == n1.shape[0]
    assert np.array_equal(n1[:N0], w.nodes)
    # volume conservation, positive children
    vol = tet_volumes(n1, t1)
    assert vol.min() > 0
    assert abs(vol.sum() - 200.0 ** 3) < 1e-6 * 200.0 ** 3
    # the last level leaves no straddling tet among the children it created
    # unflagged: labels of every tet's nodes after refinement are checked below
    idx = np.concatenate([zs.sample_rows(n1[:N0], 1500, seed=1),
                          N0 + zs.sample_rows(n1[N0:], 2500, seed=2)])
    olab, _ = oracle_mod.label_points(n1[idx], w.surfaces, w.priority)
    assert np.array_equal(l1[idx], olab)
    # flag of level k is exactly the set of straddling tets: recount level 1
    lab0 = l1[:N0]
    straddle0 = ~np.all(lab0[w.tets] == lab0[w.tets][:, :1], axis=1)
    assert per[0]["flagged_tets"] == int(straddle0.sum())


def test_refine_capacity_error_keeps_context(zef):
    w = zs.config0()
    nodes, tets = zs.lattice_5tet(6, 0.5, (-1.5, -1.5, -1.5))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    with pytest.raises(zef.ZefError) as e:
        gpu_refine(zef, ctx, nodes, tets, 3, 200_000, tets.shape[0] + 70)
    assert e.value.status == zef.ZEF_ERR_CAPACITY
    # the context still labels correctly afterwards
    lab, _, _ = ctx.label_points(torch.from_numpy(w.points[:1000]).cuda())
    torch.cuda.synchronize()
    assert lab.shape[0] == 1000


def test_refine_rejects_bad_node_index(zef):
    w = zs.config0()
    nodes, tets = zs.lattice_5tet(3, 1.0, (-1.5, -1.5, -1.5))
    bad = tets.copy()
    bad[7, 2] = nodes.shape[0] + 5
    ctx = make_ctx(zef, w.surfaces, w.priority)
    with pytest.raises(zef.ZefError) as e:
        gpu_refine(zef, ctx, nodes, bad, 1, 10_000, 10_000)
    assert e.value.status == zef.ZEF_ERR_INVALID_ARG


def test_refine_repeatable_with_cached_graph(zef):
    w = zs.config0()
    nodes, tets = zs.lattice_5tet(6, 0.5, (-1.5, -1.5, -1.5))
    ctx = make_ctx(zef, w.surfaces, w.priority)
    a = gpu_refine(zef, ctx, nodes, tets, 2, 200_000, 1_000_000)
    b = gpu_refine(zef, ctx, nodes, tets, 2, 200_000, 1_000_000)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert math.isfinite(float(a[0].sum()))
