"""GPU element labels (zef_label_elements: the four-nodes rule of Sec. 2.1.3
under the priority order of Sec. 2.1) against the FP64 oracle, through the
C ABI: element and node labels bit-exact."""
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


def _boxes():
    boxes = {1: ((-4.0, -4.0, -4.0), (4.0, 4.0, 4.0), 2),
             2: ((-2.0, -2.0, -2.0), (2.0, 2.0, 3.0), 1),
             3: ((1.0, -1.0, -1.0), (6.0, 1.0, 2.0), 3)}
    surfaces = [zs.Surface(i, f"box{i}", *zs.box_surface(lo, hi, m)) for i, (lo, hi, m) in boxes.items()]
    nodes, tets = zs.lattice_5tet(11, 1.0, (-5.5, -5.5, -5.5))
    return surfaces, nodes, tets


@pytest.mark.parametrize("priority", [[3, 2, 1], [1, 2, 3]])
@pytest.mark.parametrize("where", ["device", "host"])
def test_elements_boxes(zef, oracle_mod, priority, where):
    surfaces, nodes, tets = _boxes()
    ctx = _ctx(zef, surfaces, priority)
    oel, onl = oracle_mod.label_elements(nodes, tets, surfaces, priority)
    if where == "device":
        el, nl, st = ctx.label_elements(torch.from_numpy(nodes).cuda(), torch.from_numpy(tets).cuda(),
                                        want_node_labels=True)
        torch.cuda.synchronize()
        el, nl = el.cpu().numpy(), nl.cpu().numpy()
    else:
        el, nl, st = ctx.label_elements(nodes, tets, want_node_labels=True)
    assert np.array_equal(nl, onl)
    assert np.array_equal(el, oel)
    assert st["points"] == nodes.shape[0]
    assert {0, 1, 3} <= set(oel.tolist())


def test_elements_head_lattice(zef, oracle_mod):
    """Three-layer head (122,880 triangles) on the 6 mm five-tet lattice:
    42,875 nodes and 196,520 tets, all compared with the oracle."""
    w = zs.config1(npts_limit=0)
    nodes, tets = zs.lattice_5tet(34, 6.0, (-102.0, -102.0, -102.0))
    ctx = _ctx(zef, w.surfaces, w.priority)
    el, nl, st = ctx.label_elements(torch.from_numpy(nodes).cuda(), torch.from_numpy(tets).cuda(),
                                    want_node_labels=True)
    torch.cuda.synchronize()
    oel, onl = oracle_mod.label_elements(nodes, tets, w.surfaces, w.priority)
    assert np.array_equal(nl.cpu().numpy(), onl)
    assert np.array_equal(el.cpu().numpy(), oel)
    # every compartment and the bounding box occur
    assert set(np.unique(oel).tolist()) == {0} | set(w.priority)
    assert st["pairs_evaluated"] > 0


def test_elements_nonfinite_bad_index_empty(zef, oracle_mod):
    surfaces, nodes, tets = _boxes()
    ctx = _ctx(zef, surfaces, [1, 2, 3])
    bad_nodes = nodes.copy()
    bad_nodes[7] = np.inf
    el, nl, _ = ctx.label_elements(bad_nodes, tets, want_node_labels=True)
    oel, onl = oracle_mod.label_elements(bad_nodes, tets, surfaces, [1, 2, 3])
    assert nl[7] == -1 and np.array_equal(el, oel) and np.array_equal(nl, onl)
    # an index outside [0, n_nodes): error, -1 for that tet, context usable
    t2 = tets.copy()
    t2[5, 2] = nodes.shape[0]
    with pytest.raises(zef.ZefError) as e:
        ctx.label_elements(nodes, t2)
    assert e.value.status == zef.ZEF_ERR_INVALID_ARG
    out = np.zeros(t2.shape[0], np.int32)
    with pytest.raises(zef.ZefError):
        ctx.label_elements(nodes, t2, elem_labels=out)
    assert out[5] == -1
    el, _, _ = ctx.label_elements(nodes, tets)
    oel, _ = oracle_mod.label_elements(nodes, tets, surfaces, [1, 2, 3])
    assert np.array_equal(el, oel)
    # no tets: only the nodes are labeled
    el, nl, _ = ctx.label_elements(nodes, np.zeros((0, 4), np.int32), want_node_labels=True)
    assert el.shape == (0,)
    assert np.array_equal(nl, oracle_mod.label_points(nodes, surfaces, [1, 2, 3])[0])
