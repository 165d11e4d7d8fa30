"""Oracle of the refine-and-relabel recursion (Sec. 2.1.2 and Sec. 2.1.3 item 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per level, in the paper's order:
  1. the tissue boundary in the mesh is the set of tets whose nodes do not all
     carry the same label; those tets are flagged;
  2. each flagged tet is split into eight ("volume refinement", Fig. 2 a-b):
     one new node at the midpoint of each of its six edges, four corner
     children and the inner octahedron cut along one diagonal;
  3. only the new nodes are labeled with the solid-angle method; old nodes keep
     their labels because their positions do not change.

Readings where the paper is silent:
  * new nodes are numbered in order of first appearance, scanning flagged tets
    by index and each tet's edges in the order 01, 02, 03, 12, 13, 23;
  * a midpoint is (a + b) / 2 rounded once to float32;
  * the octahedron diagonal is the shortest of m01-m23, m02-m13, m03-m12,
    squared lengths evaluated in float32 with one rounding per operation
    (no fused multiply-add), ties to the lower diagonal index;
  * a flagged tet's slot receives child 0; children 1..7 are appended, tet by
    tet in flagged order;
  * the neighbours' 1-3 edge closure (Fig. 2 c-e) is not applied: hanging
    nodes do not affect labeling; the level count is fixed by the caller.
"""
from __future__ import annotations

import numpy as np

from . import label_points

# local nodes: 0..3 corners, 4 = m01, 5 = m02, 6 = m03, 7 = m12, 8 = m13, 9 = m23
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
CORNER_CHILDREN = ((0, 4, 5, 6), (4, 1, 7, 8), (5, 7, 2, 9), (6, 8, 9, 3))
# inner octahedron, one table per diagonal; all children keep the parent's orientation
OCTA_CHILDREN = (
    ((4, 9, 5, 6), (4, 9, 6, 8), (4, 9, 8, 7), (4, 9, 7, 5)),   # diagonal m01-m23
    ((5, 8, 6, 4), (5, 8, 9, 6), (5, 8, 7, 9), (5, 8, 4, 7)),   # diagonal m02-m13
    ((6, 7, 4, 5), (6, 7, 5, 9), (6, 7, 9, 8), (6, 7, 8, 4)),   # diagonal m03-m12
)
DIAGONALS = ((4, 9), (5, 8), (6, 7))


def midpoint_f32(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return ((a.astype(np.float64) + b.astype(np.float64)) * 0.5).astype(np.float32)


def _len2_f32(a: np.ndarray, b: np.ndarray) -> np.float32:
    d = (a.astype(np.float32) - b.astype(np.float32)).astype(np.float32)
    sq = (d * d).astype(np.float32)
    return np.float32(np.float32(sq[0] + sq[1]) + sq[2])


def flag_tets(tets: np.ndarray, node_labels: np.ndarray) -> np.ndarray:
    lab = node_labels[tets]
    return ~np.all(lab == lab[:, :1], axis=1)


def refine_level(nodes: np.ndarray, tets: np.ndarray, node_labels: np.ndarray):
    """One 1->8 split of every flagged tet.  Returns (new_nodes float32 (K, 3),
    new_tets int32, flagged indices)."""
    flagged = np.nonzero(flag_tets(tets, node_labels))[0]
    nn = nodes.shape[0]
    edge_id = {}
    new_pts = []
    local = np.empty((flagged.size, 10), dtype=np.int64)
    for r, ti in enumerate(flagged):
        t = tets[ti]
        local[r, :4] = t
        for e, (i, j) in enumerate(EDGES):
            a, b = int(t[i]), int(t[j])
            key = (a, b) if a < b else (b, a)
            nid = edge_id.get(key)
            if nid is None:
                nid = nn + len(new_pts)
                edge_id[key] = nid
                new_pts.append(midpoint_f32(nodes[key[0]], nodes[key[1]]))
            local[r, 4 + e] = nid
    new_nodes = np.array(new_pts, dtype=np.float32).reshape(-1, 3)
    all_nodes = np.concatenate([nodes, new_nodes]) if new_nodes.size else nodes
    out = np.concatenate([tets, np.zeros((7 * flagged.size, 4), dtype=tets.dtype)])
    m = tets.shape[0]
    for r, ti in enumerate(flagged):
        loc = local[r]
        lens = [_len2_f32(all_nodes[loc[a]], all_nodes[loc[b]]) for a, b in DIAGONALS]
        diag = 0
        for d in (1, 2):
            if lens[d] < lens[diag]:
                diag = d
        kids = list(CORNER_CHILDREN) + list(OCTA_CHILDREN[diag])
        out[ti] = loc[list(kids[0])]
        for c in range(1, 8):
            out[m + 7 * r + (c - 1)] = loc[list(kids[c])]
    return new_nodes, out.astype(np.int32), flagged


def refine_and_relabel(nodes, tets, surfaces, priority, levels: int, node_labels=None,
                       threads: int = 0):
    """Label every node, then `levels` rounds of flag / split / label-new-nodes.

    Returns (nodes, tets, labels, per_level) with per_level a list of dicts
    {flagged, new_nodes, tets}."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float32)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    if node_labels is None:
        node_labels, _ = label_points(nodes, surfaces, priority, threads)
    labels = np.asarray(node_labels, dtype=np.int32).copy()
    per_level = []
    for _ in range(int(levels)):
        new_nodes, tets, flagged = refine_level(nodes, tets, labels)
        if new_nodes.shape[0]:
            new_labels, _ = label_points(new_nodes, surfaces, priority, threads)
        else:
            new_labels = np.zeros(0, dtype=np.int32)
        nodes = np.concatenate([nodes, new_nodes])
        labels = np.concatenate([labels, new_labels])
        per_level.append({"flagged": int(flagged.size), "new_nodes": int(new_nodes.shape[0]),
                          "tets": int(tets.shape[0])})
    return nodes, tets, labels, per_level
