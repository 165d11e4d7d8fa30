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
  * by default the neighbours' 1-3 edge closure (Fig. 2 c-e) is not applied:
    hanging nodes do not affect labeling; the level count is fixed by the
    caller.

With ``conforming=True`` the level is closed into a conforming mesh
(Sec. 2.1.2: elements in V split into eight, their neighbours split along
the one to three edges they share with V, Fig. 2 c-e).  Readings:
  * a tet whose split edges (edges of red tets) are one edge, two edges with a
    common vertex, or the three edges of one face is split into two, three or
    four ("green"); any other non-empty pattern (two opposite edges, three
    edges not bounding a face, four or more) makes it red as well, and the
    closure repeats until no tet changes (the least such red set);
  * green templates replace corners by edge midpoints (orientation kept): one
    edge (i, j): T[j<-m], T[i<-m]; two edges (p, q), (p, r), q < r: the corner
    T[q<-m_pq, r<-m_pr], then for the shorter quad diagonal (float32 squared
    lengths, ties to m_pq-r) either T[q<-m_pq, p<-m_pr], T[p<-m_pq]
    (diagonal m_pq-r) or T[r<-m_pr, p<-m_pq], T[p<-m_pr] (diagonal q-m_pr);
    face (p, q, r), p < q < r: the corners T[q<-m_pq, r<-m_pr],
    T[p<-m_pq, r<-m_qr], T[p<-m_pr, q<-m_qr] and the centre
    T[p<-m_qr, q<-m_pr, r<-m_pq];
  * new nodes are the edge midpoints of the red tets, numbered by first
    appearance over the red tets in index order; a split tet's slot receives
    its first child; red children 1..7 are appended in red order, then the
    green children 1.. in tet index order.
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


def _edge_index(i: int, j: int) -> int:
    return EDGES.index((min(i, j), max(i, j)))


def green_pattern(mask: int):
    """Classify a 6-bit split-edge mask (bit e = EDGES[e]).  Returns None for
    an empty mask, "red" for a pattern the closure must split into eight, or
    ("edge", i, j), ("two", p, q, r) or ("face", p, q, r)."""
    bits = [e for e in range(6) if (mask >> e) & 1]
    if not bits:
        return None
    if len(bits) == 1:
        return ("edge",) + EDGES[bits[0]]
    verts = sorted({v for e in bits for v in EDGES[e]})
    if len(bits) == 2:
        (a, b), (c, d) = EDGES[bits[0]], EDGES[bits[1]]
        common = {a, b} & {c, d}
        if not common:
            return "red"                      # two opposite edges
        p = common.pop()
        q, r = sorted(({a, b} | {c, d}) - {p})
        return ("two", p, q, r)
    if len(bits) == 3 and len(verts) == 3:
        return ("face",) + tuple(verts)      # the three edges of one face
    return "red"


def _sub(loc, pairs):
    """The tet loc[0:4] with corner x replaced by local node m for (x, m)."""
    t = [loc[0], loc[1], loc[2], loc[3]]
    for x, m in pairs:
        t[x] = loc[m]
    return t


def green_children(loc, kind, nodes):
    """Children of a green tet from its local nodes (0-3 corners, 4-9 edge
    midpoints in EDGES order)."""
    if kind[0] == "edge":
        _, i, j = kind
        m = 4 + _edge_index(i, j)
        return [_sub(loc, [(j, m)]), _sub(loc, [(i, m)])]
    if kind[0] == "two":
        _, p, q, r = kind
        mpq, mpr = 4 + _edge_index(p, q), 4 + _edge_index(p, r)
        corner = _sub(loc, [(q, mpq), (r, mpr)])
        d0 = _len2_f32(nodes[loc[mpq]], nodes[loc[r]])
        d1 = _len2_f32(nodes[loc[q]], nodes[loc[mpr]])
        if d1 < d0:   # diagonal q - m_pr
            return [corner, _sub(loc, [(r, mpr), (p, mpq)]), _sub(loc, [(p, mpr)])]
        return [corner, _sub(loc, [(q, mpq), (p, mpr)]), _sub(loc, [(p, mpq)])]
    _, p, q, r = kind
    mpq, mpr, mqr = 4 + _edge_index(p, q), 4 + _edge_index(p, r), 4 + _edge_index(q, r)
    return [_sub(loc, [(q, mpq), (r, mpr)]), _sub(loc, [(p, mpq), (r, mqr)]),
            _sub(loc, [(p, mpr), (q, mqr)]), _sub(loc, [(p, mqr), (q, mpr), (r, mpq)])]


def _edge_keys(t):
    out = []
    for i, j in EDGES:
        a, b = int(t[i]), int(t[j])
        out.append((a, b) if a < b else (b, a))
    return out


def closure(tets: np.ndarray, red0: np.ndarray) -> np.ndarray:
    """Least red set containing red0 whose split edges leave every other tet
    with an empty or green pattern (repeated until no tet changes)."""
    red = red0.copy()
    split = set()
    for ti in np.nonzero(red)[0]:
        split.update(_edge_keys(tets[ti]))
    changed = True
    while changed:
        changed = False
        for ti in np.nonzero(~red)[0]:
            keys = _edge_keys(tets[ti])
            mask = sum(1 << e for e in range(6) if keys[e] in split)
            if green_pattern(mask) == "red":
                red[ti] = True
                split.update(keys)
                changed = True
    return red


def refine_level(nodes: np.ndarray, tets: np.ndarray, node_labels: np.ndarray, conforming: bool = False):
    """One 1->8 split of every flagged tet (and, when conforming, the closure
    of its neighbours).  Returns (new_nodes float32 (K, 3), new_tets int32,
    flagged indices, stats dict)."""
    flagged_mask = flag_tets(tets, node_labels)
    red_mask = closure(tets, flagged_mask) if conforming else flagged_mask
    flagged = np.nonzero(red_mask)[0]
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
    stats = {"flagged": int(flagged_mask.sum()), "promoted": int(flagged.size - flagged_mask.sum()),
             "green": 0}
    if conforming:
        extra = []
        for ti in np.nonzero(~red_mask)[0]:
            keys = _edge_keys(tets[ti])
            mids = [edge_id.get(k) for k in keys]
            mask = sum(1 << e for e in range(6) if mids[e] is not None)
            kind = green_pattern(mask)
            if kind is None:
                continue
            loc = [int(v) for v in tets[ti]] + [(-1 if x is None else x) for x in mids]
            kids = green_children(loc, kind, all_nodes)
            out[ti] = kids[0]
            extra.extend(kids[1:])
            stats["green"] += 1
        if extra:
            out = np.concatenate([out, np.array(extra, dtype=out.dtype)])
    return new_nodes, out.astype(np.int32), flagged, stats


def refine_and_relabel(nodes, tets, surfaces, priority, levels: int, node_labels=None,
                       threads: int = 0, conforming: bool = False):
    """Label every node, then `levels` rounds of flag / split / label-new-nodes.

    Returns (nodes, tets, labels, per_level) with per_level a list of dicts
    {flagged, new_nodes, tets} (plus promoted, green when conforming)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float32)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    if node_labels is None:
        node_labels, _ = label_points(nodes, surfaces, priority, threads)
    labels = np.asarray(node_labels, dtype=np.int32).copy()
    per_level = []
    for _ in range(int(levels)):
        new_nodes, tets, flagged, st = refine_level(nodes, tets, labels, conforming)
        if new_nodes.shape[0]:
            new_labels, _ = label_points(new_nodes, surfaces, priority, threads)
        else:
            new_labels = np.zeros(0, dtype=np.int32)
        nodes = np.concatenate([nodes, new_nodes])
        labels = np.concatenate([labels, new_labels])
        lv = {"flagged": st["flagged"], "new_nodes": int(new_nodes.shape[0]), "tets": int(tets.shape[0])}
        if conforming:
            lv["promoted"] = st["promoted"]
            lv["green"] = st["green"]
        per_level.append(lv)
    return nodes, tets, labels, per_level
