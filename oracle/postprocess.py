"""Oracle of the post-processing steps of Sec. 2.2: Taubin smoothing
(Sec. 2.2.1) and inflation (Sec. 2.2.2), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings where the printed formulas are garbled or silent:
  * smoothing: N_i is node i together with the nodes joined to it by a mesh
    edge (volumetric smoothing), or, for the smoothing of the tissue
    boundaries, by an edge of a boundary face -- a triangle shared by two
    tets of different element labels (a face of only one tet lies on the
    mesh's outer boundary, not between tissues); only the nodes of boundary
    faces move then, and the norms of the stopping rule run over them; the
    printed sums of neighbour positions are
    read as the Laplacian L(x)_i = sum_{j in N_i} (x_j - x_i) / |N_i|; one
    iteration is x' = x + lambda L(x) (forward step) followed by
    x'' = x' - mu L(x') (backward step); nodes marked fixed do not move; the
    iteration stops after the first iteration whose forward step satisfies
    ||x' - x||_2 / ||x^(0)||_2 <= xi, or after max_iters;
  * inflation, for one compartment surface S: an edge whose one node is
    inside S (Omega > 2 pi) and whose other node is outside crosses S; d is
    the distance from the inside node to the intersection of the edge with S
    nearest to it, e the unit vector from the inside node along the edge;
    each inside node moves by zeta d e averaged over its crossing edges; the
    triangles are closed (an edge through a shared triangle edge or vertex
    crosses there), tested with a 1e-12 rounding guard.
"""
from __future__ import annotations

import numpy as np

from . import label_points


def unique_edges(tets) -> np.ndarray:
    """Sorted unique node pairs (a < b) of the tets' six edges."""
    t = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
    pairs = np.concatenate([t[:, [i, j]] for i, j in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))])
    pairs.sort(axis=1)
    return np.unique(pairs, axis=0)


def laplacian(x: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """L(x)_i = sum over j in N_i of (x_j - x_i) / |N_i|, N_i = {i} + edge neighbours."""
    acc = np.zeros_like(x)
    a, b = edges[:, 0], edges[:, 1]
    np.add.at(acc, a, x[b] - x[a])
    np.add.at(acc, b, x[a] - x[b])
    deg = np.bincount(edges.ravel(), minlength=x.shape[0]) + 1
    return acc / deg[:, None]


def taubin_smooth(nodes, tets, lam: float, mu: float, xi: float, max_iters: int, fixed=None):
    """Returns (positions float64 (N, 3), iterations run)."""
    x = np.asarray(nodes, dtype=np.float64).reshape(-1, 3).copy()
    edges = unique_edges(tets)
    fix = np.zeros(x.shape[0], bool) if fixed is None else np.asarray(fixed, bool)
    x0 = np.linalg.norm(x)
    it = 0
    while it < max_iters:
        xh = x + lam * laplacian(x, edges)
        xh[fix] = x[fix]
        step = np.linalg.norm(xh - x) / x0
        x = xh - mu * laplacian(xh, edges)
        x[fix] = xh[fix]
        it += 1
        if step <= xi:
            break
    return x, it


def boundary_faces(tets, elem_labels) -> np.ndarray:
    """Tissue-boundary faces of a labeled tet mesh: sorted node triples of the
    triangles shared by two tets whose element labels differ."""
    t = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
    lab = np.asarray(elem_labels).reshape(-1)
    faces = np.concatenate([t[:, [0, 1, 2]], t[:, [0, 1, 3]], t[:, [0, 2, 3]], t[:, [1, 2, 3]]])
    faces.sort(axis=1)
    flab = np.concatenate([lab, lab, lab, lab])
    uniq, inv, cnt = np.unique(faces, axis=0, return_inverse=True, return_counts=True)
    inv = inv.reshape(-1)
    lo = np.full(uniq.shape[0], np.iinfo(np.int64).max)
    hi = np.full(uniq.shape[0], np.iinfo(np.int64).min)
    np.minimum.at(lo, inv, flab)
    np.maximum.at(hi, inv, flab)
    return uniq[(cnt == 2) & (lo != hi)]


def face_edges(faces) -> np.ndarray:
    """Sorted unique node pairs of the triangles' three edges."""
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    if f.size == 0:
        return np.zeros((0, 2), np.int64)
    pairs = np.concatenate([f[:, [0, 1]], f[:, [0, 2]], f[:, [1, 2]]])
    pairs.sort(axis=1)
    return np.unique(pairs, axis=0)


def taubin_smooth_surface(nodes, tets, elem_labels, lam: float, mu: float, xi: float, max_iters: int):
    """Taubin smoothing of the tissue boundaries (Sec. 2.2.1): the iteration of
    taubin_smooth over the graph of the boundary faces' edges; nodes off the
    boundary do not move.  Returns (positions float64 (N, 3), iterations run,
    number of boundary faces)."""
    x = np.asarray(nodes, dtype=np.float64).reshape(-1, 3).copy()
    faces = boundary_faces(tets, elem_labels)
    edges = face_edges(faces)
    on = np.zeros(x.shape[0], bool)
    on[faces.ravel()] = True
    x0 = np.linalg.norm(x[on])
    it = 0
    while it < max_iters and on.any():
        xh = x + lam * laplacian(x, edges)
        xh[~on] = x[~on]
        step = np.linalg.norm(xh[on] - x[on]) / x0
        x = xh - mu * laplacian(xh, edges)
        x[~on] = xh[~on]
        it += 1
        if step <= xi:
            break
    return x, it, int(faces.shape[0])


def segment_surface_distance(p, q, verts, tris):
    """Distance from p to the intersection of segment [p, q] with the
    triangles that is nearest to p (inf when none), by the plane of each
    triangle and a point-in-triangle test with barycentric coordinates."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    v = np.asarray(verts, np.float64)[np.asarray(tris)]
    a, b, c = v[:, 0], v[:, 1], v[:, 2]
    n = np.cross(b - a, c - a)
    d = q - p
    den = n @ d
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.einsum("ij,ij->i", n, a - p) / den
        x = p + t[:, None] * d
    # barycentric coordinates of x in each triangle
    v0, v1, v2 = b - a, c - a, x - a
    d00 = np.einsum("ij,ij->i", v0, v0)
    d01 = np.einsum("ij,ij->i", v0, v1)
    d11 = np.einsum("ij,ij->i", v1, v1)
    d20 = np.einsum("ij,ij->i", v2, v0)
    d21 = np.einsum("ij,ij->i", v2, v1)
    den2 = d00 * d11 - d01 * d01
    with np.errstate(divide="ignore", invalid="ignore"):
        bv = (d11 * d20 - d01 * d21) / den2
        bw = (d00 * d21 - d01 * d20) / den2
    g = 1e-12   # rounding guard: an edge through a shared triangle edge or vertex still hits
    hit = (den != 0) & (t >= -g) & (t <= 1 + g) & (bv >= -g) & (bw >= -g) & (bv + bw <= 1 + g)
    if not hit.any():
        return np.inf
    return float(t[hit].min() * np.linalg.norm(d))


def inflate(nodes, tets, surface, zeta: float):
    """One inflation of the nodes inside `surface` (an object with .id,
    .verts, .tris) towards it.  Returns (positions float64, moved node count)."""
    x = np.asarray(nodes, dtype=np.float64).reshape(-1, 3).copy()
    edges = unique_edges(tets)
    lab, _ = label_points(np.asarray(nodes, np.float32), [surface], [surface.id])
    inside = lab == surface.id
    disp = np.zeros_like(x)
    cnt = np.zeros(x.shape[0], np.int64)
    for a, b in edges:
        if inside[a] == inside[b]:
            continue
        i, j = (a, b) if inside[a] else (b, a)
        d = segment_surface_distance(x[i], x[j], surface.verts, surface.tris)
        if not np.isfinite(d):
            continue
        e = (x[j] - x[i]) / np.linalg.norm(x[j] - x[i])
        disp[i] += zeta * d * e
        cnt[i] += 1
    moved = cnt > 0
    x[moved] += disp[moved] / cnt[moved, None]
    return x, int(moved.sum())
