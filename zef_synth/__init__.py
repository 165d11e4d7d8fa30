"""Seeded synthetic inputs for the solid-angle labeling path.

This module only builds geometry: closed triangulated compartment surfaces
(geodesic spheres, perturbed ellipsoids, tori) and query points (regular
hexahedral lattices split into five tetrahedra, their nodes and tet
centroids).  It holds none of the labeling arithmetic; both the CUDA path and
the CPU oracle receive the same arrays from here.

Every coordinate is rounded to float32 before it is returned, so the float32
values handed to the GPU are exactly the values the float64 oracle promotes
(the precision reading for inputs: the paper does not state one).

Workload shapes follow the paper: closed segmentation surfaces per compartment
(Sec. 2.1.3) nested from the innermost to the outermost with a priority order
(Sec. 2.1), and a regular hexahedral lattice subdivided into five tetrahedra
with alternating diagonals (Sec. 2.1.1, Fig. 1).  The paper's own head data
(a FreeSurfer segmentation) is not available; the perturbed ellipsoids and tori
below stand in for it at the paper's sizes (Table 1: up to 372,088 surface
triangles and 4.8-7.5 million mesh nodes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Surface", "Workload", "geodesic_sphere", "perturbed_ellipsoid", "torus",
    "lattice_5tet", "tet_centroids", "config0", "config1", "config2", "config3",
    "config4", "ary_spheres", "make_config", "freq_for_triangles",
]


@dataclass
class Surface:
    """A closed, outward-oriented triangulated compartment boundary."""
    id: int
    name: str
    verts: np.ndarray  # (V, 3) float32
    tris: np.ndarray   # (T, 3) int32, 0-based, counter-clockwise seen from outside

    @property
    def ntris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class Workload:
    name: str
    surfaces: list
    priority: list               # compartment ids, first = highest priority
    points: np.ndarray | None    # (N, 3) float32 query points
    nodes: np.ndarray | None = None   # lattice nodes (refinement workload)
    tets: np.ndarray | None = None    # (M, 4) int32
    levels: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def total_tris(self) -> int:
        return sum(s.ntris for s in self.surfaces)


# --------------------------------------------------------------------------
# geodesic spheres (class-I subdivision of the icosahedron)
# --------------------------------------------------------------------------
def _icosahedron():
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
        [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
        [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def geodesic_sphere(freq: int):
    """Unit geodesic sphere: each icosahedron face split into freq^2 triangles.

    Returns (verts float64 (10 f^2 + 2, 3) on the unit sphere, tris int32
    (20 f^2, 3)) with outward orientation.  Shared edge and corner points are
    merged through exact integer barycentric keys, so the mesh is closed.
    """
    if freq < 1:
        raise ValueError("freq >= 1")
    V0, F0 = _icosahedron()
    n = int(freq)
    # grid coordinates (i along B-A, j along C-A), i + j <= n
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    m = (ii + jj) <= n
    gi, gj = ii[m], jj[m]
    ga = n - gi - gj
    grid_index = -np.ones((n + 1, n + 1), dtype=np.int64)
    grid_index[gi, gj] = np.arange(gi.size)
    # local triangles
    up = []
    dn = []
    for i in range(n):
        for j in range(n - i):
            up.append((grid_index[i, j], grid_index[i + 1, j], grid_index[i, j + 1]))
            if i + j + 1 < n:
                dn.append((grid_index[i + 1, j], grid_index[i + 1, j + 1], grid_index[i, j + 1]))
    local_tris = np.array(up + dn, dtype=np.int64)

    keys_all = []
    pos_all = []
    for fidx, (a, b, c) in enumerate(F0):
        wa, wb, wc = ga, gi, gj
        # canonical key of the barycentric point (a, b, c weighted), 12 vertices
        key = np.zeros(gi.size, dtype=np.int64)
        # corners
        corner = (wa == n) | (wb == n) | (wc == n)
        cid = np.where(wa == n, a, np.where(wb == n, b, c))
        key[corner] = cid[corner]
        # edge points (exactly one weight zero, not a corner)
        nz = (wa > 0).astype(int) + (wb > 0).astype(int) + (wc > 0).astype(int)
        edge = (nz == 2) & ~corner
        # pair of vertex ids and weight on the larger id
        v1 = np.where(wa == 0, b, a)
        w1 = np.where(wa == 0, wb, wa)
        v2 = np.where(wc == 0, b, c)
        w2 = np.where(wc == 0, wb, wc)
        lo = np.minimum(v1, v2)
        hi = np.maximum(v1, v2)
        whi = np.where(v1 > v2, w1, w2)
        ekey = 16 + (lo * 12 + hi) * (n + 1) + whi
        key[edge] = ekey[edge]
        inner = nz == 3
        base = 16 + 144 * (n + 1)
        ikey = base + (fidx * (n + 1) + gi) * (n + 1) + gj
        key[inner] = ikey[inner]
        pos = (np.outer(wa, V0[a]) + np.outer(wb, V0[b]) + np.outer(wc, V0[c])) / n
        keys_all.append(key)
        pos_all.append(pos)
    keys = np.concatenate(keys_all)
    pos = np.concatenate(pos_all)
    uk, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    verts = pos[first]
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    tris = []
    off = 0
    for fidx in range(20):
        tris.append(inv[off + local_tris])
        off += gi.size
    tris = np.concatenate(tris).astype(np.int32)
    return verts, tris


def freq_for_triangles(t: float) -> int:
    """Geodesic frequency whose 20 f^2 triangle count is closest to t."""
    return max(1, int(round(math.sqrt(t / 20.0))))


# --------------------------------------------------------------------------
# real spherical harmonics (for seeded smooth radial perturbations)
# --------------------------------------------------------------------------
def _real_sh(lmax: int, u: np.ndarray) -> list:
    """Real spherical harmonics Y_lm(u) for 1 <= l <= lmax, |m| <= l."""
    x = np.clip(u[:, 2], -1.0, 1.0)
    phi = np.arctan2(u[:, 1], u[:, 0])
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    out = []
    # P[l][m] via the standard three-term recurrence in l for fixed m
    P = {}
    for m in range(lmax + 1):
        pmm = np.ones_like(x)
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * sx
            fact += 2.0
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = x * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            k = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                y = k * P[(l, 0)]
            elif m > 0:
                y = math.sqrt(2.0) * k * np.cos(m * phi) * P[(l, m)]
            else:
                y = math.sqrt(2.0) * k * np.sin(am * phi) * P[(l, am)]
            out.append((l, m, y))
    return out


def _sh_field(u: np.ndarray, rng: np.random.Generator, lmax: int) -> np.ndarray:
    s = np.zeros(u.shape[0])
    for l, m, y in _real_sh(lmax, u):
        s += rng.standard_normal() / (l + 1) * y
    return s


def _as_f32_surface(verts64: np.ndarray, tris: np.ndarray):
    v = np.ascontiguousarray(verts64, dtype=np.float64).astype(np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    # orientation from the float32 vertices, signed volume in float64
    vv = v.astype(np.float64)
    a, b, c = vv[t[:, 0]], vv[t[:, 1]], vv[t[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    if vol < 0:
        t = t[:, [0, 2, 1]].copy()
    return v, t


def perturbed_ellipsoid(freq: int, axes, amp: float = 3.0, seed: int = 0,
                        center=(0.0, 0.0, 0.0), lmax: int = 8):
    """Geodesic sphere scaled to semi-axes `axes` plus a radial perturbation
    amp * S(u) / max|S|, S a seeded random real spherical-harmonic field of
    degree 1..lmax with N(0, 1)/(l + 1) coefficients (l = 0 excluded)."""
    u, tris = geodesic_sphere(freq)
    rng = np.random.default_rng(seed)
    x = u * np.asarray(axes, dtype=np.float64)[None, :]
    if amp != 0.0:
        s = _sh_field(u, rng, lmax)
        s = s / np.max(np.abs(s))
        x = x + (amp * s)[:, None] * u
    x = x + np.asarray(center, dtype=np.float64)[None, :]
    return _as_f32_surface(x, tris)


def box_surface(lo, hi, m: int = 1):
    """Closed, outward-oriented triangulation of the axis-aligned box
    [lo, hi]: every face split into an m x m grid of quads, two triangles
    each (12 m^2 triangles).  A point strictly inside the box has winding
    number 1, a point strictly outside 0."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ids = {}
    verts = []

    def vid(g):
        if g not in ids:
            ids[g] = len(verts)
            verts.append(lo + (hi - lo) * np.asarray(g, dtype=np.float64) / m)
        return ids[g]

    tris = []
    for axis in range(3):
        u, w = [a for a in range(3) if a != axis]
        for side in (0, m):
            outward = np.zeros(3)
            outward[axis] = 1.0 if side == m else -1.0
            for i in range(m):
                for j in range(m):
                    quad = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        g = [0, 0, 0]
                        g[axis], g[u], g[w] = side, i + di, j + dj
                        quad.append(vid(tuple(g)))
                    for t in ((quad[0], quad[1], quad[2]), (quad[0], quad[2], quad[3])):
                        p = [verts[k] for k in t]
                        nrm = np.cross(p[1] - p[0], p[2] - p[0])
                        tris.append(t if nrm @ outward > 0 else (t[0], t[2], t[1]))
    return np.asarray(verts, dtype=np.float32), np.asarray(tris, dtype=np.int32)


def torus(R: float, r: float, m: int, k: int, seed: int = 0, amp: float = 0.0,
          center=(0.0, 0.0, 0.0), axis: int = 2):
    """Genus-1 torus of major radius R, minor radius r, an m x k quad grid
    split into 2 m k triangles, outward oriented, optional seeded radial
    perturbation of the tube (|delta| <= amp)."""
    uu = 2 * np.pi * np.arange(m) / m
    vv = 2 * np.pi * np.arange(k) / k
    U, Vg = np.meshgrid(uu, vv, indexing="ij")
    rr = np.full(U.shape, float(r))
    if amp != 0.0:
        rng = np.random.default_rng(seed)
        f = np.zeros(U.shape)
        for a in range(1, 4):
            for b in range(1, 4):
                c1, c2 = rng.standard_normal(2)
                f += (c1 * np.cos(a * U + b * Vg) + c2 * np.sin(a * U - b * Vg)) / (a + b)
        rr = rr + amp * f / np.max(np.abs(f))
    X = (R + rr * np.cos(Vg)) * np.cos(U)
    Y = (R + rr * np.cos(Vg)) * np.sin(U)
    Z = rr * np.sin(Vg)
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    if axis == 0:
        P = P[:, [2, 0, 1]]
    elif axis == 1:
        P = P[:, [0, 2, 1]]
    P = P + np.asarray(center, dtype=np.float64)[None, :]
    idx = np.arange(m * k).reshape(m, k)
    i0 = idx
    i1 = np.roll(idx, -1, axis=0)
    i2 = np.roll(idx, -1, axis=1)
    i3 = np.roll(np.roll(idx, -1, axis=0), -1, axis=1)
    t1 = np.stack([i0.ravel(), i1.ravel(), i3.ravel()], 1)
    t2 = np.stack([i0.ravel(), i3.ravel(), i2.ravel()], 1)
    tris = np.concatenate([t1, t2])
    return _as_f32_surface(P, tris)


# --------------------------------------------------------------------------
# regular lattice split into five tetrahedra (Sec. 2.1.1, Fig. 1)
# --------------------------------------------------------------------------
# corner c of a hexahedron has offset bits (x, y, z) = (c & 1, c >> 1 & 1, c >> 2 & 1)
_EVEN = np.array([[0, 3, 5, 6], [1, 0, 3, 5], [2, 0, 3, 6], [4, 0, 5, 6], [7, 3, 5, 6]])
_ODD = np.array([[1, 2, 4, 7], [0, 1, 2, 4], [3, 1, 2, 7], [5, 1, 4, 7], [6, 2, 4, 7]])
_OFF = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])


def _orient_local(tab):
    out = tab.copy()
    for r in range(out.shape[0]):
        a, b, c, d = (_OFF[out[r, q]].astype(float) for q in range(4))
        if np.dot(b - a, np.cross(c - a, d - a)) < 0:
            out[r, [2, 3]] = out[r, [3, 2]]
    return out


_EVEN_O = _orient_local(_EVEN)
_ODD_O = _orient_local(_ODD)


def lattice_5tet(n, h: float, origin):
    """Nodes (float32, x fastest) and positively oriented tets (int32) of an
    n[0] x n[1] x n[2] hexahedral lattice with spacing h, each hexahedron
    split into five tetrahedra; the split alternates with (i + j + k) parity
    so that face diagonals of neighbouring cells coincide."""
    nx, ny, nz = (int(v) for v in (n if np.ndim(n) else (n, n, n)))
    ox, oy, oz = (float(v) for v in origin)
    ix = np.arange(nx + 1)
    iy = np.arange(ny + 1)
    iz = np.arange(nz + 1)
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    nodes = np.stack([ox + h * X.ravel(), oy + h * Y.ravel(), oz + h * Z.ravel()], 1)
    nodes = nodes.astype(np.float32)

    def nid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    corners = np.stack([nid(cx + _OFF[c, 0], cy + _OFF[c, 1], cz + _OFF[c, 2]) for c in range(8)], 1)
    parity = (cx + cy + cz) & 1
    tets = np.empty((cx.size, 5, 4), dtype=np.int64)
    even = parity == 0
    tets[even] = corners[even][:, _EVEN_O]
    tets[~even] = corners[~even][:, _ODD_O]
    return nodes, tets.reshape(-1, 4).astype(np.int32)


def tet_centroids(nodes: np.ndarray, tets: np.ndarray, chunk: int = 1 << 22) -> np.ndarray:
    out = np.empty((tets.shape[0], 3), dtype=np.float32)
    nd = nodes.astype(np.float64)
    for s in range(0, tets.shape[0], chunk):
        t = tets[s:s + chunk]
        c = (nd[t[:, 0]] + nd[t[:, 1]] + nd[t[:, 2]] + nd[t[:, 3]]) * 0.25
        out[s:s + chunk] = c.astype(np.float32)
    return out


def lattice_centroids(ncell: int, h: float, origin) -> np.ndarray:
    """Centroids of the five-tet split of an ncell^3 lattice, computed cell by
    cell without materialising the node array (for the largest workloads)."""
    offs_even = np.array([_OFF[r].mean(0) for r in _EVEN_O])  # (5, 3)
    offs_odd = np.array([_OFF[r].mean(0) for r in _ODD_O])
    n = int(ncell)
    out = np.empty((n ** 3 * 5, 3), dtype=np.float32)
    ix = np.arange(n)
    org = np.asarray(origin, dtype=np.float64)
    for k in range(n):
        cy, cx = np.meshgrid(ix, ix, indexing="ij")
        cx, cy = cx.ravel(), cy.ravel()
        par = (cx + cy + k) & 1
        base = np.stack([cx, cy, np.full_like(cx, k)], 1).astype(np.float64)
        off = np.where(par[:, None, None] == 0, offs_even[None], offs_odd[None])
        c = org + h * (base[:, None, :] + off)
        s = k * n * n * 5
        out[s:s + n * n * 5] = c.reshape(-1, 3).astype(np.float32)
    return out


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def config0() -> Workload:
    """Unit geodesic sphere of frequency 8 (642 vertices, 1280 triangles);
    a 32^3 grid over [-1.5, 1.5]^3 plus 4096 uniform points (seed 0)."""
    v, t = geodesic_sphere(8)
    v32, t32 = _as_f32_surface(v, t)
    g = np.linspace(-1.5, 1.5, 32)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    rnd = np.random.default_rng(0).uniform(-1.5, 1.5, size=(4096, 3))
    pts = np.concatenate([grid, rnd]).astype(np.float32)
    return Workload("icosphere-f8 / 36,864 points", [Surface(1, "sphere", v32, t32)], [1], pts)


def _three_layer(seed0: int = 1):
    # semi-axes by size (scalp > skull > brain), freq 32 / 32 / 64
    spec = [("brain", 3, (75.0, 70.0, 64.0), 64, seed0 + 2),
            ("skull", 2, (92.0, 86.0, 80.0), 32, seed0 + 1),
            ("scalp", 1, (100.0, 94.0, 88.0), 32, seed0 + 0)]
    surfs = []
    for name, cid, axes, f, sd in spec:
        v, t = perturbed_ellipsoid(f, axes, amp=3.0, seed=sd)
        surfs.append(Surface(cid, name, v, t))
    return surfs


def config1(npts_limit: int | None = None) -> Workload:
    """Three nested perturbed ellipsoids (brain 81,920, skull 20,480, scalp
    20,480 triangles); query points are the 5,000,000 tet centroids of a 2 mm
    lattice over [-100, 100]^3 mm."""
    surfs = _three_layer()
    pts = lattice_centroids(100, 2.0, (-100.0, -100.0, -100.0))
    if npts_limit is not None:
        pts = pts[:npts_limit]
    return Workload("3-layer head / 2 mm centroids (5.0M points, 122,880 tris)", surfs,
                    [3, 2, 1], pts)


def _deep_structures(rng, count, tmin, tmax, box, first_id, amp=1.0, torus_every=4,
                     intersect_pairs=True):
    """Uneven deep compartments: perturbed ellipsoids and tori with triangle
    counts log-uniform in [tmin, tmax]; some nested, some overlapping."""
    surfs = []
    centers = []
    for q in range(count):
        T = float(np.exp(rng.uniform(np.log(tmin), np.log(tmax))))
        cid = first_id + q
        if torus_every and q % torus_every == torus_every - 1:
            R = rng.uniform(8.0, 14.0)
            r = rng.uniform(2.5, 4.0)
            k = max(6, int(round(math.sqrt(T / 2.0 * r / R))))
            m = max(8, int(round(T / 2.0 / k)))
            c = rng.uniform(-box, box, size=3)
            v, t = torus(R, r, m, k, seed=int(rng.integers(1 << 30)), amp=min(amp, 0.5 * r),
                         center=c, axis=int(rng.integers(3)))
            surfs.append(Surface(cid, f"torus{q}", v, t))
            centers.append((c, R + r))
            continue
        f = freq_for_triangles(T)
        if q % 5 == 1 and centers:
            # nested: a scaled copy inside an earlier ellipsoid
            pc, prad = centers[int(rng.integers(len(centers)))]
            axes = np.full(3, 0.45 * prad) * rng.uniform(0.8, 1.0, size=3)
            c = pc + rng.uniform(-0.1, 0.1, size=3) * prad
        elif q % 5 == 2 and centers and intersect_pairs:
            # intersecting: centre offset so that the overlap depth is U(0, 2) mm
            pc, prad = centers[-1]
            axes = rng.uniform(6.0, 14.0, size=3)
            d = prad + axes.min() - rng.uniform(0.0, 2.0)
            dirv = rng.standard_normal(3)
            dirv /= np.linalg.norm(dirv)
            c = pc + d * dirv
        else:
            axes = rng.uniform(6.0, 18.0, size=3)
            c = rng.uniform(-box, box, size=3)
        v, t = perturbed_ellipsoid(f, axes, amp=min(amp, 0.2 * float(np.min(axes))),
                                   seed=int(rng.integers(1 << 30)), center=c)
        surfs.append(Surface(cid, f"deep{q}", v, t))
        centers.append((c, float(np.min(axes))))
    return surfs


def config2(npts_limit: int | None = None) -> Workload:
    """Twenty deep compartments (2k-150k triangles, log-uniform, seed 2),
    ellipsoids and tori, some nested and some intersecting; 1 mm lattice
    centroids over [-80, 80]^3 (20,480,000 points)."""
    rng = np.random.default_rng(2)
    surfs = _deep_structures(rng, 20, 2000, 150000, 45.0, 1, amp=1.0)
    prio = [s.id for s in surfs]
    pts = None if npts_limit == 0 else lattice_centroids(160, 1.0, (-80.0, -80.0, -80.0))
    if npts_limit is not None and pts is not None:
        pts = pts[:npts_limit]
    return Workload("20 deep compartments / 1 mm centroids (20.5M points)", surfs, prio, pts)


def config3() -> Workload:
    """Three-layer head plus 8 deep compartments (2k-30k triangles); a 4 mm
    lattice over [-100, 100]^3 (51^3 nodes) refined 3 levels."""
    surfs = _three_layer()
    rng = np.random.default_rng(3)
    deep = _deep_structures(rng, 8, 2000, 30000, 35.0, 4, amp=1.0)
    nodes, tets = lattice_5tet(50, 4.0, (-100.0, -100.0, -100.0))
    prio = [s.id for s in deep] + [3, 2, 1]
    return Workload("head + 8 deep / 4 mm lattice, 3 refine levels", surfs + deep, prio,
                    None, nodes=nodes, tets=tets, levels=3)


def config4(npts_limit: int | None = None, with_points: bool = True) -> Workload:
    """Full-scale synthetic head: 5 large nested surfaces (scalp, skull, CSF,
    grey, white; frequencies 122/118/114/110/106) plus 19 subcortical surfaces
    of 2k-30k triangles; 1 mm lattice centroids over [-112, 112]^3
    (56,197,120 points)."""
    big = [("white", 5, (76.0, 68.0, 62.0), 106, 15),
           ("grey", 4, (86.0, 78.0, 72.0), 110, 14),
           ("csf", 3, (94.0, 86.0, 80.0), 114, 13),
           ("skull", 2, (102.0, 94.0, 88.0), 118, 12),
           ("scalp", 1, (110.0, 102.0, 96.0), 122, 11)]
    rng = np.random.default_rng(4)
    deep = _deep_structures(rng, 19, 2000, 30000, 35.0, 6, amp=1.0)
    surfs = []
    for name, cid, axes, f, sd in big:
        v, t = perturbed_ellipsoid(f, axes, amp=3.0, seed=sd)
        surfs.append(Surface(cid, name, v, t))
    prio = [s.id for s in deep] + [5, 4, 3, 2, 1]
    pts = None
    if with_points:
        pts = lattice_centroids(224, 1.0, (-112.0, -112.0, -112.0))
        if npts_limit is not None:
            pts = pts[:npts_limit]
    return Workload("full head 24 compartments / 1 mm centroids (56.2M points)",
                    deep + surfs, prio, pts)


def ary_spheres() -> Workload:
    """Three concentric geodesic spheres of radii 87 / 92 / 100 mm (the Ary
    model geometry, Sec. 2.4) with frequencies 38 / 38 / 39; 1 mm lattice
    nodes over [-101, 101]^3."""
    surfs = []
    for cid, (name, rad, f) in enumerate([("brain", 87.0, 38), ("skull", 92.0, 38),
                                          ("scalp", 100.0, 39)]):
        u, t = geodesic_sphere(f)
        v, t = _as_f32_surface(u * rad, t)
        surfs.append(Surface(3 - cid, name, v, t))
    g = np.arange(-101.0, 102.0, 1.0)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)
    return Workload("Ary 3-sphere / 1 mm nodes", surfs, [3, 2, 1], pts)


def make_config(k: int, **kw) -> Workload:
    return [config0, config1, config2, config3, config4][k](**kw)


def sample_rows(a: np.ndarray, k: int, seed: int = 0) -> np.ndarray:
    """Sorted seeded sample of k row indices of a (without replacement)."""
    rng = np.random.default_rng(seed)
    k = min(k, a.shape[0])
    return np.sort(rng.choice(a.shape[0], size=k, replace=False))
