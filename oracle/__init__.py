"""Plain FP64 CPU oracle for solid-angle labeling (Sec. 2.1.3, Eq. 1; Sec. 2.1).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package.  It shares no code with the CUDA path
(``paper_2203_10000_gb300``) and never calls it.

* ``solid_angle``   -- Omega(p) for one closed surface, the sum of the Van
  Oosterom-Strackee triangle solid angles in double (oracle.c).
* ``label_points``  -- the paper's labeling decision: a point is enclosed by a
  compartment surface when s = Omega / 4 pi reaches the threshold T; T = 1/2
  with a strict comparison, i.e. inside iff Omega > 2 pi.  Nested and
  intersecting compartments are resolved by the layer hierarchy: the first
  compartment of the priority list that encloses the point wins (Sec. 2.1);
  a point enclosed by none gets 0, the temporary bounding box.
* ``label_elements`` -- element labels by the four-nodes rule (Sec. 2.1.3: a
  tetrahedron whose four nodes are inside a compartment surface belongs to
  that compartment) under the same priority list.
* ``refine.refine_and_relabel`` -- the refinement/re-labeling recursion
  (Sec. 2.1.2, 2.1.3 item 2).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

TWO_PI = 2.0 * math.pi


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no fast-math, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_omega.argtypes = [P, I64, P, I64, P, I64, P, ctypes.c_int]
            lib.oracle_omega.restype = ctypes.c_int
            lib.oracle_triangle_terms.argtypes = [P, P, I64, P, I64, P]
            lib.oracle_triangle_terms.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1, 3))


def solid_angle(points, verts, tris, threads: int = 0) -> np.ndarray:
    """Omega(p) in double for every point against one triangulated surface.

    float32 inputs are promoted to double exactly.  Triangles are summed in
    index order."""
    lib = _load()
    p, v, t = _f64(points), _f64(verts), _i32(tris)
    out = np.empty(p.shape[0], dtype=np.float64)
    rc = lib.oracle_omega(p.ctypes.data, p.shape[0], v.ctypes.data, v.shape[0], t.ctypes.data,
                          t.shape[0], out.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("triangle index out of range")
    return out


def triangle_terms(point, verts, tris) -> np.ndarray:
    """Per-triangle solid angles Omega_t of one point (for closed-form pins)."""
    lib = _load()
    p = _f64(point)
    v, t = _f64(verts), _i32(tris)
    out = np.empty(t.shape[0], dtype=np.float64)
    rc = lib.oracle_triangle_terms(p.ctypes.data, v.ctypes.data, v.shape[0], t.ctypes.data,
                                   t.shape[0], out.ctypes.data)
    if rc != 0:
        raise ValueError("triangle index out of range")
    return out


def inside(omega) -> np.ndarray:
    """Threshold decision s >= T read as Omega > 2 pi (T = 1/2, strict)."""
    return np.asarray(omega) > TWO_PI


def label_points(points, surfaces, priority, threads: int = 0):
    """Labels and the Omega matrix of all points.

    surfaces: sequence of objects with .id, .verts, .tris (or (id, verts, tris)
    tuples).  priority: compartment ids, first = highest priority.
    Returns (labels int32 (N,), omega float64 (C, N) with rows in priority
    order).  A point with a non-finite coordinate gets label -1 and NaN Omega.
    """
    by_id = {}
    for s in surfaces:
        if isinstance(s, tuple):
            sid, v, t = s
        else:
            sid, v, t = s.id, s.verts, s.tris
        by_id[int(sid)] = (v, t)
    prio = [int(i) for i in priority]
    if sorted(prio) != sorted(by_id):
        raise ValueError("priority must be a permutation of the compartment ids")
    p = _f64(points)
    finite = np.all(np.isfinite(p), axis=1)
    pf = p[finite]
    omega = np.full((len(prio), p.shape[0]), np.nan)
    for row, cid in enumerate(prio):
        v, t = by_id[cid]
        omega[row, finite] = solid_angle(pf, v, t, threads)
    labels = np.zeros(p.shape[0], dtype=np.int32)
    decided = np.zeros(p.shape[0], dtype=bool)
    for row, cid in enumerate(prio):
        hit = finite & ~decided & inside(omega[row])
        labels[hit] = cid
        decided |= hit
    labels[~finite] = -1
    return labels, omega


def label_elements(nodes, tets, surfaces, priority, threads: int = 0):
    """Element labels by the four-nodes rule (Sec. 2.1.3) with the priority
    list of Sec. 2.1: a tet gets the first compartment in priority order whose
    surface encloses all four of its nodes (Omega > 2 pi at each node), 0 when
    none does, and -1 when a node has a non-finite coordinate.

    Returns (element labels int32 (M,), node labels int32 (N,))."""
    node_labels, omega = label_points(nodes, surfaces, priority, threads)
    t = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
    if t.size and (t.min() < 0 or t.max() >= node_labels.shape[0]):
        raise ValueError("tet node index out of range")
    ins = inside(omega)                      # (C, N); NaN rows compare False
    prio = [int(i) for i in priority]
    labels = np.zeros(t.shape[0], dtype=np.int32)
    decided = np.zeros(t.shape[0], dtype=bool)
    for row, cid in enumerate(prio):
        all_four = ins[row][t].all(axis=1)   # every node of the tet inside
        hit = ~decided & all_four
        labels[hit] = cid
        decided |= hit
    labels[(node_labels[t] < 0).any(axis=1)] = -1
    return labels, node_labels
