"""ctypes binding of libzef (include/zef.h): argument marshalling only.

Every step of the labeling path runs in the library's CUDA kernels.  Arrays
may be numpy arrays (host) or torch tensors (host or CUDA); outputs are
returned on the device of the points.  Importing this module raises
ImportError when libzef.so has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ZEF_LIBRARY selects another build of the library (the debug variant built by
# build.build(debug=True)); default: the release build
LIB_PATH = os.environ.get("ZEF_LIBRARY") or os.path.join(_HERE, "_build", "libzef.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libzef.so is not built ({LIB_PATH}); run paper_2203_10000_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)

ZEF_OK = 0
ZEF_ERR_INVALID_ARG = 1
ZEF_ERR_SURFACE_NOT_CLOSED = 2
ZEF_ERR_SURFACE_ORIENTATION = 3
ZEF_ERR_OOM = 4
ZEF_ERR_CUDA = 5
ZEF_ERR_TIMEOUT = 6
ZEF_ERR_NOT_READY = 7
ZEF_ERR_CAPACITY = 8
ZEF_ERR_BOUNDS = 9
ZEF_AUTO_ORIENT = 1
ZEF_FP32_RESCUE = 0
ZEF_FP64_PLAIN = 1
ZEF_FP32_ONLY = 2
ZEF_NO_TILE_COHERENCE = 1
ZEF_POINT_WALK = 2
ZEF_OMEGA_RAW = 4
MAX_COMPARTMENTS = 64

STATUS_NAMES = {0: "ZEF_OK", 1: "ZEF_ERR_INVALID_ARG", 2: "ZEF_ERR_SURFACE_NOT_CLOSED",
                3: "ZEF_ERR_SURFACE_ORIENTATION", 4: "ZEF_ERR_OOM", 5: "ZEF_ERR_CUDA",
                6: "ZEF_ERR_TIMEOUT", 7: "ZEF_ERR_NOT_READY", 8: "ZEF_ERR_CAPACITY", 9: "ZEF_ERR_BOUNDS"}

# exported symbols of include/zef.h (checked by the CPU tests)
EXPORTED = ["zef_create", "zef_destroy", "zef_last_error", "zef_add_compartment",
            "zef_compartment_info", "zef_compartment_priority", "zef_label_points",
            "zef_refine_and_relabel", "zef_synchronize", "zef_version"]


class LabelOpts(ctypes.Structure):
    _fields_ = [("margin", ctypes.c_float), ("winding_tol", ctypes.c_float),
                ("precision", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("points_per_thread", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class LabelStats(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("nonfinite_points", ctypes.c_int64),
                ("pairs_nominal", ctypes.c_int64), ("pairs_evaluated", ctypes.c_int64),
                ("pairs_rescued", ctypes.c_int64), ("uncertain_pairs", ctypes.c_int64),
                ("work_items", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("block_threads", ctypes.c_int32), ("points_per_thread", ctypes.c_int32),
                ("ms_total", ctypes.c_float), ("ms_label", ctypes.c_float),
                ("ms_rescue", ctypes.c_float), ("reserved", ctypes.c_float),
                ("coherent_pairs", ctypes.c_int64), ("representative_pairs", ctypes.c_int64),
                ("lane_walk_items", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Mesh(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("tets", ctypes.c_void_p),
                ("node_labels", ctypes.c_void_p), ("num_nodes", ctypes.c_int64),
                ("num_tets", ctypes.c_int64), ("node_capacity", ctypes.c_int64),
                ("tet_capacity", ctypes.c_int64), ("labels_valid", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class LevelStats(ctypes.Structure):
    _fields_ = [("flagged_tets", ctypes.c_int64), ("new_nodes", ctypes.c_int64),
                ("nodes", ctypes.c_int64), ("tets", ctypes.c_int64),
                ("pairs_evaluated", ctypes.c_int64), ("uncertain_pairs", ctypes.c_int64),
                ("promoted_tets", ctypes.c_int64), ("green_tets", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_lib.zef_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, _P]
_lib.zef_create.restype = ctypes.c_int
_lib.zef_destroy.argtypes = [_P]
_lib.zef_destroy.restype = None
_lib.zef_last_error.argtypes = [_P]
_lib.zef_last_error.restype = ctypes.c_char_p
_lib.zef_add_compartment.argtypes = [_P, _I32, _P, _I64, _P, _I64, ctypes.c_uint32]
_lib.zef_add_compartment.restype = ctypes.c_int
_lib.zef_compartment_info.argtypes = [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]
_lib.zef_compartment_info.restype = ctypes.c_int
_lib.zef_compartment_priority.argtypes = [_P, _P, _I32]
_lib.zef_compartment_priority.restype = ctypes.c_int
_lib.zef_label_points.argtypes = [_P, _P, _I64, _P, _P, ctypes.POINTER(LabelOpts),
                                  ctypes.POINTER(LabelStats)]
_lib.zef_label_points.restype = ctypes.c_int
_lib.zef_label_points_async.argtypes = [_P, _P, _I64, _P, ctypes.POINTER(LabelOpts)]
_lib.zef_label_points_async.restype = ctypes.c_int
_lib.zef_label_elements.argtypes = [_P, _P, _I64, _P, _I64, _P, _P, ctypes.POINTER(LabelOpts),
                                    ctypes.POINTER(LabelStats)]
_lib.zef_label_elements.restype = ctypes.c_int
class SmoothOpts(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("mu", ctypes.c_float), ("xi", ctypes.c_float),
                ("max_iters", ctypes.c_int32)]


_lib.zef_taubin_smooth.argtypes = [_P, _P, _I64, _P, _I64, _P, ctypes.POINTER(SmoothOpts), ctypes.POINTER(_I32)]
_lib.zef_taubin_smooth.restype = ctypes.c_int
_lib.zef_inflate.argtypes = [_P, _P, _I64, _P, _I64, _I32, ctypes.c_float, ctypes.POINTER(_I64)]
_lib.zef_inflate.restype = ctypes.c_int
_lib.zef_taubin_smooth_surface.argtypes = [_P, _P, _I64, _P, _I64, _P, ctypes.POINTER(SmoothOpts),
                                           ctypes.POINTER(_I32), ctypes.POINTER(_I64)]
_lib.zef_taubin_smooth_surface.restype = ctypes.c_int


class RelabelPass(ctypes.Structure):
    _fields_ = [("evaluated", ctypes.c_int64), ("changed", ctypes.c_int64)]


_lib.zef_relabel_boundary.argtypes = [_P, _P, _I64, _P, _I64, _P, _I32, ctypes.POINTER(LabelOpts),
                                      ctypes.POINTER(RelabelPass), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]
_lib.zef_relabel_boundary.restype = ctypes.c_int
_lib.zef_label_points_noalloc.argtypes = [_P, _P, _I64, _P, _P, ctypes.POINTER(LabelOpts),
                                          ctypes.POINTER(LabelStats)]
_lib.zef_label_points_noalloc.restype = ctypes.c_int
ZEF_REFINE_CONFORMING = 1
NOALLOC_MAX_POINTS = 65536
_lib.zef_refine_and_relabel.argtypes = [_P, ctypes.POINTER(Mesh), _I32, ctypes.POINTER(LabelOpts),
                                        ctypes.POINTER(LevelStats)]
_lib.zef_refine_and_relabel.restype = ctypes.c_int
_lib.zef_synchronize.argtypes = [_P]
_lib.zef_synchronize.restype = ctypes.c_int
_lib.zef_version.argtypes = []
_lib.zef_version.restype = ctypes.c_int32
_lib.zef_debug_strip_stats.argtypes = [_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]
_lib.zef_debug_strip_stats.restype = ctypes.c_int
_lib.zef_debug_strip_entries.argtypes = [_P, _I32, _P, _I64, ctypes.POINTER(_I64)]
_lib.zef_debug_strip_entries.restype = ctypes.c_int
_lib.zef_debug_wait_probe.argtypes = [_P, _I64]
_lib.zef_debug_wait_probe.restype = ctypes.c_int
_lib.zef_debug_cap_tree.argtypes = [_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P, _P, _P]
_lib.zef_debug_cap_tree.restype = ctypes.c_int
_lib.zef_debug_fma_rate.argtypes = [_P, _I32, ctypes.POINTER(ctypes.c_double)]
_lib.zef_debug_fma_rate.restype = ctypes.c_int
_lib.zef_debug_half_angle.argtypes = [_P, _P, _P, _P, _I64]
_lib.zef_debug_half_angle.restype = ctypes.c_int


def lib():
    return _lib


class ZefError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def version() -> int:
    return int(_lib.zef_version())


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _contig(x, dtype_np, dtype_name):
    """(pointer, keepalive, is_cuda) of a C-contiguous array of the dtype."""
    if _is_torch(x):
        import torch
        tdt = {"float32": torch.float32, "int32": torch.int32}[dtype_name]
        t = x.to(tdt).contiguous()
        return t.data_ptr(), t, t.is_cuda
    a = np.ascontiguousarray(x, dtype=dtype_np)
    return a.ctypes.data, a, False


def make_opts(margin=0.0, winding_tol=0.0, precision=ZEF_FP32_RESCUE, block_threads=0,
              points_per_thread=0, kernel=0, coherence=True, point_walk=False,
              omega_raw=False) -> LabelOpts:
    o = LabelOpts()
    o.kernel = kernel
    o.flags = ((0 if coherence else ZEF_NO_TILE_COHERENCE) | (ZEF_POINT_WALK if point_walk else 0)
               | (ZEF_OMEGA_RAW if omega_raw else 0))
    o.margin = margin
    o.winding_tol = winding_tol
    o.precision = precision
    o.block_threads = block_threads
    o.points_per_thread = points_per_thread
    return o


_CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy


class Context:
    """One libzef context on one CUDA device (zef_create / zef_destroy)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = _P()
        if stream is None and device >= 0:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
                    # handle 0 is torch's legacy default stream: pass
                    # cudaStreamLegacy so the library's work stays ordered
                    # with torch's (a NULL stream would make the context
                    # create its own non-blocking stream)
                    if stream == 0:
                        stream = _CUDA_STREAM_LEGACY
            except Exception:  # pragma: no cover
                stream = None
        st = _lib.zef_create(ctypes.byref(self._h), int(device), _P(stream) if stream else None)
        if st != ZEF_OK:
            raise ZefError(st, "zef_create failed")
        self.device = device
        self.ids = []
        self._inflight = []   # buffers of label_points_async calls not yet synchronized

    def close(self):
        if self._h:
            _lib.zef_destroy(self._h)   # waits for every stream of the context
            self._h = _P()
        self._inflight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != ZEF_OK:
            msg = _lib.zef_last_error(self._h)
            raise ZefError(st, msg.decode() if msg else "")

    @property
    def handle(self):
        return self._h

    def add_compartment(self, cid: int, verts, tris, auto_orient: bool = False):
        vp, vk, _ = _contig(verts, np.float32, "float32")
        tp, tk, _ = _contig(tris, np.int32, "int32")
        nv = int(np.prod(vk.shape)) // 3
        nt = int(np.prod(tk.shape)) // 3
        self._check(_lib.zef_add_compartment(self._h, int(cid), vp, nv, tp, nt,
                                             ZEF_AUTO_ORIENT if auto_orient else 0))
        self.ids.append(int(cid))

    def info(self):
        c = _I32()
        t = _I64()
        self._check(_lib.zef_compartment_info(self._h, ctypes.byref(c), ctypes.byref(t)))
        return int(c.value), int(t.value)

    def strip_stats(self, index: int):
        e = _I64()
        s = _I64()
        self._check(_lib.zef_debug_strip_stats(self._h, int(index), ctypes.byref(e), ctypes.byref(s)))
        return int(e.value), int(s.value)

    def strip_entries(self, index: int) -> np.ndarray:
        cnt = _I64()
        self._check(_lib.zef_debug_strip_entries(self._h, int(index), None, 0, ctypes.byref(cnt)))
        out = np.empty((cnt.value, 8), dtype=np.float32)
        self._check(_lib.zef_debug_strip_entries(self._h, int(index), out.ctypes.data, cnt.value,
                                                 ctypes.byref(cnt)))
        return out

    def wait_probe(self, limit_ns: int) -> int:
        """Run the bounded-wait probe; returns the status code (expected
        ZEF_ERR_TIMEOUT) without raising."""
        return int(_lib.zef_debug_wait_probe(self._h, int(limit_ns)))

    def cap_tree(self, index: int):
        """(boxes float32 (n, 6), links int32 (n, 9), entries float32 (m, 8))
        of compartment `index`'s cap tree (diagnostics)."""
        nn, ne = _I64(0), _I64(0)
        self._check(_lib.zef_debug_cap_tree(self._h, int(index), ctypes.byref(nn), ctypes.byref(ne),
                                            None, None, None))
        boxes = np.empty((nn.value, 6), np.float32)
        links = np.empty((nn.value, 9), np.int32)
        ent = np.empty((ne.value, 8), np.float32)
        self._check(_lib.zef_debug_cap_tree(self._h, int(index), ctypes.byref(nn), ctypes.byref(ne),
                                            boxes.ctypes.data, links.ctypes.data, ent.ctypes.data))
        return boxes, links, ent

    def fma_rate(self, fp64: bool = False) -> float:
        """Measured FMA throughput of the device in TFLOP/s (diagnostics)."""
        v = ctypes.c_double(0.0)
        self._check(_lib.zef_debug_fma_rate(self._h, 1 if fp64 else 0, ctypes.byref(v)))
        return float(v.value)

    def half_angle(self, y, x, out):
        """The FP32 label kernel's atan2(y, x) applied elementwise to device
        float32 tensors (diagnostics)."""
        for t in (y, x, out):
            if not _is_torch(t) or not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous():
                raise ValueError("half_angle wants contiguous float32 CUDA tensors")
        n = y.numel()
        if x.numel() != n or out.numel() != n:
            raise ValueError("size mismatch")
        self._check(_lib.zef_debug_half_angle(self._h, y.data_ptr(), x.data_ptr(), out.data_ptr(), n))
        return out

    def set_priority(self, ids):
        a = np.ascontiguousarray(ids, dtype=np.int32)
        self._check(_lib.zef_compartment_priority(self._h, a.ctypes.data, int(a.size)))

    def label_points(self, pts, labels=None, omega=None, opts: LabelOpts | None = None,
                     want_omega: bool = False, stats: bool = True):
        """Labels (and optionally Omega [C][N]) of the points.  Returns
        (labels, omega or None, stats dict or None)."""
        pp, pk, cuda = _contig(pts, np.float32, "float32")
        n = int(np.prod(pk.shape)) // 3
        C, _ = self.info()
        if labels is None:
            if cuda:
                import torch
                labels = torch.empty(n, dtype=torch.int32, device=pk.device)
            else:
                labels = np.empty(n, dtype=np.int32)
        if omega is None and want_omega:
            if cuda:
                import torch
                omega = torch.empty((C, n), dtype=torch.float32, device=pk.device)
            else:
                omega = np.empty((C, n), dtype=np.float32)
        lp = labels.data_ptr() if _is_torch(labels) else labels.ctypes.data
        op = None
        if omega is not None:
            op = omega.data_ptr() if _is_torch(omega) else omega.ctypes.data
        st = LabelStats()
        o = opts if opts is not None else make_opts()
        self._check(_lib.zef_label_points(self._h, pp, n, lp, op, ctypes.byref(o),
                                          ctypes.byref(st) if stats else None))
        return labels, omega, (st.as_dict() if stats else None)

    def label_points_async(self, pts, labels, opts: LabelOpts | None = None):
        """Enqueue the labeling of pts into labels (both host or CUDA; host
        tensors should be pinned) and return at once; the copies overlap the
        neighbouring calls' labeling.  pts and labels are kept referenced and
        must not be touched until synchronize() returns."""
        pp, pk, _ = _contig(pts, np.float32, "float32")
        if pk is not pts:
            raise ValueError("label_points_async wants contiguous float32 points (no temporary copy)")
        n = int(np.prod(pk.shape)) // 3
        if _is_torch(labels):
            if labels.dtype.itemsize != 4 or not labels.is_contiguous() or labels.numel() != n:
                raise ValueError("labels must be a contiguous int32 tensor of n elements")
            lp = labels.data_ptr()
        else:
            if labels.dtype != np.int32 or not labels.flags.c_contiguous or labels.size != n:
                raise ValueError("labels must be a contiguous int32 array of n elements")
            lp = labels.ctypes.data
        o = opts if opts is not None else make_opts()
        self._check(_lib.zef_label_points_async(self._h, pp, n, lp, ctypes.byref(o)))
        self._inflight.append((pts, labels))

    def label_elements(self, nodes, tets, elem_labels=None, node_labels=None,
                       opts: LabelOpts | None = None, want_node_labels: bool = False,
                       stats: bool = True):
        """Element labels by the four-nodes rule with the priority order.
        nodes [N][3] float32, tets [M][4] int32 (numpy or torch, host or
        CUDA).  Returns (elem_labels, node_labels or None, stats or None)."""
        pp, pk, cuda = _contig(nodes, np.float32, "float32")
        tp, tk, tcuda = _contig(tets, np.int32, "int32")
        n = int(np.prod(pk.shape)) // 3
        m = int(np.prod(tk.shape)) // 4
        if elem_labels is None:
            if tcuda:
                import torch
                elem_labels = torch.empty(m, dtype=torch.int32, device=tk.device)
            else:
                elem_labels = np.empty(m, dtype=np.int32)
        if node_labels is None and want_node_labels:
            if cuda:
                import torch
                node_labels = torch.empty(n, dtype=torch.int32, device=pk.device)
            else:
                node_labels = np.empty(n, dtype=np.int32)
        ep = elem_labels.data_ptr() if _is_torch(elem_labels) else elem_labels.ctypes.data
        npp = None
        if node_labels is not None:
            npp = node_labels.data_ptr() if _is_torch(node_labels) else node_labels.ctypes.data
        st = LabelStats()
        o = opts if opts is not None else make_opts()
        self._check(_lib.zef_label_elements(self._h, pp, n, tp, m, ep, npp, ctypes.byref(o),
                                            ctypes.byref(st) if stats else None))
        return elem_labels, node_labels, (st.as_dict() if stats else None)

    @staticmethod
    def _inplace_f32(nodes):
        if _is_torch(nodes):
            if nodes.dtype.itemsize != 4 or not nodes.is_contiguous() or nodes.is_floating_point() is False:
                raise ValueError("nodes must be a contiguous float32 tensor")
            return nodes.data_ptr()
        if nodes.dtype != np.float32 or not nodes.flags.c_contiguous:
            raise ValueError("nodes must be a contiguous float32 array")
        return nodes.ctypes.data

    def taubin_smooth(self, nodes, tets, lam: float = 0.4, mu: float = 0.4, xi: float = 0.0,
                      max_iters: int = 10, fixed=None) -> int:
        """Taubin smoothing of `nodes` in place; returns the iterations run."""
        xp = self._inplace_f32(nodes)
        tp, tk, _ = _contig(tets, np.int32, "int32")
        fp, fk = None, None
        if fixed is not None:
            if _is_torch(fixed):
                fk = fixed.contiguous()
                fp = fk.data_ptr()
            else:
                fk = np.ascontiguousarray(fixed, dtype=np.uint8)
                fp = fk.ctypes.data
        n = int(np.prod(nodes.shape)) // 3
        m = int(np.prod(tk.shape)) // 4
        o = SmoothOpts(lam, mu, xi, int(max_iters))
        it = _I32(0)
        self._check(_lib.zef_taubin_smooth(self._h, xp, n, tp, m, fp, ctypes.byref(o), ctypes.byref(it)))
        return int(it.value)

    def taubin_smooth_surface(self, nodes, tets, elem_labels, lam: float = 0.4, mu: float = 0.4,
                              xi: float = 0.1, max_iters: int = 100):
        """Taubin smoothing of the tissue boundaries (faces between tets of
        different element labels) of `nodes` in place; returns (iterations,
        boundary faces)."""
        xp = self._inplace_f32(nodes)
        tp, tk, _ = _contig(tets, np.int32, "int32")
        lp, lk, _ = _contig(elem_labels, np.int32, "int32")
        n = int(np.prod(nodes.shape)) // 3
        m = int(np.prod(tk.shape)) // 4
        o = SmoothOpts(lam, mu, xi, int(max_iters))
        it = _I32(0)
        nf = _I64(0)
        self._check(_lib.zef_taubin_smooth_surface(self._h, xp, n, tp, m, lp, ctypes.byref(o), ctypes.byref(it),
                                                   ctypes.byref(nf)))
        return int(it.value), int(nf.value)

    def inflate(self, nodes, tets, compartment_id: int, zeta: float = 0.05) -> int:
        """One inflation of `nodes` in place towards the compartment's surface;
        returns the number of nodes moved."""
        xp = self._inplace_f32(nodes)
        tp, tk, _ = _contig(tets, np.int32, "int32")
        n = int(np.prod(nodes.shape)) // 3
        m = int(np.prod(tk.shape)) // 4
        moved = _I64(0)
        self._check(_lib.zef_inflate(self._h, xp, n, tp, m, int(compartment_id), float(zeta), ctypes.byref(moved)))
        return int(moved.value)

    def relabel_boundary(self, nodes, tets, node_labels, max_passes: int = 64,
                         opts: LabelOpts | None = None):
        """Recursive re-labeling at the tissue boundaries; node_labels (int32,
        same residency as nodes and tets) is repaired in place.  Returns
        (per_pass [(evaluated, changed), ...], converged)."""
        pp, pk, _ = _contig(nodes, np.float32, "float32")
        tp, tk, _ = _contig(tets, np.int32, "int32")
        if _is_torch(node_labels):
            if node_labels.dtype.itemsize != 4 or not node_labels.is_contiguous():
                raise ValueError("node_labels must be a contiguous int32 tensor")
            lp = node_labels.data_ptr()
        else:
            if node_labels.dtype != np.int32 or not node_labels.flags.c_contiguous:
                raise ValueError("node_labels must be a contiguous int32 array")
            lp = node_labels.ctypes.data
        n = int(np.prod(pk.shape)) // 3
        m = int(np.prod(tk.shape)) // 4
        per = (RelabelPass * max(1, int(max_passes)))()
        npass, conv = _I32(0), _I32(0)
        o = opts if opts is not None else make_opts()
        self._check(_lib.zef_relabel_boundary(self._h, pp, n, tp, m, lp, int(max_passes), ctypes.byref(o),
                                              per, ctypes.byref(npass), ctypes.byref(conv)))
        return [(int(per[i].evaluated), int(per[i].changed)) for i in range(npass.value)], bool(conv.value)

    def refine_and_relabel(self, nodes, tets, node_labels, num_nodes: int, num_tets: int,
                           levels: int, labels_valid: bool = False, opts: LabelOpts | None = None,
                           conforming: bool = False):
        """In-place refinement of preallocated arrays (capacities = their
        lengths).  Returns (num_nodes, num_tets, per-level stats)."""
        m = Mesh()
        m.nodes = nodes.data_ptr() if _is_torch(nodes) else nodes.ctypes.data
        m.tets = tets.data_ptr() if _is_torch(tets) else tets.ctypes.data
        m.node_labels = node_labels.data_ptr() if _is_torch(node_labels) else node_labels.ctypes.data
        m.num_nodes = int(num_nodes)
        m.num_tets = int(num_tets)
        m.node_capacity = int(nodes.shape[0])
        m.tet_capacity = int(tets.shape[0])
        m.labels_valid = 1 if labels_valid else 0
        m.flags = ZEF_REFINE_CONFORMING if conforming else 0
        per = (LevelStats * max(1, levels))()
        o = opts if opts is not None else make_opts()
        self._check(_lib.zef_refine_and_relabel(self._h, ctypes.byref(m), int(levels), ctypes.byref(o), per))
        return int(m.num_nodes), int(m.num_tets), [per[i].as_dict() for i in range(levels)]

    def synchronize(self):
        try:
            self._check(_lib.zef_synchronize(self._h))
        finally:
            self._inflight.clear()
