/*
 * zef.h -- C ABI of the GB300 solid-angle labeling library (libzef).
 *
 * The library decides which closed compartment surface encloses each query
 * point of a tetrahedral mesh, following Galaz Prieto et al., "Multi-compartment
 * human head modeling: generating adaptive tetrahedral mesh with GPU
 * acceleration" (arXiv:2203.10000):
 *
 *   Sec. 2.1.3, Eq. 1   s(p) = Omega(p) / 4 pi, Omega the solid angle that the
 *                       closed surface subtends at p; p is enclosed when
 *                       s >= T.  Here T = 1/2 with a strict comparison:
 *                       inside  <=>  Omega > 2 pi.  Omega is evaluated per
 *                       triangle in closed form (Van Oosterom & Strackee,
 *                       IEEE TBME 30(2), 1983) and summed over the surface.
 *   Sec. 2.1            nested compartments take precedence from the innermost
 *                       to the outermost; where boundaries intersect, the one
 *                       first in the layer hierarchy wins; a temporary
 *                       bounding box is the outermost compartment (label 0).
 *   Sec. 2.1.2, 2.1.3   refinement of the tets on a tissue boundary and
 *                       recursive re-labeling of the new nodes only.
 *
 * Conventions shared by every call
 *   - Every call returns a zef_status.  On failure the outputs are
 *     unspecified, the context stays usable and zef_last_error() describes the
 *     failure.
 *   - Array arguments may live in host memory or in device memory of the
 *     context's device; the library detects which (cudaPointerGetAttributes).
 *     The caller keeps ownership of every buffer it passes.  All arrays are
 *     dense, row-major, C-contiguous.
 *   - When every array argument of a call is device memory the call is
 *     asynchronous on the context's stream, except that a non-NULL stats
 *     argument makes it synchronize.  With any host array the call
 *     synchronizes before it returns.
 *   - Coordinates are float32 in any consistent unit (the workloads use mm).
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef ZEF_H
#define ZEF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZEF_VERSION_MAJOR 1
#define ZEF_VERSION_MINOR 0

/* Maximum number of compartments in one context (bit masks are 64 bits). */
#define ZEF_MAX_COMPARTMENTS 64

typedef struct zef_ctx zef_ctx; /* opaque; owns all device memory it allocates */

typedef enum zef_status {
    ZEF_OK = 0,
    ZEF_ERR_INVALID_ARG = 1,          /* null/negative/inconsistent argument */
    ZEF_ERR_SURFACE_NOT_CLOSED = 2,   /* an undirected edge not used by exactly two
                                         triangles in opposite directions */
    ZEF_ERR_SURFACE_ORIENTATION = 3,  /* signed volume <= 0 and no ZEF_AUTO_ORIENT */
    ZEF_ERR_OOM = 4,                  /* device or host allocation failed */
    ZEF_ERR_CUDA = 5,                 /* a CUDA runtime call failed */
    ZEF_ERR_TIMEOUT = 6,              /* a bounded device wait expired (the kernel
                                         stopped early and reported it) */
    ZEF_ERR_NOT_READY = 7,            /* no compartment registered */
    ZEF_ERR_CAPACITY = 8,             /* refinement needs more nodes/tets than the
                                         caller's capacities */
    ZEF_ERR_BOUNDS = 9                /* only the debug build (ZEF_DEBUG_BOUNDS):
                                         a device-side index check failed; the
                                         access was skipped and the results of
                                         the call are not valid */
} zef_status;

/* zef_add_compartment flags */
#define ZEF_AUTO_ORIENT 1u /* flip every triangle when the signed volume is negative */

/* Arithmetic of zef_label_points */
typedef enum zef_precision {
    ZEF_FP32_RESCUE = 0, /* FP32 solid angles with compensated accumulation;
                            pairs whose result is not certain are re-evaluated
                            in FP64 over the full surface (default) */
    ZEF_FP64_PLAIN = 1,  /* every pair in FP64 (the plain baseline kernel) */
    ZEF_FP32_ONLY = 2    /* FP32 without the FP64 re-evaluation (diagnostics) */
} zef_precision;

typedef struct zef_label_opts {
    /* |Omega32 - 2 pi| < margin marks a (point, compartment) pair uncertain.
       Default 1e-3 (<= 0 selects the default). */
    float margin;
    /* A pair is also uncertain when Omega32 is farther than winding_tol from
       the nearest multiple of 4 pi k (Omega of a closed surface at a point
       off the surface is 4 pi times the winding number k).  A pair that is
       certain reports Omega = 4 pi k exactly.  Default 1e-5 (<= 0 selects
       it): every FP32 sum the library certifies is then within 1e-5 sr of
       the exact solid angle.  The label argument needs far less -- the
       rounding error of an FP32 sum stays orders of magnitude below
       2 pi - winding_tol, and the errors of about 4 pi that a wrong sign of a
       near-zero N can cause are caught by the conditioning test -- so a
       looser value (say 1e-4) re-evaluates fewer pairs with the same labels. */
    float winding_tol;
    /* zef_precision */
    int32_t precision;
    /* Threads per block and points per thread of the FP32 kernel; 0 = the
       autotuned choice.  Valid: threads 128 or 256, points 2 or 4. */
    int32_t block_threads;
    int32_t points_per_thread;
    /* Form of the FP32 kernel: 0 = cap trees (default): for each tile of
       points the patches whose box misses the tile are replaced by their
       caps, exact since outside that box a cap subtends its patch, and the
       remaining leaves and caps are streamed as strips; 1 = the whole surface
       as triangle strips, one atan2 per group of four triangles taken of the
       product of their (D + iN) factors with 2 pi wraps counted exactly;
       2 = whole-surface strips, one atan2 per triangle. */
    int32_t kernel;
    /* ZEF_NO_TILE_COHERENCE, ZEF_POINT_WALK, ZEF_OMEGA_RAW (any
       combination), or 0 (see below). */
    uint32_t flags;
    int32_t reserved;
} zef_label_opts;

/* zef_label_opts.flags.  By default a tile of points whose bounding box meets
   no triangle's bounding box of a compartment -- a convex region the surface
   does not cross, where the winding number is constant -- takes its Omega
   (exactly 4 pi times that winding number) from one representative point;
   the representative must be certain, or the tile is evaluated point by
   point.  This flag evaluates every point instead. */
#define ZEF_NO_TILE_COHERENCE 1u
/* Kernel form 0: by default the points of a tile share one list of leaf and
   cap segments (the tree walked for the tile's box), except where that list
   is longer than 4096 entries and more than three times the longest of the
   points' own walks (a tile whose box spans much of a surface): there every
   point walks the tree for itself.  This flag makes every point walk the
   tree for itself. */
#define ZEF_POINT_WALK 2u
/* Diagnostics: Omega receives the FP32 sum itself (Kahan-compensated, as the
   kernel computed it) for every (point, compartment) pair that the FP32
   kernel evaluated point by point and certified, instead of the certified
   4 pi k.  Pairs decided without their own sum keep their exact 4 pi k (0
   outside the box or hull bound, the representative's k on coherent tiles
   and groups); re-evaluated pairs keep their FP64 sum; with ZEF_FP32_ONLY
   the uncertain pairs keep their FP32 sum.  Labels are unchanged.  Used to
   measure the FP32 arithmetic's own error against the FP64 oracle. */
#define ZEF_OMEGA_RAW 4u

typedef struct zef_label_stats {
    int64_t points;            /* N */
    int64_t nonfinite_points;  /* points with a NaN/Inf coordinate (label -1) */
    int64_t pairs_nominal;     /* N * sum_c T_c */
    int64_t pairs_evaluated;   /* point x triangle pairs computed (FP32 + FP64) */
    int64_t pairs_rescued;     /* point x triangle pairs re-evaluated in FP64 */
    int64_t uncertain_pairs;   /* (point, compartment) pairs sent to FP64 */
    int64_t work_items;        /* (compartment, point tile) items after culling */
    int64_t tiles;             /* point tiles */
    int32_t block_threads;     /* launch shape used */
    int32_t points_per_thread;
    float ms_total;            /* device time of the call (CUDA events) */
    float ms_label;            /* device time of the main labeling kernel */
    float ms_rescue;           /* device time of the FP64 re-evaluation */
    float reserved;
    int64_t coherent_pairs;    /* (point, compartment) pairs decided by the
                                  representative point of a tile or group */
    int64_t representative_pairs; /* of pairs_evaluated: point x triangle pairs
                                     of those representatives */
    int64_t lane_walk_items;   /* kernel form 0: (tile, compartment) pairs whose
                                  points each walked their own cap tree (the
                                  tile's shared list of segments was too long) */
    int64_t kernel_launches;   /* CUDA kernels the library launched for this call
                                  (autotuning runs excluded) */
} zef_label_stats;

/* Mesh for zef_refine_and_relabel.  All four arrays must be device memory or
   all host memory.  Capacities bound the growth: nodes grow by at most six
   per flagged tet and level, tets by seven. */
typedef struct zef_mesh {
    float *nodes;          /* [node_capacity][3] */
    int32_t *tets;         /* [tet_capacity][4], 0-based node indices */
    int32_t *node_labels;  /* [node_capacity] */
    int64_t num_nodes;     /* in: current count; out: count after refinement */
    int64_t num_tets;      /* in/out likewise */
    int64_t node_capacity;
    int64_t tet_capacity;
    int32_t labels_valid;  /* nonzero: node_labels[0, num_nodes) already hold
                              labels; 0: label every node first */
    int32_t flags;         /* ZEF_REFINE_CONFORMING or 0 */
} zef_mesh;

/* zef_mesh.flags: close every level into a conforming mesh (Sec. 2.1.2,
   Fig. 2 c-e).  Besides the 1 -> 8 split of the flagged tets, a tet whose
   split edges are one edge, two edges with a common vertex, or the three
   edges of one face is split into two, three or four ("green"); a tet with
   any other pattern is split into eight as well, repeated until no tet
   changes.  Green templates replace corners by edge midpoints: one edge
   (i, j): T[j<-m], T[i<-m]; two edges (p, q), (p, r) with q < r: the corner
   T[q<-m_pq, r<-m_pr], then T[q<-m_pq, p<-m_pr], T[p<-m_pq] when the quad
   diagonal m_pq-r is not longer than q-m_pr (float32 squared lengths), else
   T[r<-m_pr, p<-m_pq], T[p<-m_pr]; face (p, q, r), p < q < r: the corners
   T[q<-m_pq, r<-m_pr], T[p<-m_pq, r<-m_qr], T[p<-m_pr, q<-m_qr] and the
   centre T[p<-m_qr, q<-m_pr, r<-m_pq].  New nodes are the edge midpoints of
   the tets split into eight, numbered by first appearance over those tets in
   index order; a split tet's slot receives its first child, the other
   children of the eight-way splits are appended in their order, then the
   other children of the green splits in tet index order. */
#define ZEF_REFINE_CONFORMING 1

typedef struct zef_level_stats {
    int64_t flagged_tets;   /* tets whose four node labels were not all equal */
    int64_t new_nodes;      /* unique edge midpoints added and labeled */
    int64_t nodes;          /* node count after the level */
    int64_t tets;           /* tet count after the level */
    int64_t pairs_evaluated;
    int64_t uncertain_pairs;
    int64_t promoted_tets;  /* conforming: tets split into eight by the closure */
    int64_t green_tets;     /* conforming: tets split along one to three edges */
} zef_level_stats;

typedef struct zef_relabel_pass {
    int64_t evaluated;      /* boundary nodes whose solid angles were re-evaluated */
    int64_t changed;        /* of those, nodes whose label changed */
} zef_relabel_pass;

/* Pass as `device` to zef_create for a host-only context: it makes no CUDA
   call; compartments can be registered and validated, while labeling and
   refinement return ZEF_ERR_NOT_READY. */
#define ZEF_HOST_ONLY (-1)

/* Create a context on CUDA device `device` (or ZEF_HOST_ONLY).  `cuda_stream`
   is a cudaStream_t of that device to run on (for example a PyTorch stream);
   NULL makes the context create its own non-blocking stream.  *out is NULL on
   failure. */
zef_status zef_create(zef_ctx **out, int device, void *cuda_stream);

/* Release every resource of the context.  NULL is ignored. */
void zef_destroy(zef_ctx *ctx);

/* Message of the last failing call on this context (static text for a NULL
   context).  Valid until the next call on the context. */
const char *zef_last_error(const zef_ctx *ctx);

/* Register a closed triangulated compartment surface (Sec. 2.1.3: dS closed).
     id     > 0, unique within the context; it is the label of enclosed points
     verts  [nv][3] float32
     tris   [nt][3] int32, 0-based; every undirected edge must be used by
            exactly two triangles, in opposite directions (closed, oriented)
     flags  ZEF_AUTO_ORIENT or 0
   Outward orientation (positive signed volume) is required unless
   ZEF_AUTO_ORIENT is set, in which case an inward surface is flipped.  The
   data are copied; the call synchronizes.  Registration order is the default
   priority order. */
zef_status zef_add_compartment(zef_ctx *ctx, int32_t id, const float *verts, int64_t nv,
                               const int32_t *tris, int64_t nt, uint32_t flags);

/* Number of registered compartments and their total triangle count. */
zef_status zef_compartment_info(const zef_ctx *ctx, int32_t *num_compartments,
                                int64_t *total_triangles);

/* Set the layer hierarchy (Sec. 2.1): `ids` is a permutation of all
   registered ids; ids[0] has the highest priority, i.e. a point enclosed by
   several compartments gets the first of them in this list.  Host array. */
zef_status zef_compartment_priority(zef_ctx *ctx, const int32_t *ids, int32_t n);

/* Label N query points (Sec. 2.1.3 initial labeling, Sec. 2.1 priority).
     pts     [n][3] float32
     labels  [n] int32 out: id of the first compartment in priority order
             whose surface encloses the point (Omega > 2 pi); 0 when none;
             -1 for a point with a non-finite coordinate
     omega   nullable; [C][n] float32 out, row r = the r-th compartment in
             priority order: the solid angle Omega in steradians: 4 pi k
             exactly wherever the winding number k is certified (0 outside
             the compartment's bounding box or convex-hull bound, the tile's
             k where the surface provably does not cross a tile, the FP32
             sum's k within winding_tol), the FP64 sum for the pairs
             re-evaluated in FP64, the FP32 sum with ZEF_FP32_ONLY for
             uncertain pairs; NaN for non-finite points
     opts    nullable = defaults;  stats nullable (non-NULL synchronizes) */
zef_status zef_label_points(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                            float *omega, const zef_label_opts *opts, zef_label_stats *stats);

/* Pipelined labeling of batches in host memory: the labels of
   zef_label_points (Sec. 2.1.3 initial labeling, Sec. 2.1 priority) without
   waiting for them.  The call enqueues the copy of pts into one of two
   device staging slots (used in turn) on a copy-in stream, the labeling on
   the context stream and the copy of the labels back on a copy-out stream,
   and returns; so the copy-in of the next call and the copy-out of this one
   run while the neighbouring calls label.
     pts     [n][3] float32, host or device; host memory should be
             page-locked (pageable memory is copied synchronously, without
             overlap); it must stay unchanged until zef_synchronize returns
     labels  [n] int32 out, host or device; complete after zef_synchronize
     opts    nullable = defaults
   No solid angles or statistics (use zef_label_points).  Argument errors
   return at once; errors of the device work are returned by the next
   zef_synchronize, which waits for all three streams.  A slot whose
   capacity grows waits for its previous use and reallocates. */
zef_status zef_label_points_async(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                                  const zef_label_opts *opts);

/* Element labels by the four-nodes rule (Sec. 2.1.3: a tetrahedron whose
   four nodes all lie inside dS is an element of S) under the priority order
   of Sec. 2.1: the label of a tet is the first compartment in priority order
   whose surface encloses all four of its nodes (Omega > 2 pi at each), 0 when
   none does, -1 when one of its nodes has a non-finite coordinate.  Every
   (node, compartment) pair is decided (no priority early exit): a node
   labeled with one compartment may also lie inside a later one.
     nodes        [n_nodes][3] float32
     tets         [n_tets][4] int32 node indices, 0 <= index < n_nodes
     elem_labels  [n_tets] int32 out
     node_labels  nullable; [n_nodes] int32 out, as zef_label_points' labels
     opts, stats  as zef_label_points; stats describe the node labeling
   Host or device arrays (the rules of zef_label_points).  A tet with an index
   outside [0, n_nodes) gets -1 and the call returns ZEF_ERR_INVALID_ARG (an
   all-device call without stats does not synchronize: the next
   zef_synchronize reports it). */
zef_status zef_label_elements(zef_ctx *ctx, const float *nodes, int64_t n_nodes,
                              const int32_t *tets, int64_t n_tets, int32_t *elem_labels,
                              int32_t *node_labels, const zef_label_opts *opts,
                              zef_label_stats *stats);

/* Largest point count of one zef_label_points_noalloc call. */
#define ZEF_NOALLOC_MAX_POINTS 65536

/* zef_label_points that allocates nothing during the call.  The paper has no
   counterpart; this exists for callers that cannot let a library allocate
   device memory: cudaMalloc / cudaFree may synchronize the whole device and
   stall every other stream (fatal to a latency-critical loop), and a
   framework that owns a fixed device-memory budget through its own allocator
   cannot have memory taken behind its back.
     pts, labels, omega, opts, stats: as zef_label_points, but pts, labels and
             omega must be DEVICE pointers (ZEF_ERR_INVALID_ARG otherwise)
     n       0 <= n <= ZEF_NOALLOC_MAX_POINTS, else ZEF_ERR_INVALID_ARG
   All scratch comes from one fixed-size array compiled into the library
   (about 12 MB, held on every GPU that loads the library until the process
   exits).  The compartments must already be registered (ZEF_ERR_NOT_READY
   otherwise).  Every call looks up the array's device address on the
   context's device (cudaGetSymbolAddress); the first call on a device may
   load the library's device code, so make that first call before any
   stream capture.  Every call in the process shares the one array of its
   device, which keeps the last call's contents; each call clears what must
   start at zero.  Calls that overlap on the GPU (other streams, contexts or
   host threads) race on the array and corrupt each other's results:
   serialize them. */
zef_status zef_label_points_noalloc(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                                    float *omega, const zef_label_opts *opts, zef_label_stats *stats);

/* Recursive refinement and re-labeling (Sec. 2.1.2, Sec. 2.1.3 item 2):
   `levels` times, every tet whose four node labels are not all equal is split
   into eight (one new node per edge midpoint, shared between tets), and only
   the new nodes are labeled.  The flagged tet's slot receives its first child;
   the other seven are appended.  The level loop runs as one CUDA graph with
   device-resident counts.  per_level: nullable, `levels` entries. */
zef_status zef_refine_and_relabel(zef_ctx *ctx, zef_mesh *mesh, int32_t levels,
                                  const zef_label_opts *opts, zef_level_stats *per_level);

/* Recursive re-labeling at the tissue boundaries (Sec. 2.1.3 item 2, Fig. 3)
   after the nodes of a labeled mesh changed (moved, or the surfaces were
   replaced).  One pass: the tets whose four node labels are not all equal
   form the boundary; the nodes of those tets that this call has not yet
   evaluated are re-labeled with the solid-angle method; a changed label can
   move the boundary.  Passes repeat until one changes no label (the boundary
   no longer changes) or `max_passes` (1..1024) passes ran.  Each node is
   evaluated at most once per call (its position does not change during it).
   The pass loop runs on the device as one CUDA graph with a conditional
   while-node: no host round trip between passes.
     nodes        [n_nodes][3] float32
     tets         [n_tets][4] int32 node indices, 0 <= index < n_nodes
     node_labels  [n_nodes] int32, in: the current labels, out: repaired
     opts         as zef_label_points (nullable)
     per_pass     nullable; max_passes entries (passes not run are zeroed)
     passes, converged  nullable outs: passes run; 1 when the last pass
                  changed no label, 0 when the pass limit stopped the loop
   nodes, tets and node_labels must all be host or all device memory; the
   call synchronizes.  An index outside [0, n_nodes) stops the loop and
   returns ZEF_ERR_INVALID_ARG. */
zef_status zef_relabel_boundary(zef_ctx *ctx, const float *nodes, int64_t n_nodes,
                                const int32_t *tets, int64_t n_tets, int32_t *node_labels,
                                int32_t max_passes, const zef_label_opts *opts,
                                zef_relabel_pass *per_pass, int32_t *passes, int32_t *converged);

/* Taubin smoothing parameters (Sec. 2.2.1; the experiments of the paper use
   lambda = mu = 0.4). */
typedef struct zef_smooth_opts {
    float lambda;       /* forward step, 0 <= lambda < 1 */
    float mu;           /* backward step, 0 <= mu < 1 */
    float xi;           /* stop after the first iteration whose forward step
                           satisfies ||x' - x||_2 / ||x^(0)||_2 <= xi */
    int32_t max_iters;  /* 1 .. 100000 */
} zef_smooth_opts;

/* Taubin smoothing of the mesh nodes in place (Sec. 2.2.1, volumetric: the
   neighbourhood N_i of node i is i itself and every node joined to it by a
   tet edge).  One iteration: x' = x + lambda L(x), then x'' = x' - mu L(x'),
   with L(x)_i = sum over j in N_i of (x_j - x_i) / |N_i|, summed in
   ascending neighbour order in float32 (deterministic); nodes with
   fixed[i] != 0 (nullable array) do not move.  The iteration loop runs on
   the device as one CUDA graph with a conditional while-node.
     nodes      [n_nodes][3] float32, in/out
     tets       [n_tets][4] int32 node indices
     fixed      nullable; [n_nodes] uint8
     iterations nullable out: iterations run
   nodes, tets and fixed must all be host or all device memory; the call
   synchronizes.  Errors: ZEF_ERR_INVALID_ARG (parameters, an index outside
   [0, n_nodes), mixed residency), ZEF_ERR_NOT_READY (host-only context). */
zef_status zef_taubin_smooth(zef_ctx *ctx, float *nodes, int64_t n_nodes, const int32_t *tets,
                             int64_t n_tets, const uint8_t *fixed, const zef_smooth_opts *opts,
                             int32_t *iterations);

/* Taubin smoothing of the tissue boundaries (Sec. 2.2.1: both the volume and
   the tissue boundaries are smoothed; the paper's experiments stop the
   boundary smoothing at xi = 0.1).  A boundary face is a triangle shared by
   two tets whose element labels differ (a face of a single tet lies on the
   mesh's outer boundary, not between tissues).  The neighbourhood N_i of a
   node on a boundary face is the node and every node joined to it by an edge
   of a boundary face; the iteration is zef_taubin_smooth's over that graph,
   so nodes on no boundary face do not move, and the norms of the stopping
   rule run over the boundary nodes.
     nodes           [n_nodes][3] float32, in/out
     tets            [n_tets][4] int32 node indices
     elem_labels     [n_tets] int32 element labels (zef_label_elements' output,
                     or any other labeling)
     opts            as zef_taubin_smooth
     iterations      nullable out: iterations run (0 when there is no
                     boundary face)
     boundary_faces  nullable out: boundary faces found
   nodes, tets and elem_labels must all be host or all device memory; the
   call synchronizes.  Errors as zef_taubin_smooth. */
zef_status zef_taubin_smooth_surface(zef_ctx *ctx, float *nodes, int64_t n_nodes, const int32_t *tets,
                                     int64_t n_tets, const int32_t *elem_labels, const zef_smooth_opts *opts,
                                     int32_t *iterations, int64_t *boundary_faces);

/* One inflation of the nodes inside compartment `compartment_id`'s surface S
   towards S (Sec. 2.2.2).  A mesh edge with one node inside S (Omega > 2 pi)
   and the other outside crosses S; the inside node i moves by
   zeta t (x_j - x_i) averaged over its crossing edges (i, j), t the edge
   parameter of the intersection with S nearest to x_i (float32
   Moller-Trumbore against S's triangles, inclusive by 2^-20 so that an edge
   through a shared triangle edge still hits), i.e. by zeta times the
   distance to S along the unit edge vector.  Every other node keeps its
   position.
     nodes  [n_nodes][3] float32, in/out;  tets [n_tets][4] int32
     zeta   0 <= zeta < 1 (0.05 in the paper's experiments)
     moved  nullable out: nodes moved
   nodes and tets must both be host or both device memory; the call
   synchronizes.  Errors: ZEF_ERR_INVALID_ARG (unknown id, zeta, an index
   outside [0, n_nodes)), ZEF_ERR_NOT_READY. */
zef_status zef_inflate(zef_ctx *ctx, float *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                       int32_t compartment_id, float zeta, int64_t *moved);

/* Wait for the context's stream (and the copy streams of
   zef_label_points_async) and report any error a kernel recorded
   (ZEF_ERR_TIMEOUT, ZEF_ERR_CAPACITY, ZEF_ERR_BOUNDS). */
zef_status zef_synchronize(zef_ctx *ctx);

/* Library version, encoded as major * 1000 + minor. */
int32_t zef_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ZEF_H */
