// Internal declarations of libzef (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "zef.h"

namespace zef {

// NVTX range over a host scope (a profiler attached through NVTX shows the
// library's stages by these names; without one the calls cost nothing).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  // end this range and open the next stage's
  void next(const char *name) {
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// One strip-stream entry, 32 bytes (two float4, TMA-friendly):
//   v = (x, y, z, weight): the vertex entering the sliding triangle window;
//       weight 1 when the window (previous two vertices + this one) is a
//       triangle of the surface, 0 for the two entries that prime a strip;
//   n = (nx, ny, nz, kappa): that triangle's doubled-area normal with the
//       surface's orientation, and kappa = KAPPA * |n| for the conditioning
//       test; n = 0 and kappa = 0 on the other entries, whose windows repeat
//       a vertex (so N = 0, D >= 0: an identity factor).
struct __align__(16) Entry {
  float4 v;
  float4 n;
};

// Device view of one compartment.
struct __align__(16) DevComp {
  float lo[3];
  float hi[3];
  int32_t entry_off;  // first Entry of the compartment (multiple of 16)
  int32_t entry_cnt;  // number of entries, padded to a multiple of 16
  int32_t tri_off;    // first triangle in the plain triangle list
  int32_t tri_cnt;
  int32_t id;         // user id
  int32_t row;        // priority row (0 = highest priority)
  int32_t cap_root;   // root of the cap tree (zef_tree.cpp)
  int32_t cseg_off;   // first entry of the compartment's cap-tree segment block
  int32_t cseg_leaf;  // entries of its leaf segments (the caps' follow)
  int32_t pad_;
};

// Node of a compartment's cap tree (zef_tree.cpp): the box of the patch's
// vertices, children (-1 for a leaf), the leaf's strip segment and the
// node's cap segment (entries of the cap-tree segment array) with the
// triangles each holds.  Nodes are stored in pre-order, so a depth-first
// walk needs no stack: descend to this + 1, or continue at skip.
constexpr int kCapLeaf = 64;  // most triangles of a leaf
struct __align__(16) CapNode {
  float lo[3];
  int32_t left;
  float hi[3];
  int32_t right;
  int32_t leaf_begin, leaf_cnt;  // leaf: strip segment of its triangles
  int32_t cap_begin, cap_cnt;    // the node's cap: zigzag strip segment
  int32_t leaf_tris, cap_tris;
  int32_t tri_begin;             // leaf: first of its triangles in the tree-ordered index array
  int32_t skip;                  // the node after this subtree in pre-order (left child = this + 1)
};
static_assert(sizeof(CapNode) == 64, "CapNode is four 16-byte words");
void build_cap_tree(const float *V, const int32_t *T, int64_t nt, int64_t node_base, int64_t seg_base,
                    int64_t tidx_base, std::vector<CapNode> &nodes, std::vector<Entry> &seg,
                    std::vector<int32_t> &tidx, int32_t *root, int64_t *leaf_entries);

// Device status word bits (ctx->d_status[0]); [1] holds detail.
enum : uint32_t {
  ST_TIMEOUT = 1u,
  ST_CAPACITY = 2u,
  ST_INVALID = 4u,
  ST_BOUNDS = 8u,   // debug build: a device-side index check failed
};

// Debug build (compiled with ZEF_DEBUG_BOUNDS): the labeling kernels check the
// indices they compute before they use them; a failed check records
// ST_BOUNDS with a site code in the context's status word and skips the
// access (it never traps).  In the release build every check is `true`.
#if defined(ZEF_DEBUG_BOUNDS) && defined(__CUDACC__)
__device__ __forceinline__ bool bounds_ok(bool ok, uint32_t *status, uint32_t site) {
  if (!ok) {
    atomicOr(status, ST_BOUNDS);
    atomicExch(status + 1, site);
  }
  return ok;
}
#define ZEF_BOUNDS_OK(cond, status, site) ::zef::bounds_ok((cond), (status), (site))
#else
#define ZEF_BOUNDS_OK(cond, status, site) true
#endif

// every zef_label_opts.flags bit the library knows
constexpr uint32_t kLabelFlagsAll = ZEF_NO_TILE_COHERENCE | ZEF_POINT_WALK | ZEF_OMEGA_RAW;

constexpr int kGroup = 16;        // Kahan group: entries summed plainly before compensation
constexpr int kChunk = 256;       // entries per TMA chunk
constexpr int kTriChunk = 128;    // plain triangles per TMA chunk (FP64 baseline)
constexpr float kKappa = 1.0f / 8192.0f;  // conditioning threshold of a pair
constexpr int kMortonBits = 7;    // bits per axis of the binning key
constexpr int kBuckets = 1 << (3 * kMortonBits);
// binning keys past the Morton cells: finite points outside the surfaces'
// union box, then non-finite points (the two tails of the sorted order, in
// that order; their points are labelled by the key pass and not scattered,
// so each tail's count is one histogram word, added once per block)
constexpr uint32_t kKeyOutside = (uint32_t)kBuckets;
constexpr uint32_t kKeyNonfinite = (uint32_t)kBuckets + 1;
constexpr int64_t kHistLen = (int64_t)kBuckets + 2;  // key histogram / cursor entries
constexpr int kWorkBuckets = 4096;                    // log-scale work buckets of the tile list
// exclusive scan: threads per block, values per thread, values per block
constexpr int kScanT = 256;
constexpr int kScanV = 8;
constexpr int kScanB = kScanT * kScanV;
// block sums needed to scan len values (one per block, plus one spare)
constexpr int64_t scan_block_sums(int64_t len) { return (len + kScanB - 1) / kScanB + 1; }

// Union box of the registered surfaces in the caller's (unscaled)
// coordinates, with the Morton cell scale 2^kMortonBits / extent per axis.
struct UnionBox {
  float lo[3], hi[3], sc[3];
};

// Convex-hull bound of a compartment: kDop fixed unit directions d_k (a
// Fibonacci sphere); h_k >= max over the surface's vertices of d_k . v, with
// a conservative rounding margin.  A point p with d_k . p > h_k for some k lies
// outside the convex hull of the closed surface, where its winding number --
// hence Omega -- is exactly 0.
constexpr int kDop = 96;
void dop_directions(float (*dirs)[3]);  // fills kDop unit vectors (host)

struct CompHost {
  int32_t id;
  int64_t nv, nt;
  float lo[3], hi[3];
  int64_t entry_off, entry_cnt, tri_off, nstrips;
  int32_t cap_root;                // cap tree: root node, segment block, leaf entries
  int64_t cseg_off, cseg_leaf;
  double dop[kDop];  // max over the vertices of d_k . v (unscaled coordinates)
};

// Grow-only device buffers of the labeling pipeline.
struct LabelBuffers {
  int64_t cap_points = 0;   // points the buffers hold
  int64_t cap_tiles = 0;
  int64_t cap_items = 0;
  int64_t cap_unc = 0;      // capacity of unc_list (0: no list)
  float4 *spts = nullptr;       // sorted points (x, y, z, unused)
  int32_t *perm = nullptr;      // sorted position -> original index
  uint32_t *keys = nullptr;     // binning key per original point
  unsigned long long *in_mask = nullptr;   // per sorted point: inside bits (priority rows)
  unsigned long long *unc_mask = nullptr;  // per sorted point: uncertain bits
  float *tile_box = nullptr;    // [tiles][6]
  uint32_t *hist = nullptr;     // kHistLen key cursor, then kWorkBuckets work cursor
  uint32_t *flags = nullptr;    // [C * tiles] work-list flags, scanned in place
  uint32_t *block_sums = nullptr;
  int2 *items = nullptr;        // (tile, comp)
  int2 *unc_list = nullptr;     // uncertain (sorted point, priority row) pairs
  int64_t *counters = nullptr;  // device counters, see Counter enum
  int32_t *labels_tmp = nullptr;
  float *pts_tmp = nullptr;     // staging for host inputs
  float *omega_tmp = nullptr;
  int64_t cap_omega = 0;
  float *tune_pts = nullptr;    // autotuner sample (2^20 points)
};

constexpr int64_t kUncListCap = 1 << 15;  // uncertain-pair list of the cap-tree re-evaluation
constexpr int kSplitPairs = 1024;         // up to this many listed pairs split over several blocks
constexpr int kMaxParts = 8;              // blocks per split pair
// the list, then the split pairs' partial sums and completion counts
constexpr size_t kUncBytes = (size_t)kUncListCap * 8 + (size_t)kSplitPairs * kMaxParts * 8 + (size_t)kSplitPairs * 4;

enum Counter {
  CNT_N = 0,          // points of this call
  CNT_OFF,            // offset of the first point in the caller's array
  CNT_ITEMS,          // work items
  CNT_WORK,           // persistent-kernel work cursor
  CNT_UNC,            // uncertain (point, comp) pairs
  CNT_UNC_WORK,       // rescue cursor
  CNT_NONFINITE,
  CNT_PAIRS_EVAL,     // FP32 (or FP64 plain) pairs
  CNT_PAIRS_RESCUE,   // FP64 re-evaluation pairs
  CNT_NIN,            // sorted points inside the surfaces' union box (they come first)
  CNT_NFIN,           // finite points (the non-finite ones are the sorted tail)
  CNT_SPARE,
  CNT_TILES,
  CNT_LEVEL_FLAGGED,  // refinement
  CNT_LEVEL_NEW,
  CNT_NODES,
  CNT_TETS,
  CNT_ABORT,          // refinement stopped (capacity)
  CNT_OWN_LEN,        // 6 x flagged tets of the level
  CNT_COHERENT,       // (point, compartment) pairs decided by a tile representative
  CNT_REP_PAIRS,      // point x triangle pairs of tile and group representatives
  CNT_LEVEL_SEED,     // conforming refinement: tets flagged by their labels
  CNT_CL_CHANGED,     // closure: tets promoted in the current pass
  CNT_CL_ITER,        // closure passes of the level
  CNT_CL_GREEN,       // tets split along one to three edges
  CNT_CL_GEXTRA,      // children those splits add
  CNT_LANE_TILES,     // cap trees: (tile, compartment) pairs evaluated by per-lane walks
  CNT_UNC_LIST,       // uncertain pairs appended to the pair list (may exceed its capacity)
  CNT_COUNT_ = 32
};

// zef_label_opts.kernel -> kernel template form: 0 (default) cap trees = 2,
// 1 strips with grouped products = 0, 2 strips with one atan2 per triangle = 1
inline int kernel_variant(int kernel) { return kernel == 0 ? 2 : kernel - 1; }

struct LaunchShape {
  int threads;
  int ppt;
  int variant = 0;  // zef_label_opts.kernel
};

}  // namespace zef

struct zef_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::string err;

  std::vector<zef::CompHost> comps;
  std::vector<int32_t> priority;      // ids, highest priority first
  std::vector<zef::Entry> h_entries;
  std::vector<float4> h_tris;         // 3 per triangle (w unused)
  std::vector<zef::CapNode> h_nodes;  // cap trees of all compartments
  std::vector<zef::Entry> h_cseg;     // cap-tree strip segments
  std::vector<int32_t> h_ctidx;       // cap-tree leaves' triangles (compartment-local indices), tree order

  bool dirty = true;
  uint64_t gen = 0;   // upload generation: cached graphs keyed on it see every change of the surfaces
  // power of two applied to every coordinate on the device so that the
  // registered surfaces fit in [-64, 64]^3 (exact; solid angles are scale
  // invariant); keeps products of four (D, N) factors far from overflow
  float scale = 1.f;
  zef::Entry *d_entries = nullptr;
  float4 *d_tris = nullptr;
  zef::DevComp *d_comps = nullptr;
  int32_t *d_row_ids = nullptr;       // priority row -> id
  int32_t *d_lpt = nullptr;           // LPT rank -> comp index
  float *d_dop = nullptr;             // [C][kDop] hull support bounds (scaled coordinates)
  zef::CapNode *d_nodes = nullptr;    // cap trees (scaled)
  zef::Entry *d_cseg = nullptr;       // cap-tree strip segments (scaled)
  int32_t *d_ctidx = nullptr;         // cap-tree leaves' triangles
  int64_t d_ctidx_cap = 0;
  int64_t d_nodes_cap = 0, d_cseg_cap = 0;
  int64_t d_entries_cap = 0, d_tris_cap = 0;

  uint32_t *d_status = nullptr;       // [2]
  zef::LabelBuffers lb;
  int64_t *h_counters = nullptr;      // pinned mirror of the counters

  cudaEvent_t ev[6] = {};
  zef::UnionBox ubox = {};            // union box of the surfaces (unscaled), set at upload
  int64_t launches = 0;               // kernels launched by the labeling pipeline (running count)

  // autotuner cache: key -> shape
  std::vector<std::pair<uint64_t, zef::LaunchShape>> tune_cache;

  // zef_label_points_async: a copy-in and a copy-out stream beside the
  // context stream, and two staging slots used in turn, so that one call's
  // copies overlap the neighbouring calls' labeling.  Events: h2d (slot's
  // points landed), done (labeling that read the slot finished), d2h
  // (slot's labels copied out).
  struct PipeSlot {
    float *pts = nullptr;
    int32_t *labels = nullptr;
    int64_t cap = 0;
    cudaEvent_t h2d = nullptr, done = nullptr, d2h = nullptr;
  };
  cudaStream_t s_in = nullptr, s_out = nullptr;
  PipeSlot pipe[2];
  int pipe_next = 0;

  // element-label scratch (zef_label_elements)
  int32_t *el_node_labels = nullptr;
  unsigned long long *el_masks = nullptr;
  int32_t *el_tets = nullptr;
  int32_t *el_labels = nullptr;
  int64_t el_cap_nodes = 0, el_cap_masks = 0, el_cap_tets = 0, el_cap_labels = 0;

  // post-processing scratch (smoothing, inflation)
  void *pp_buf[18] = {};
  size_t pp_cap[18] = {};

  // recursive re-labeling scratch and its cached graph
  void *rb_buf[9] = {};
  size_t rb_cap[9] = {};
  cudaGraphExec_t rb_exec = nullptr;
  uint64_t rb_key = 0;

  // refinement scratch
  void *rf_buf[10] = {};
  size_t rf_cap[10] = {};
  cudaGraphExec_t rf_exec = nullptr;
  uint64_t rf_key = 0;
};

namespace zef {

// ---- host helpers (zef_host.cpp)
zef_status fail(zef_ctx *ctx, zef_status st, const std::string &msg);
zef_status cuda_fail(zef_ctx *ctx, cudaError_t e, const char *what);
zef_status ensure_uploaded(zef_ctx *ctx);
zef_status label_points_impl(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels, float *omega,
                             const zef_label_opts *opts, zef_label_stats *stats, unsigned long long *d_masks,
                             bool full_masks);
zef_status label_points_async_impl(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                                   const zef_label_opts *opts);
template <class T>
zef_status ensure_buffer(zef_ctx *ctx, T **p, int64_t *cap, int64_t need);

// ---- labeling pipeline (zef_label.cu)
struct LabelPlan {
  const float *pts;          // base of the caller's point array (device)
  int32_t *labels;           // base of the label array (device)
  float *omega;              // nullable, [C][n_cap] rows (device)
  int64_t omega_ld;          // row stride of omega
  int64_t n_cap;             // upper bound of the points of this call
  const int64_t *d_n;        // device: number of points
  const int64_t *d_off;      // device: offset of the first point
  zef_label_opts opts;
  LaunchShape shape;
  bool timed;                // record events around the main kernels
  unsigned long long *masks = nullptr;  // nullable: per-point inside bits (priority rows), caller's order
  bool full_masks = false;   // evaluate every compartment (no priority early exit)
};

zef_status label_reserve(zef_ctx *ctx, int64_t n_cap);
zef_status label_enqueue(zef_ctx *ctx, const LabelPlan &plan);
zef_status label_set_count(zef_ctx *ctx, int64_t n, int64_t off);
zef_status launch_wait_probe(zef_ctx *ctx, int64_t limit_ns);
zef_status relabel_run(zef_ctx *ctx, const float *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                       int32_t *node_labels, int32_t max_passes, const zef_label_opts &opts,
                       zef_relabel_pass *per_pass, int32_t *passes, int32_t *converged);
zef_status taubin_run(zef_ctx *ctx, float *nodes, int64_t n, const int32_t *tets, int64_t m, const uint8_t *fixed,
                      const zef_smooth_opts &o, int32_t *iters_out);
zef_status inflate_run(zef_ctx *ctx, float *nodes, int64_t n, const int32_t *tets, int64_t m, int32_t id,
                       float zeta, int64_t *moved_out);
zef_status taubin_surface_run(zef_ctx *ctx, float *nodes, int64_t n, const int32_t *tets, int64_t m,
                              const int32_t *elem_labels, const zef_smooth_opts &o, int32_t *iters_out,
                              int64_t *faces_out);
zef_status launch_elem_labels(zef_ctx *ctx, const int32_t *tets, int64_t n_tets, int64_t n_nodes,
                              const int32_t *node_labels, const unsigned long long *masks, int32_t *elem);
zef_status debug_fma_rate(zef_ctx *ctx, int fp64, double *tflops);
zef_status launch_debug_half_angle(zef_ctx *ctx, const float *y, const float *x, float *out, int64_t n);
zef_status upload_dop_directions(zef_ctx *ctx);
zef_status scan_exclusive(zef_ctx *ctx, uint32_t *data, const int64_t *len_ptr, int64_t len_mul,
                          int64_t len_cap, int64_t *total_out, uint32_t *bsums);
int grid_blocks(zef_ctx *ctx, int64_t work, int threads);
LaunchShape choose_shape(zef_ctx *ctx, const zef_label_opts &o, int64_t n, bool *need_tune);
zef_status autotune(zef_ctx *ctx, const LabelPlan &plan, LaunchShape *best);
void fill_default_opts(zef_label_opts *o);
bool shape_valid(int threads, int ppt);

// ---- refinement (zef_refine.cu)
zef_status refine_run(zef_ctx *ctx, zef_mesh *mesh, int32_t levels, const zef_label_opts &opts,
                      zef_level_stats *per_level);

}  // namespace zef
