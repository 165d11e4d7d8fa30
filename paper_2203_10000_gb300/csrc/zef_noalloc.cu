// zef_label_points_noalloc: zef_label_points for callers that must not
// allocate device memory during the call.
//
// Why: cudaMalloc / cudaFree can synchronize the whole device and stall every
// stream on it, and some callers run under a fixed device-memory budget owned
// by their own allocator.  A latency-critical loop, or a framework that hands
// out every byte of device memory itself, cannot let the library allocate
// behind its back.  zef_label_points grows its work buffers on demand; this
// entry point instead takes all of its scratch from the file-scope array
// below, whose size is fixed at compile time.
//
// The array is a static __device__ object: every GPU that loads the library
// holds it (kScratchBytes, about 12 MB) until the process exits.  In host
// code its name is only a host-side stand-in, so every call looks up its
// device address with cudaGetSymbolAddress on the context's device (made
// current).  The lookup is not cached: a cached address would dangle after
// cudaDeviceReset, which rebuilds the device's context and reloads the
// library's device code.
#include <cuda_runtime.h>

#include <cstring>

#include "zef_internal.h"

namespace {

using namespace zef;

constexpr int64_t kMaxPoints = ZEF_NOALLOC_MAX_POINTS;
constexpr int64_t kMinTile = 32 * 2;                         // smallest tile of any shape
constexpr int64_t kMaxTiles = (kMaxPoints + kMinTile - 1) / kMinTile;
constexpr int64_t kMaxFlags = kMaxTiles * ZEF_MAX_COMPARTMENTS;  // FP64 (tile, compartment) flags
// block sums of the largest scan the pipeline runs here: the key histogram,
// or the FP64 kernel's flags
constexpr int64_t kMaxBlockSums = scan_block_sums(kHistLen > kMaxFlags ? kHistLen : kMaxFlags);

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the pieces inside the scratch array
constexpr size_t kOffSpts = 0;
constexpr size_t kOffPerm = align256(kOffSpts + kMaxPoints * sizeof(float4));
constexpr size_t kOffKeys = align256(kOffPerm + kMaxPoints * sizeof(int32_t));
constexpr size_t kOffIn = align256(kOffKeys + kMaxPoints * sizeof(uint32_t));
constexpr size_t kOffUnc = align256(kOffIn + kMaxPoints * sizeof(unsigned long long));
constexpr size_t kOffBox = align256(kOffUnc + kMaxPoints * sizeof(unsigned long long));
constexpr size_t kOffHist = align256(kOffBox + kMaxTiles * 6 * sizeof(float));
constexpr size_t kOffFlags = align256(kOffHist + (kHistLen + kWorkBuckets) * sizeof(uint32_t));
constexpr size_t kOffSums = align256(kOffFlags + kMaxFlags * sizeof(uint32_t));
constexpr size_t kOffItems = align256(kOffSums + kMaxBlockSums * sizeof(uint32_t));
constexpr size_t kOffUncList = align256(kOffItems + kMaxFlags * sizeof(int2));
constexpr size_t kOffCnt = align256(kOffUncList + kUncBytes);
constexpr size_t kScratchBytes = align256(kOffCnt + CNT_COUNT_ * sizeof(int64_t));

// What the pipeline may touch must fit the pieces above: tiles of the
// smallest shape (32 x 2 points) over kMaxPoints points, the (tile,
// compartment) flags and items of the plain FP64 kernel (tiles of 256 points,
// so at most kMaxTiles of them as well), the block sums of the key scan and
// of the flag scan, and the uncertain-pair list.
static_assert(kMaxTiles * kMinTile >= kMaxPoints, "tile boxes and keys cover every point");
static_assert(kMaxFlags >= kMaxTiles * ZEF_MAX_COMPARTMENTS, "FP64 flags and items");
static_assert(kMaxBlockSums >= scan_block_sums(kHistLen), "block sums of the key scan");
static_assert(kMaxBlockSums >= scan_block_sums(kMaxFlags), "block sums of the flag scan");
static_assert(kOffCnt - kOffUncList >= kUncBytes, "uncertain-pair list");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device.
cudaError_t scratch_address(void **out) { return cudaGetSymbolAddress(out, g_scratch); }

bool device_pointer(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" zef_status zef_label_points_noalloc(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                                               float *omega, const zef_label_opts *opts,
                                               zef_label_stats *stats) {
  NvtxRange nvtx_("zef.label_points_noalloc");
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context cannot label");
  if (ctx->comps.empty()) return fail(ctx, ZEF_ERR_NOT_READY, "no compartment registered");
  if (ctx->dirty) return fail(ctx, ZEF_ERR_NOT_READY, "compartments are not uploaded");
  if (n < 0 || n > kMaxPoints)
    return fail(ctx, ZEF_ERR_INVALID_ARG,
                "zef_label_points_noalloc takes at most ZEF_NOALLOC_MAX_POINTS (65536) points");
  if (n > 0 && (!pts || !labels)) return fail(ctx, ZEF_ERR_INVALID_ARG, "bad points/labels arguments");
  zef_label_opts o;
  if (opts) o = *opts; else std::memset(&o, 0, sizeof(o));
  fill_default_opts(&o);
  if (o.precision < 0 || o.precision > 2 || o.kernel < 0 || o.kernel > 2)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad precision or kernel");
  if (o.flags & ~kLabelFlagsAll) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown label flags");
  if ((o.block_threads || o.points_per_thread) && !shape_valid(o.block_threads, o.points_per_thread))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad launch shape (threads 128/256, points 2/4)");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n == 0) return ZEF_OK;

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev != ctx->device ? prev : -1};

  if (!device_pointer(pts, ctx->device) || !device_pointer(labels, ctx->device) ||
      (omega && !device_pointer(omega, ctx->device)))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "zef_label_points_noalloc needs device pointers");
  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
  unsigned char *s = static_cast<unsigned char *>(base);

  LabelBuffers view;
  view.cap_points = kMaxPoints;
  view.cap_tiles = kMaxTiles;
  view.cap_items = kMaxFlags;
  view.spts = reinterpret_cast<float4 *>(s + kOffSpts);
  view.perm = reinterpret_cast<int32_t *>(s + kOffPerm);
  view.keys = reinterpret_cast<uint32_t *>(s + kOffKeys);
  view.in_mask = reinterpret_cast<unsigned long long *>(s + kOffIn);
  view.unc_mask = reinterpret_cast<unsigned long long *>(s + kOffUnc);
  view.tile_box = reinterpret_cast<float *>(s + kOffBox);
  view.hist = reinterpret_cast<uint32_t *>(s + kOffHist);
  view.flags = reinterpret_cast<uint32_t *>(s + kOffFlags);
  view.block_sums = reinterpret_cast<uint32_t *>(s + kOffSums);
  view.items = reinterpret_cast<int2 *>(s + kOffItems);
  view.unc_list = reinterpret_cast<int2 *>(s + kOffUncList);
  view.cap_unc = kUncListCap;
  view.counters = reinterpret_cast<int64_t *>(s + kOffCnt);

  LabelPlan plan;
  plan.pts = pts;
  plan.labels = labels;
  plan.omega = omega;
  plan.omega_ld = n;
  plan.n_cap = n;
  plan.d_n = view.counters + CNT_N;
  plan.d_off = view.counters + CNT_OFF;
  plan.opts = o;
  if (o.precision == ZEF_FP64_PLAIN) plan.shape = LaunchShape{128, 2};
  else if (o.block_threads) plan.shape = LaunchShape{o.block_threads, o.points_per_thread, kernel_variant(o.kernel)};
  else plan.shape = LaunchShape{256, 2, kernel_variant(o.kernel)};
  plan.timed = stats != nullptr;

  // The pipeline enqueues its kernels with the pointers of ctx->lb; point it
  // at the static scratch for the duration of the enqueue only.  Every piece
  // that must start at zero is cleared by the pipeline itself (counters,
  // histogram, masks, Omega).
  LabelBuffers saved = ctx->lb;
  ctx->lb = view;
  const int64_t launches0 = ctx->launches;
  zef_status st = label_set_count(ctx, n, 0);
  if (st == ZEF_OK) st = label_enqueue(ctx, plan);
  const int64_t launches = ctx->launches - launches0;
  ctx->lb = saved;
  if (st) return st;
  if (stats) {
    st = zef_synchronize(ctx);
    if (st) return st;
    e = cudaMemcpy(ctx->h_counters, view.counters, CNT_COUNT_ * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read counters");
    const int64_t *h = ctx->h_counters;
    int64_t tt = 0;
    for (auto &c : ctx->comps) tt += c.nt;
    stats->points = n;
    stats->nonfinite_points = h[CNT_NONFINITE];
    stats->pairs_nominal = n * tt;
    stats->pairs_rescued = h[CNT_PAIRS_RESCUE];
    stats->pairs_evaluated = h[CNT_PAIRS_EVAL] + h[CNT_PAIRS_RESCUE];
    stats->uncertain_pairs = h[CNT_UNC];
    stats->work_items = h[CNT_ITEMS];
    stats->tiles = h[CNT_TILES];
    stats->coherent_pairs = h[CNT_COHERENT];
    stats->representative_pairs = h[CNT_REP_PAIRS];
    stats->lane_walk_items = h[CNT_LANE_TILES];
    stats->kernel_launches = launches;
    stats->block_threads = plan.shape.threads;
    stats->points_per_thread = plan.shape.ppt;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[5]);
    stats->ms_total = ms;
    cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
    stats->ms_label = ms;
    cudaEventElapsedTime(&ms, ctx->ev[3], ctx->ev[4]);
    stats->ms_rescue = ms;
  }
  return ZEF_OK;
}
