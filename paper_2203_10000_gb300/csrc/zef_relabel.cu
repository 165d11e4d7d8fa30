// zef_relabel.cu -- recursive re-labeling at the tissue boundaries
// (Sec. 2.1.3 item 2, Fig. 3) as one CUDA graph.
//
// One pass (the body of a conditional while-node):
//   k_rb_mark     tets whose four node labels are not all equal (the tissue
//                 boundary): their nodes not yet evaluated in this call
//                 become candidates (flag 1)
//   scan          candidate flags -> positions, count K (= the label
//                 pipeline's point count)
//   k_rb_gather   candidate positions into a contiguous list; mark evaluated
//   label pipeline  the K candidates (zef_label.cu)
//   k_rb_apply    new labels back to the nodes; count the changed ones
//   k_rb_next     per-pass statistics; the loop continues while a pass
//                 changed a label and the pass limit is not reached
// The graph is instantiated once per (arrays, sizes, options) and cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "zef_internal.h"

#define CK(call, what)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

namespace zef {

namespace {

// relabel statistics words (device)
enum RbWord { RB_PASS = 0, RB_ABORT, RB_EVAL, RB_CHANGED, RB_PASS_CHANGED, RB_PER_PASS };

struct RB {
  const float *nodes;
  const int32_t *tets;
  int32_t *labels;
  int64_t n_nodes, n_tets;
  uint8_t *fresh;    // node evaluated during this call
  uint32_t *cand;    // candidate flags, scanned in place into positions
  float *pts;        // gathered candidate positions [n_nodes][3]
  int32_t *idx;      // gathered candidate node index
  int32_t *lab;      // labels of the gathered candidates
  int64_t *cnt;      // label pipeline counters (CNT_N, CNT_OFF, ...)
  int64_t *rs;       // RbWord words, then (evaluated, changed) per pass
  int32_t max_passes;
  uint32_t *status;
  cudaGraphConditionalHandle handle;
};

__global__ void k_rb_init(RB r) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < RB_PER_PASS + 2 * r.max_passes; ++k) r.rs[k] = 0;
    r.cnt[CNT_OFF] = 0;
    r.cnt[CNT_N] = 0;
  }
}

__global__ void __launch_bounds__(256) k_rb_mark(RB r) {
  if (r.rs[RB_ABORT]) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < r.n_tets;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = r.tets[4 * t + k];
      bad |= v[k] < 0 || v[k] >= r.n_nodes;
    }
    if (bad) {
      // a node index outside [0, n_nodes): stop the loop, report it
      atomicOr(r.status, ST_INVALID);
      atomicExch((unsigned long long *)(r.rs + RB_ABORT), 1ull);
      continue;
    }
    const int32_t l0 = r.labels[v[0]];
    if (l0 == r.labels[v[1]] && l0 == r.labels[v[2]] && l0 == r.labels[v[3]]) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (!r.fresh[v[k]]) r.cand[v[k]] = 1u;
  }
}

// after the scan: the pipeline's point count (0 once aborted)
__global__ void k_rb_count(RB r) {
  if (threadIdx.x != 0) return;
  if (r.rs[RB_ABORT]) r.cnt[CNT_N] = 0;
  r.rs[RB_PASS_CHANGED] = 0;
}

__global__ void __launch_bounds__(256) k_rb_gather(RB r) {
  const int64_t K = r.cnt[CNT_N];
  if (K == 0) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < r.n_nodes;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t pos = r.cand[v];
    const uint32_t next = (v + 1 < r.n_nodes) ? r.cand[v + 1] : (uint32_t)K;
    if (next == pos) continue;  // not a candidate
    r.pts[3 * (int64_t)pos + 0] = r.nodes[3 * v + 0];
    r.pts[3 * (int64_t)pos + 1] = r.nodes[3 * v + 1];
    r.pts[3 * (int64_t)pos + 2] = r.nodes[3 * v + 2];
    r.idx[pos] = (int32_t)v;
    r.fresh[v] = 1;
  }
}

__global__ void __launch_bounds__(256) k_rb_apply(RB r) {
  const int64_t K = r.cnt[CNT_N];
  unsigned long long changed = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = r.idx[j], l = r.lab[j];
    if (r.labels[v] != l) {
      r.labels[v] = l;
      ++changed;
    }
  }
  for (int o = 16; o > 0; o >>= 1) changed += __shfl_xor_sync(0xffffffffu, changed, o);
  if ((threadIdx.x & 31) == 0 && changed)
    atomicAdd((unsigned long long *)(r.rs + RB_PASS_CHANGED), changed);
}

__global__ void k_rb_next(RB r) {
  if (threadIdx.x != 0) return;
  const int64_t p = r.rs[RB_PASS];
  const int64_t K = r.cnt[CNT_N], changed = r.rs[RB_PASS_CHANGED];
  r.rs[RB_PER_PASS + 2 * p] = K;
  r.rs[RB_PER_PASS + 2 * p + 1] = changed;
  r.rs[RB_EVAL] += K;
  r.rs[RB_CHANGED] += changed;
  r.rs[RB_PASS] = p + 1;
  const bool more = !r.rs[RB_ABORT] && changed > 0 && p + 1 < r.max_passes;
  cudaGraphSetConditional(r.handle, more ? 1u : 0u);
}

bool on_device(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

zef_status rb_grow(zef_ctx *ctx, int idx, size_t bytes) {
  if (ctx->rb_buf[idx] && ctx->rb_cap[idx] >= bytes) return ZEF_OK;
  if (ctx->rb_buf[idx]) cudaFree(ctx->rb_buf[idx]);
  ctx->rb_buf[idx] = nullptr;
  ctx->rb_cap[idx] = 0;
  CK(cudaMalloc(&ctx->rb_buf[idx], std::max<size_t>(bytes, 256)), "cudaMalloc(relabel)");
  ctx->rb_cap[idx] = bytes;
  return ZEF_OK;
}

uint64_t mix(uint64_t h, uint64_t v) { return h ^ (v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2)); }

uint64_t bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, sizeof(u));
  return u;
}

}  // namespace

zef_status relabel_run(zef_ctx *ctx, const float *nodes_in, int64_t n, const int32_t *tets_in, int64_t m,
                       int32_t *labels_io, int32_t max_passes, const zef_label_opts &opts,
                       zef_relabel_pass *per_pass, int32_t *passes, int32_t *converged) {
  NvtxRange nvtx_("zef.relabel_boundary");
  if (n == 0) {
    if (converged) *converged = 1;
    return ZEF_OK;
  }
  const bool dn = on_device(nodes_in, ctx->device), dl = on_device(labels_io, ctx->device),
             dt = m == 0 ? dn : on_device(tets_in, ctx->device);
  if (!(dn == dl && dl == dt)) return fail(ctx, ZEF_ERR_INVALID_ARG, "nodes, tets and labels must all be host or all device");
  const bool host = !dn;
  zef_status st;
  // 0 fresh, 1 cand, 2 pts, 3 idx, 4 lab, 5 block sums, 6 stats, 7 staged nodes + labels, 8 staged tets
  const int64_t bs_len = n / 2048 + 2;
  if ((st = rb_grow(ctx, 0, (size_t)n))) return st;
  if ((st = rb_grow(ctx, 1, (size_t)n * sizeof(uint32_t)))) return st;
  if ((st = rb_grow(ctx, 2, (size_t)n * 3 * sizeof(float)))) return st;
  if ((st = rb_grow(ctx, 3, (size_t)n * sizeof(int32_t)))) return st;
  if ((st = rb_grow(ctx, 4, (size_t)n * sizeof(int32_t)))) return st;
  if ((st = rb_grow(ctx, 5, (size_t)bs_len * sizeof(uint32_t)))) return st;
  if ((st = rb_grow(ctx, 6, (size_t)(RB_PER_PASS + 2 * max_passes) * sizeof(int64_t)))) return st;
  const float *nodes = nodes_in;
  const int32_t *tets = tets_in;
  int32_t *labels = labels_io;
  if (host) {
    if ((st = rb_grow(ctx, 7, (size_t)n * 3 * sizeof(float) + (size_t)n * sizeof(int32_t)))) return st;
    if ((st = rb_grow(ctx, 8, (size_t)std::max<int64_t>(m, 1) * 4 * sizeof(int32_t)))) return st;
    float *dnodes = (float *)ctx->rb_buf[7];
    int32_t *dlab = (int32_t *)(dnodes + 3 * n);
    int32_t *dtets = (int32_t *)ctx->rb_buf[8];
    CK(cudaMemcpyAsync(dnodes, nodes_in, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
       "copy nodes");
    CK(cudaMemcpyAsync(dlab, labels_io, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream),
       "copy labels");
    if (m > 0)
      CK(cudaMemcpyAsync(dtets, tets_in, (size_t)m * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream),
         "copy tets");
    nodes = dnodes;
    labels = dlab;
    tets = dtets;
  }
  if ((st = label_reserve(ctx, n))) return st;
  LabelBuffers &b = ctx->lb;

  LaunchShape shape{256, 2, kernel_variant(opts.kernel)};
  if (opts.precision == ZEF_FP64_PLAIN) shape = LaunchShape{128, 2};
  else if (opts.block_threads) shape = LaunchShape{opts.block_threads, opts.points_per_thread, kernel_variant(opts.kernel)};

  RB r;
  r.nodes = nodes;
  r.tets = tets;
  r.labels = labels;
  r.n_nodes = n;
  r.n_tets = m;
  r.fresh = (uint8_t *)ctx->rb_buf[0];
  r.cand = (uint32_t *)ctx->rb_buf[1];
  r.pts = (float *)ctx->rb_buf[2];
  r.idx = (int32_t *)ctx->rb_buf[3];
  r.lab = (int32_t *)ctx->rb_buf[4];
  r.cnt = b.counters;
  r.rs = (int64_t *)ctx->rb_buf[6];
  r.max_passes = max_passes;
  r.status = ctx->d_status;
  r.handle = 0;
  uint32_t *bsums = (uint32_t *)ctx->rb_buf[5];

  uint64_t key = 0x7e1abe1ull;
  for (uint64_t v : {(uint64_t)(uintptr_t)nodes, (uint64_t)(uintptr_t)tets, (uint64_t)(uintptr_t)labels,
                     (uint64_t)n, (uint64_t)m, (uint64_t)max_passes, (uint64_t)(uintptr_t)r.fresh,
                     (uint64_t)(uintptr_t)r.cand, (uint64_t)(uintptr_t)r.pts, (uint64_t)(uintptr_t)r.idx,
                     (uint64_t)(uintptr_t)r.lab, (uint64_t)(uintptr_t)r.rs, (uint64_t)(uintptr_t)bsums,
                     (uint64_t)(uintptr_t)b.spts, (uint64_t)(uintptr_t)b.flags, (uint64_t)(uintptr_t)b.hist,
                     (uint64_t)(uintptr_t)b.counters, (uint64_t)b.cap_points, (uint64_t)shape.threads,
                     (uint64_t)shape.ppt, (uint64_t)shape.variant, (uint64_t)opts.precision, bits(opts.margin),
                     bits(opts.winding_tol), (uint64_t)opts.flags, (uint64_t)(uintptr_t)ctx->d_entries, ctx->gen})
    key = mix(key, v);
  if (!ctx->rb_exec || ctx->rb_key != key) {
    if (ctx->rb_exec) {
      cudaGraphExecDestroy(ctx->rb_exec);
      ctx->rb_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle handle;
    cudaError_t ce = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(ctx, ce, "conditional graph node");
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    r.handle = handle;
    // capture one pass into the body on a private stream
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate(capture)");
    cudaStream_t user = ctx->stream;
    ctx->stream = cap;
    st = ZEF_OK;
    ce = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const int g_t = grid_blocks(ctx, std::max<int64_t>(m, 1), 256);
      const int g_n = grid_blocks(ctx, n, 256);
      cudaMemsetAsync(r.cand, 0, (size_t)n * sizeof(uint32_t), cap);
      k_rb_mark<<<g_t, 256, 0, cap>>>(r);
      st = scan_exclusive(ctx, r.cand, nullptr, 1, n, b.counters + CNT_N, bsums);
      if (st == ZEF_OK) {
        k_rb_count<<<1, 32, 0, cap>>>(r);
        k_rb_gather<<<g_n, 256, 0, cap>>>(r);
        LabelPlan p;
        p.pts = r.pts;
        p.labels = r.lab;
        p.omega = nullptr;
        p.omega_ld = 0;
        p.n_cap = n;
        p.d_n = b.counters + CNT_N;
        p.d_off = b.counters + CNT_OFF;
        p.opts = opts;
        p.shape = shape;
        p.timed = false;
        st = label_enqueue(ctx, p);
      }
      if (st == ZEF_OK) {
        k_rb_apply<<<g_n, 256, 0, cap>>>(r);
        k_rb_next<<<1, 32, 0, cap>>>(r);
      }
      cudaGraph_t out = body;
      cudaError_t ee = cudaStreamEndCapture(cap, &out);
      if (st == ZEF_OK && ee != cudaSuccess) st = cuda_fail(ctx, ee, "cudaStreamEndCapture");
    } else {
      st = cuda_fail(ctx, ce, "cudaStreamBeginCaptureToGraph");
    }
    ctx->stream = user;
    cudaStreamDestroy(cap);
    if (st == ZEF_OK) {
      cudaError_t ie = cudaGraphInstantiate(&ctx->rb_exec, graph, 0);
      if (ie != cudaSuccess) st = cuda_fail(ctx, ie, "cudaGraphInstantiate(relabel)");
      else ctx->rb_key = key;
    }
    cudaGraphDestroy(graph);
    if (st) return st;
  }
  CK(cudaMemsetAsync(r.fresh, 0, (size_t)n, ctx->stream), "clear evaluated flags");
  k_rb_init<<<1, 32, 0, ctx->stream>>>(r);
  CK(cudaGetLastError(), "k_rb_init");
  CK(cudaGraphLaunch(ctx->rb_exec, ctx->stream), "cudaGraphLaunch(relabel)");
  std::vector<int64_t> rs((size_t)(RB_PER_PASS + 2 * max_passes), 0);
  CK(cudaMemcpyAsync(rs.data(), r.rs, rs.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
     "read relabel stats");
  if (host)
    CK(cudaMemcpyAsync(labels_io, labels, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
       "copy labels back");
  st = zef_synchronize(ctx);
  const int64_t np = std::min<int64_t>(rs[RB_PASS], max_passes);
  if (passes) *passes = (int32_t)np;
  if (converged) *converged = (!rs[RB_ABORT] && np > 0 && rs[RB_PER_PASS + 2 * (np - 1) + 1] == 0) ? 1 : 0;
  if (per_pass)
    for (int64_t p = 0; p < np; ++p) {
      per_pass[p].evaluated = rs[RB_PER_PASS + 2 * p];
      per_pass[p].changed = rs[RB_PER_PASS + 2 * p + 1];
    }
  return st;
}

}  // namespace zef
