// Host side of libzef: context, surface registration (Sec. 2.1.3: closed
// segmentation boundaries), priority (Sec. 2.1), argument checking and the C
// entry points.  All arithmetic of the labeling path runs in the kernels of
// zef_label.cu / zef_refine.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <numeric>
#include <unordered_map>

#include "zef_debug.h"
#include "zef_internal.h"

using namespace zef;

namespace zef {

zef_status fail(zef_ctx *ctx, zef_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return st;
}

// kDop directions of a Fibonacci sphere: z_k = 1 - (2k + 1) / K, azimuth k
// times the golden angle; rounded to float (the device tests use the same
// float values).
void dop_directions(float (*dirs)[3]) {
  const double golden = 3.14159265358979323846 * (3.0 - std::sqrt(5.0));
  for (int k = 0; k < kDop; ++k) {
    const double z = 1.0 - (2.0 * k + 1.0) / kDop;
    const double r = std::sqrt(std::max(0.0, 1.0 - z * z));
    dirs[k][0] = (float)(r * std::cos(golden * k));
    dirs[k][1] = (float)(r * std::sin(golden * k));
    dirs[k][2] = (float)z;
  }
}

zef_status cuda_fail(zef_ctx *ctx, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  zef_status st = (e == cudaErrorMemoryAllocation) ? ZEF_ERR_OOM : ZEF_ERR_CUDA;
  return fail(ctx, st, m);
}

}  // namespace zef

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

namespace {

const char *kNullCtxMsg = "zef: null context";

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev < 0) return;  // host-only context
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Is p device memory (device or managed) of `device`?  Host otherwise.
bool is_device_ptr(const void *p, int device) {
  if (device < 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  if (a.type == cudaMemoryTypeManaged) return true;
  return false;
}

// ---------------------------------------------------------------- strips
// Greedy triangle strips over a closed oriented manifold mesh.  A strip is a
// vertex sequence s0, s1, s2, ... whose consecutive triples are triangles;
// every triangle appears in exactly one strip.
struct Stripper {
  const int32_t *tris;
  int64_t nt;
  std::vector<int64_t> nbr;  // [t*3 + e] triangle across edge e = (v_e, v_{e+1})

  // neighbour of triangle t across the undirected edge {a, b}; -1 if none
  int64_t across(int64_t t, int32_t a, int32_t b) const {
    const int32_t *f = tris + 3 * t;
    for (int e = 0; e < 3; ++e) {
      int32_t x = f[e], y = f[(e + 1) % 3];
      if ((x == a && y == b) || (x == b && y == a)) return nbr[3 * t + e];
    }
    return -1;
  }
  static int32_t third(const int32_t *f, int32_t a, int32_t b) {
    for (int e = 0; e < 3; ++e)
      if (f[e] != a && f[e] != b) return f[e];
    return -1;
  }
  // length (triangles) of the strip starting at t with first vertex f[r]
  template <bool Commit>
  int64_t walk(int64_t t, int r, std::vector<uint8_t> &used, std::vector<int32_t> *seq,
               std::vector<int64_t> *tri_seq) {
    const int32_t *f = tris + 3 * t;
    int32_t s0 = f[r], s1 = f[(r + 1) % 3], s2 = f[(r + 2) % 3];
    std::vector<int64_t> touched;
    int64_t len = 1;
    if (Commit) {
      seq->push_back(s0);
      seq->push_back(s1);
      seq->push_back(s2);
      tri_seq->push_back(t);
      used[t] = 1;
    } else {
      used[t] = 2;
      touched.push_back(t);
    }
    int64_t cur = t;
    int32_t a = s1, b = s2;
    for (;;) {
      int64_t nx = across(cur, a, b);
      if (nx < 0 || used[nx]) break;
      int32_t c = third(tris + 3 * nx, a, b);
      if (Commit) {
        seq->push_back(c);
        tri_seq->push_back(nx);
        used[nx] = 1;
      } else {
        used[nx] = 2;
        touched.push_back(nx);
      }
      ++len;
      cur = nx;
      a = b;
      b = c;
    }
    if (!Commit)
      for (int64_t q : touched) used[q] = 0;
    return len;
  }
};

}  // namespace

// ---------------------------------------------------------------- entry points
extern "C" {

int32_t zef_version(void) { return ZEF_VERSION_MAJOR * 1000 + ZEF_VERSION_MINOR; }

const char *zef_last_error(const zef_ctx *ctx) {
  if (!ctx) return kNullCtxMsg;
  return ctx->err.c_str();
}

zef_status zef_create(zef_ctx **out, int device, void *cuda_stream) {
  if (!out) return ZEF_ERR_INVALID_ARG;
  *out = nullptr;
  if (device == ZEF_HOST_ONLY) {
    zef_ctx *h = new (std::nothrow) zef_ctx();
    if (!h) return ZEF_ERR_OOM;
    h->device = ZEF_HOST_ONLY;
    *out = h;
    return ZEF_OK;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ZEF_ERR_INVALID_ARG;
  }
  zef_ctx *ctx = new (std::nothrow) zef_ctx();
  if (!ctx) return ZEF_ERR_OOM;
  ctx->device = device;
  DeviceGuard g(device);
  zef_status st = ZEF_OK;
  do {
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaDeviceGetAttribute"); break; }
    if (cuda_stream) {
      ctx->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaStreamCreate"); break; }
      ctx->own_stream = true;
    }
    e = cudaMalloc(&ctx->d_status, 4 * sizeof(uint32_t));
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaMalloc(status)"); break; }
    e = cudaMemset(ctx->d_status, 0, 4 * sizeof(uint32_t));
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaMemset(status)"); break; }
    e = cudaMallocHost(&ctx->h_counters, CNT_COUNT_ * sizeof(int64_t));
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaMallocHost"); break; }
    if ((st = upload_dop_directions(ctx)) != ZEF_OK) break;
    for (auto &ev : ctx->ev) {
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaEventCreate"); break; }
    }
  } while (0);
  if (st != ZEF_OK) {
    zef_destroy(ctx);
    return st;
  }
  *out = ctx;
  return ZEF_OK;
}

void zef_destroy(zef_ctx *ctx) {
  if (!ctx) return;
  if (ctx->device == ZEF_HOST_ONLY) {
    delete ctx;
    return;
  }
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->s_in) cudaStreamSynchronize(ctx->s_in);
  if (ctx->s_out) cudaStreamSynchronize(ctx->s_out);
  auto fr = [](void *p) {
    if (p) cudaFree(p);
  };
  for (auto &sl : ctx->pipe) {
    fr(sl.pts);
    fr(sl.labels);
    for (cudaEvent_t e : {sl.h2d, sl.done, sl.d2h})
      if (e) cudaEventDestroy(e);
  }
  if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
  if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
  fr(ctx->d_entries);
  fr(ctx->d_tris);
  fr(ctx->d_nodes);
  fr(ctx->d_cseg);
  fr(ctx->d_ctidx);
  fr(ctx->d_comps);
  fr(ctx->d_row_ids);
  fr(ctx->d_lpt);
  fr(ctx->d_dop);
  fr(ctx->d_status);
  LabelBuffers &b = ctx->lb;
  fr(b.spts); fr(b.perm); fr(b.keys); fr(b.in_mask); fr(b.unc_mask); fr(b.tile_box);
  fr(b.hist); fr(b.flags); fr(b.block_sums); fr(b.items); fr(b.unc_list); fr(b.counters);
  fr(b.labels_tmp); fr(b.pts_tmp); fr(b.omega_tmp); fr(b.tune_pts);
  fr(ctx->el_node_labels); fr(ctx->el_masks); fr(ctx->el_tets); fr(ctx->el_labels);
  for (auto &p : ctx->rf_buf) fr(p);
  for (auto &p : ctx->rb_buf) fr(p);
  for (auto &p : ctx->pp_buf) fr(p);
  if (ctx->rb_exec) cudaGraphExecDestroy(ctx->rb_exec);
  if (ctx->rf_exec) cudaGraphExecDestroy(ctx->rf_exec);
  if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
  for (auto &ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaGetLastError();
  delete ctx;
}

zef_status zef_compartment_info(const zef_ctx *ctx, int32_t *num_compartments, int64_t *total) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  if (num_compartments) *num_compartments = (int32_t)ctx->comps.size();
  if (total) {
    int64_t s = 0;
    for (auto &c : ctx->comps) s += c.nt;
    *total = s;
  }
  return ZEF_OK;
}

zef_status zef_add_compartment(zef_ctx *ctx, int32_t id, const float *verts, int64_t nv,
                               const int32_t *tris, int64_t nt, uint32_t flags) {
  NvtxRange nvtx_("zef.add_compartment");
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (id <= 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "compartment id must be > 0");
  for (auto &c : ctx->comps)
    if (c.id == id) return fail(ctx, ZEF_ERR_INVALID_ARG, "duplicate compartment id");
  if ((int)ctx->comps.size() >= ZEF_MAX_COMPARTMENTS)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "too many compartments (max 64)");
  if (!verts || !tris || nv < 4 || nt < 4)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "a closed surface needs >= 4 vertices and >= 4 triangles");
  if (nt > (int64_t)1 << 28 || nv > (int64_t)1 << 30)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "surface too large");
  if (flags & ~ZEF_AUTO_ORIENT) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown flags");
  DeviceGuard g(ctx->device);

  std::vector<float> V(3 * nv);
  std::vector<int32_t> T(3 * nt);
  if (is_device_ptr(verts, ctx->device)) {
    CK(cudaMemcpy(V.data(), verts, V.size() * sizeof(float), cudaMemcpyDeviceToHost), "copy verts");
  } else {
    std::memcpy(V.data(), verts, V.size() * sizeof(float));
  }
  if (is_device_ptr(tris, ctx->device)) {
    CK(cudaMemcpy(T.data(), tris, T.size() * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy tris");
  } else {
    std::memcpy(T.data(), tris, T.size() * sizeof(int32_t));
  }
  for (float x : V)
    if (!std::isfinite(x)) return fail(ctx, ZEF_ERR_INVALID_ARG, "non-finite vertex coordinate");
  for (int64_t t = 0; t < nt; ++t) {
    int32_t a = T[3 * t], b = T[3 * t + 1], c = T[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv)
      return fail(ctx, ZEF_ERR_INVALID_ARG, "triangle index out of range");
    if (a == b || b == c || a == c)
      return fail(ctx, ZEF_ERR_SURFACE_NOT_CLOSED, "degenerate triangle (repeated vertex)");
  }

  // closedness: every directed edge once, and its reverse present
  std::vector<uint64_t> de(3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int e = 0; e < 3; ++e)
      de[3 * t + e] = ((uint64_t)(uint32_t)T[3 * t + e] << 32) | (uint32_t)T[3 * t + (e + 1) % 3];
  std::vector<int64_t> order(3 * nt);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return de[x] < de[y]; });
  for (size_t i = 1; i < order.size(); ++i)
    if (de[order[i]] == de[order[i - 1]])
      return fail(ctx, ZEF_ERR_SURFACE_NOT_CLOSED,
                  "surface not closed/oriented: a directed edge is used twice");
  auto find_edge = [&](uint64_t key) -> int64_t {
    size_t lo = 0, hi = order.size();
    while (lo < hi) {
      size_t mid = (lo + hi) / 2;
      if (de[order[mid]] < key) lo = mid + 1; else hi = mid;
    }
    if (lo < order.size() && de[order[lo]] == key) return order[lo];
    return -1;
  };
  Stripper sp;
  sp.nbr.assign(3 * nt, -1);
  for (int64_t i = 0; i < 3 * nt; ++i) {
    uint64_t k = de[i];
    uint64_t rk = (k << 32) | (k >> 32);
    int64_t j = find_edge(rk);
    if (j < 0)
      return fail(ctx, ZEF_ERR_SURFACE_NOT_CLOSED,
                  "surface not closed: an edge has no opposite half-edge");
    sp.nbr[i] = j / 3;
  }

  // orientation: signed volume in double
  double vol = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    const float *a = &V[3 * T[3 * t]], *b = &V[3 * T[3 * t + 1]], *c = &V[3 * T[3 * t + 2]];
    double cx = (double)b[1] * c[2] - (double)b[2] * c[1];
    double cy = (double)b[2] * c[0] - (double)b[0] * c[2];
    double cz = (double)b[0] * c[1] - (double)b[1] * c[0];
    vol += (double)a[0] * cx + (double)a[1] * cy + (double)a[2] * cz;
  }
  if (!(vol > 0.0)) {
    if (!(flags & ZEF_AUTO_ORIENT) || vol == 0.0)
      return fail(ctx, ZEF_ERR_SURFACE_ORIENTATION,
                  "surface has non-positive signed volume (inward orientation)");
    for (int64_t t = 0; t < nt; ++t) std::swap(T[3 * t + 1], T[3 * t + 2]);
    // neighbour table follows the flipped edges: edge e=(v0,v1)->(v0,v2) etc.
    for (int64_t t = 0; t < nt; ++t) {
      int64_t n0 = sp.nbr[3 * t], n1 = sp.nbr[3 * t + 1], n2 = sp.nbr[3 * t + 2];
      sp.nbr[3 * t] = n2;      // (v0, v2)
      sp.nbr[3 * t + 1] = n1;  // (v2, v1)
      sp.nbr[3 * t + 2] = n0;  // (v1, v0)
    }
  }

  CompHost ch;
  ch.id = id;
  ch.nv = nv;
  ch.nt = nt;
  for (int k = 0; k < 3; ++k) {
    ch.lo[k] = std::numeric_limits<float>::infinity();
    ch.hi[k] = -std::numeric_limits<float>::infinity();
  }
  std::vector<uint8_t> referenced(nv, 0);
  for (int64_t i = 0; i < 3 * nt; ++i) referenced[T[i]] = 1;
  float dirs[kDop][3];
  dop_directions(dirs);
  for (int k = 0; k < kDop; ++k) ch.dop[k] = -std::numeric_limits<double>::infinity();
  for (int64_t v = 0; v < nv; ++v) {
    if (!referenced[v]) continue;
    const float *p = &V[3 * v];
    for (int k = 0; k < 3; ++k) {
      ch.lo[k] = std::min(ch.lo[k], p[k]);
      ch.hi[k] = std::max(ch.hi[k], p[k]);
    }
    for (int k = 0; k < kDop; ++k) {
      const double t = (double)dirs[k][0] * p[0] + (double)dirs[k][1] * p[1] + (double)dirs[k][2] * p[2];
      ch.dop[k] = std::max(ch.dop[k], t);
    }
  }

  // strips
  sp.tris = T.data();
  sp.nt = nt;
  std::vector<uint8_t> used(nt, 0);
  std::vector<Entry> ent;
  ent.reserve(nt + nt / 4 + 32);
  int64_t nstrips = 0;
  auto vtx = [&](int32_t v) { return &V[3 * (int64_t)v]; };
  // A non-triangle entry (weight 0) has n = 0, hence N = 0 exactly, and its
  // window always repeats a vertex, so D = 2 r_u (r_u r_w + R_u . R_w) >= 0:
  // the factor (D, N) is a positive real and adds no angle.  kappa = 0 makes
  // the conditioning test catch an FP32 D <= 0 there.
  auto push_prime = [&](const float *p) {
    Entry e;
    e.v = make_float4(p[0], p[1], p[2], 0.f);
    e.n = make_float4(0.f, 0.f, 0.f, 0.f);
    ent.push_back(e);
  };
  for (int64_t t = 0; t < nt; ++t) {
    if (used[t]) continue;
    int best_r = 0;
    int64_t best_len = -1;
    for (int r = 0; r < 3; ++r) {
      int64_t len = sp.walk<false>(t, r, used, nullptr, nullptr);
      if (len > best_len) { best_len = len; best_r = r; }
    }
    std::vector<int32_t> seq;
    std::vector<int64_t> tseq;
    sp.walk<true>(t, best_r, used, &seq, &tseq);
    ++nstrips;
    // priming: the first strip starts from the window (s0, s0); a later strip
    // follows the window (y, z) of the previous one with z, x0, x0, x1, so
    // the windows are (y,z,z), (z,z,x0), (z,x0,x0), (x0,x0,x1)
    if (!ent.empty()) {
      const float4 z = ent.back().v;
      const float zp[3] = {z.x, z.y, z.z};
      push_prime(zp);
      push_prime(vtx(seq[0]));
    }
    push_prime(vtx(seq[0]));
    push_prime(vtx(seq[1]));
    for (size_t k = 2; k < seq.size(); ++k) {
      Entry e;
      const float *p = vtx(seq[k]);
      e.v = make_float4(p[0], p[1], p[2], 0.f);
      {
        const int32_t *f = &T[3 * tseq[k - 2]];
        const float *a = vtx(f[0]), *b = vtx(f[1]), *c = vtx(f[2]);
        double e1[3], e2[3];
        for (int q = 0; q < 3; ++q) {
          e1[q] = (double)b[q] - a[q];
          e2[q] = (double)c[q] - a[q];
        }
        double nx = e1[1] * e2[2] - e1[2] * e2[1];
        double ny = e1[2] * e2[0] - e1[0] * e2[2];
        double nz = e1[0] * e2[1] - e1[1] * e2[0];
        double nn = std::sqrt(nx * nx + ny * ny + nz * nz);
        // +1 when the window order (seq[k-2], seq[k-1], seq[k]) keeps the
        // triangle's orientation, -1 when it reverses it (strips alternate)
        const int32_t wa = seq[k - 2], wb = seq[k - 1];
        int ia = 0;
        while (f[ia] != wa) ++ia;
        e.v.w = (f[(ia + 1) % 3] == wb) ? 1.f : -1.f;
        e.n = make_float4((float)nx, (float)ny, (float)nz, (float)(kKappa * nn));
      }
      ent.push_back(e);
    }
  }
  while (ent.size() % kGroup) {
    const float4 z = ent.back().v;
    const float zp[3] = {z.x, z.y, z.z};
    push_prime(zp);
  }
  ch.nstrips = nstrips;
  ch.entry_off = (int64_t)ctx->h_entries.size();
  ch.entry_cnt = (int64_t)ent.size();
  ch.tri_off = (int64_t)(ctx->h_tris.size() / 3);
  if (ch.entry_off + ch.entry_cnt > INT32_MAX || ch.tri_off + nt > INT32_MAX)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "total surface size exceeds the library limit");
  // cap tree (exact far-field replacement of patches, zef_tree.cpp)
  {
    const int64_t node_base = (int64_t)ctx->h_nodes.size(), seg_base = (int64_t)ctx->h_cseg.size();
    int64_t leaf = 0;
    build_cap_tree(V.data(), T.data(), nt, node_base, seg_base, (int64_t)ctx->h_ctidx.size(), ctx->h_nodes,
                   ctx->h_cseg, ctx->h_ctidx, &ch.cap_root, &leaf);
    ch.cseg_off = seg_base;
    ch.cseg_leaf = leaf;
    if ((int64_t)ctx->h_nodes.size() > INT32_MAX || (int64_t)ctx->h_cseg.size() > INT32_MAX)
      return fail(ctx, ZEF_ERR_INVALID_ARG, "total surface size exceeds the library limit");
  }
  ctx->h_entries.insert(ctx->h_entries.end(), ent.begin(), ent.end());
  for (int64_t t = 0; t < nt; ++t)
    for (int q = 0; q < 3; ++q) {
      const float *p = vtx(T[3 * t + q]);
      ctx->h_tris.push_back(make_float4(p[0], p[1], p[2], 0.f));
    }
  ctx->comps.push_back(ch);
  ctx->priority.push_back(id);
  ctx->dirty = true;
  ctx->tune_cache.clear();
  return ensure_uploaded(ctx);
}

zef_status zef_compartment_priority(zef_ctx *ctx, const int32_t *ids, int32_t n) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ids || n != (int32_t)ctx->comps.size())
    return fail(ctx, ZEF_ERR_INVALID_ARG, "priority must list every registered compartment once");
  std::vector<int32_t> a(ids, ids + n), b;
  for (auto &c : ctx->comps) b.push_back(c.id);
  std::vector<int32_t> sa = a, sb = b;
  std::sort(sa.begin(), sa.end());
  std::sort(sb.begin(), sb.end());
  if (sa != sb || std::adjacent_find(sa.begin(), sa.end()) != sa.end())
    return fail(ctx, ZEF_ERR_INVALID_ARG, "priority is not a permutation of the registered ids");
  ctx->priority = a;
  ctx->dirty = true;
  DeviceGuard g(ctx->device);
  return ensure_uploaded(ctx);
}

zef_status zef_synchronize(zef_ctx *ctx) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  if (ctx->device == ZEF_HOST_ONLY) return ZEF_OK;
  DeviceGuard g(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (ctx->s_in) {
    CK(cudaStreamSynchronize(ctx->s_in), "cudaStreamSynchronize(copy-in)");
    CK(cudaStreamSynchronize(ctx->s_out), "cudaStreamSynchronize(copy-out)");
  }
  uint32_t st[2] = {0, 0};
  CK(cudaMemcpy(st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost), "read status");
  if (st[0]) {
    CK(cudaMemset(ctx->d_status, 0, 2 * sizeof(uint32_t)), "clear status");
    if (st[0] & ST_TIMEOUT)
      return fail(ctx, ZEF_ERR_TIMEOUT, "a bounded device wait expired (site " + std::to_string(st[1]) + ")");
    if (st[0] & ST_INVALID)
      return fail(ctx, ZEF_ERR_INVALID_ARG, "a tet references a node index outside [0, num_nodes)");
    if (st[0] & ST_CAPACITY)
      return fail(ctx, ZEF_ERR_CAPACITY, "refinement exceeded the mesh capacities");
    if (st[0] & ST_BOUNDS)
      return fail(ctx, ZEF_ERR_BOUNDS, "a device-side index check failed (site " + std::to_string(st[1]) + ")");
  }
  return ZEF_OK;
}

zef_status zef_label_points(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels, float *omega,
                            const zef_label_opts *opts, zef_label_stats *stats) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  return zef::label_points_impl(ctx, pts, n, labels, omega, opts, stats, nullptr, false);
}

zef_status zef_label_points_async(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                                  const zef_label_opts *opts) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  return zef::label_points_async_impl(ctx, pts, n, labels, opts);
}

zef_status zef_label_elements(zef_ctx *ctx, const float *nodes, int64_t n_nodes, const int32_t *tets,
                              int64_t n_tets, int32_t *elem_labels, int32_t *node_labels,
                              const zef_label_opts *opts, zef_label_stats *stats) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (n_tets < 0 || n_nodes < 0 || (n_tets > 0 && (!tets || !elem_labels)))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad tets/elem_labels arguments");
  if (n_tets > ((int64_t)1 << 31) - 1) return fail(ctx, ZEF_ERR_INVALID_ARG, "too many tets (max 2^31-1)");
  if (n_tets > 0 && n_nodes == 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "tets without nodes");
  if (ctx->comps.empty()) return fail(ctx, ZEF_ERR_NOT_READY, "no compartment registered");
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context cannot label");
  if (n_nodes > 0 && !nodes) return fail(ctx, ZEF_ERR_INVALID_ARG, "bad nodes argument");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_nodes == 0) return ZEF_OK;
  DeviceGuard g(ctx->device);
  const bool dnl = node_labels && is_device_ptr(node_labels, ctx->device);
  const bool dtet = n_tets == 0 || is_device_ptr(tets, ctx->device);
  const bool delem = n_tets == 0 || is_device_ptr(elem_labels, ctx->device);
  zef_status st = ensure_buffer(ctx, &ctx->el_masks, &ctx->el_cap_masks, n_nodes);
  if (st) return st;
  int32_t *d_nl = node_labels;
  if (!dnl) {
    st = ensure_buffer(ctx, &ctx->el_node_labels, &ctx->el_cap_nodes, n_nodes);
    if (st) return st;
    d_nl = ctx->el_node_labels;
  }
  const int32_t *d_tets = tets;
  if (!dtet) {
    st = ensure_buffer(ctx, &ctx->el_tets, &ctx->el_cap_tets, 4 * n_tets);
    if (st) return st;
    d_tets = ctx->el_tets;
  }
  int32_t *d_elem = elem_labels;
  if (!delem) {
    st = ensure_buffer(ctx, &ctx->el_labels, &ctx->el_cap_labels, n_tets);
    if (st) return st;
    d_elem = ctx->el_labels;
  }
  // node labels and inside bits of every (node, compartment) pair
  st = zef::label_points_impl(ctx, nodes, n_nodes, d_nl, nullptr, opts, stats, ctx->el_masks, true);
  if (st) return st;
  if (!dtet)
    CK(cudaMemcpyAsync(ctx->el_tets, tets, (size_t)n_tets * 4 * sizeof(int32_t), cudaMemcpyHostToDevice,
                       ctx->stream), "copy tets");
  st = launch_elem_labels(ctx, d_tets, n_tets, n_nodes, d_nl, ctx->el_masks, d_elem);
  if (st) return st;
  if (!delem)
    CK(cudaMemcpyAsync(elem_labels, d_elem, (size_t)n_tets * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->stream), "copy element labels");
  if (node_labels && !dnl)
    CK(cudaMemcpyAsync(node_labels, d_nl, (size_t)n_nodes * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->stream), "copy node labels");
  if (stats || !dtet || !delem || (node_labels && !dnl) || !is_device_ptr(nodes, ctx->device))
    return zef_synchronize(ctx);
  return ZEF_OK;
}

}  // extern "C"

namespace zef {

// zef_label_points; with d_masks (device, nullable) the inside bits of every
// point are written in the caller's order, and full_masks turns the priority
// early exit off so that every bit is decided.
// Checks shared by the labeling entry points; *o gets the options with
// their defaults filled in.
static zef_status check_label_call(zef_ctx *ctx, const float *pts, int64_t n, const int32_t *labels,
                                   const zef_label_opts *opts, zef_label_opts *o) {
  if (ctx->comps.empty()) return fail(ctx, ZEF_ERR_NOT_READY, "no compartment registered");
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context cannot label");
  if (n < 0 || (n > 0 && (!pts || !labels)))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad points/labels arguments");
  if (n > ((int64_t)1 << 31) - 1) return fail(ctx, ZEF_ERR_INVALID_ARG, "too many points (max 2^31-1)");
  if (opts) *o = *opts; else std::memset(o, 0, sizeof(*o));
  fill_default_opts(o);
  if (o->precision < 0 || o->precision > 2 || o->kernel < 0 || o->kernel > 2)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad precision or kernel");
  if (o->flags & ~kLabelFlagsAll) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown label flags");
  if ((o->block_threads || o->points_per_thread) && !shape_valid(o->block_threads, o->points_per_thread))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad launch shape (threads 128/256, points 2/4)");
  return ZEF_OK;
}

// Enqueue one labeling of the device points d_pts[n] on the context stream
// (labels into d_lab, solid angles into d_om when non-null); *shape gets the
// launch shape, *launches the library kernels enqueued.  Autotuning (first
// call of a new shape key) synchronizes; nothing else does.
static zef_status enqueue_labeling(zef_ctx *ctx, const float *d_pts, int64_t n, int32_t *d_lab, float *d_om,
                                   const zef_label_opts &o, unsigned long long *d_masks, bool full_masks,
                                   bool timed, LaunchShape *shape, int64_t *launches) {
  LabelPlan plan;
  plan.pts = d_pts;
  plan.labels = d_lab;
  plan.omega = d_om;
  plan.omega_ld = n;
  plan.n_cap = n;
  plan.d_n = ctx->lb.counters + CNT_N;
  plan.d_off = ctx->lb.counters + CNT_OFF;
  plan.opts = o;
  plan.masks = d_masks;
  plan.full_masks = full_masks;
  bool need_tune = false;
  plan.shape = choose_shape(ctx, o, n, &need_tune);
  plan.timed = timed;
  zef_status st;
  if (need_tune && (st = autotune(ctx, plan, &plan.shape))) return st;
  const int64_t launches0 = ctx->launches;
  if ((st = label_set_count(ctx, n, 0))) return st;
  if ((st = label_enqueue(ctx, plan))) return st;
  *shape = plan.shape;
  *launches = ctx->launches - launches0;
  return ZEF_OK;
}

// Pipelined labeling (zef_label_points_async): slot k = call parity.  The
// copy-in stream waits until the labeling that last read slot k finished,
// copies the points and records h2d; the context stream waits for h2d (and
// for the copy-out of the slot's previous labels), labels and records done;
// the copy-out stream waits for done, copies the labels and records d2h.
zef_status label_points_async_impl(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels,
                                   const zef_label_opts *opts) {
  NvtxRange nvtx_("zef.label_points_async");
  zef_label_opts o;
  zef_status st = check_label_call(ctx, pts, n, labels, opts, &o);
  if (st) return st;
  if (n == 0) return ZEF_OK;
  DeviceGuard g(ctx->device);
  if ((st = ensure_uploaded(ctx))) return st;
  if ((st = label_reserve(ctx, n))) return st;
  const bool dpts = is_device_ptr(pts, ctx->device), dlab = is_device_ptr(labels, ctx->device);
  LaunchShape shape;
  int64_t launches = 0;
  if (dpts && dlab) return enqueue_labeling(ctx, pts, n, labels, nullptr, o, nullptr, false, false, &shape, &launches);
  if (!ctx->s_in) {
    CK(cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking), "cudaStreamCreate(copy-in)");
    CK(cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking), "cudaStreamCreate(copy-out)");
    for (auto &sl : ctx->pipe) {
      CK(cudaEventCreateWithFlags(&sl.h2d, cudaEventDisableTiming), "cudaEventCreate");
      CK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "cudaEventCreate");
      CK(cudaEventCreateWithFlags(&sl.d2h, cudaEventDisableTiming), "cudaEventCreate");
    }
  }
  zef_ctx::PipeSlot &sl = ctx->pipe[ctx->pipe_next];
  ctx->pipe_next ^= 1;
  if (sl.cap < n) {
    // the slot's previous copies and labeling must be over before it is freed
    CK(cudaEventSynchronize(sl.done), "wait for the slot");
    CK(cudaEventSynchronize(sl.d2h), "wait for the slot");
    if (sl.pts) cudaFree(sl.pts);
    if (sl.labels) cudaFree(sl.labels);
    sl.pts = nullptr;
    sl.labels = nullptr;
    sl.cap = 0;
    CK(cudaMalloc(&sl.pts, (size_t)n * 3 * sizeof(float)), "cudaMalloc(staging points)");
    CK(cudaMalloc(&sl.labels, (size_t)n * sizeof(int32_t)), "cudaMalloc(staging labels)");
    sl.cap = n;
  }
  const float *d_pts = pts;
  if (!dpts) {
    CK(cudaStreamWaitEvent(ctx->s_in, sl.done, 0), "cudaStreamWaitEvent");
    CK(cudaMemcpyAsync(sl.pts, pts, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->s_in),
       "copy points");
    CK(cudaEventRecord(sl.h2d, ctx->s_in), "cudaEventRecord");
    CK(cudaStreamWaitEvent(ctx->stream, sl.h2d, 0), "cudaStreamWaitEvent");
    d_pts = sl.pts;
  }
  int32_t *d_lab = labels;
  if (!dlab) {
    CK(cudaStreamWaitEvent(ctx->stream, sl.d2h, 0), "cudaStreamWaitEvent");
    d_lab = sl.labels;
  }
  if ((st = enqueue_labeling(ctx, d_pts, n, d_lab, nullptr, o, nullptr, false, false, &shape, &launches))) return st;
  CK(cudaEventRecord(sl.done, ctx->stream), "cudaEventRecord");
  if (!dlab) {
    CK(cudaStreamWaitEvent(ctx->s_out, sl.done, 0), "cudaStreamWaitEvent");
    CK(cudaMemcpyAsync(labels, sl.labels, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->s_out),
       "copy labels");
    CK(cudaEventRecord(sl.d2h, ctx->s_out), "cudaEventRecord");
  }
  return ZEF_OK;
}

zef_status label_points_impl(zef_ctx *ctx, const float *pts, int64_t n, int32_t *labels, float *omega,
                             const zef_label_opts *opts, zef_label_stats *stats, unsigned long long *d_masks,
                             bool full_masks) {
  NvtxRange nvtx_("zef.label_points");
  zef_label_opts o;
  zef_status st = check_label_call(ctx, pts, n, labels, opts, &o);
  if (st) return st;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n == 0) return ZEF_OK;
  DeviceGuard g(ctx->device);
  st = ensure_uploaded(ctx);
  if (st) return st;
  st = label_reserve(ctx, n);
  if (st) return st;
  const int C = (int)ctx->comps.size();
  bool dpts = is_device_ptr(pts, ctx->device);
  bool dlab = is_device_ptr(labels, ctx->device);
  bool dom = omega ? is_device_ptr(omega, ctx->device) : true;
  LabelBuffers &b = ctx->lb;
  const float *d_pts = pts;
  if (!dpts) {
    CK(cudaMemcpyAsync(b.pts_tmp, pts, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice,
                       ctx->stream), "copy points");
    d_pts = b.pts_tmp;
  }
  int32_t *d_lab = dlab ? labels : b.labels_tmp;
  float *d_om = omega;
  if (omega && !dom) {
    if (b.cap_omega < (int64_t)C * n) {
      if (b.omega_tmp) cudaFree(b.omega_tmp);
      b.omega_tmp = nullptr;
      b.cap_omega = 0;
      CK(cudaMalloc(&b.omega_tmp, (size_t)C * n * sizeof(float)), "cudaMalloc(omega)");
      b.cap_omega = (int64_t)C * n;
    }
    d_om = b.omega_tmp;
  }
  LaunchShape shape;
  int64_t launches = 0;
  st = enqueue_labeling(ctx, d_pts, n, d_lab, d_om, o, d_masks, full_masks, stats != nullptr, &shape, &launches);
  if (st) return st;
  if (!dlab)
    CK(cudaMemcpyAsync(labels, d_lab, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
       "copy labels");
  if (omega && !dom)
    CK(cudaMemcpyAsync(omega, d_om, (size_t)C * n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream),
       "copy omega");
  if (stats || !dpts || !dlab || !dom) {
    st = zef_synchronize(ctx);
    if (st) return st;
  }
  if (stats) {
    CK(cudaMemcpy(ctx->h_counters, b.counters, CNT_COUNT_ * sizeof(int64_t), cudaMemcpyDeviceToHost),
       "read counters");
    const int64_t *h = ctx->h_counters;
    stats->points = n;
    stats->nonfinite_points = h[CNT_NONFINITE];
    int64_t tt = 0;
    for (auto &c : ctx->comps) tt += c.nt;
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
    stats->block_threads = shape.threads;
    stats->points_per_thread = shape.ppt;
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

}  // namespace zef

extern "C" {

zef_status zef_relabel_boundary(zef_ctx *ctx, const float *nodes, int64_t n_nodes, const int32_t *tets,
                                int64_t n_tets, int32_t *node_labels, int32_t max_passes,
                                const zef_label_opts *opts, zef_relabel_pass *per_pass, int32_t *passes,
                                int32_t *converged) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->comps.empty()) return fail(ctx, ZEF_ERR_NOT_READY, "no compartment registered");
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context cannot label");
  if (max_passes < 1 || max_passes > 1024) return fail(ctx, ZEF_ERR_INVALID_ARG, "max_passes must be in [1, 1024]");
  if (n_nodes < 0 || n_tets < 0 || (n_nodes > 0 && (!nodes || !node_labels)) || (n_tets > 0 && !tets))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad nodes/tets/labels arguments");
  if (n_nodes > ((int64_t)1 << 31) - 1 || n_tets > ((int64_t)1 << 31) - 1)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "too many nodes or tets (max 2^31-1)");
  if (n_tets > 0 && n_nodes == 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "tets without nodes");
  zef_label_opts o;
  if (opts) o = *opts; else std::memset(&o, 0, sizeof(o));
  fill_default_opts(&o);
  if (o.precision < 0 || o.precision > 2 || o.kernel < 0 || o.kernel > 2)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad precision or kernel");
  if (o.flags & ~kLabelFlagsAll) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown label flags");
  if ((o.block_threads || o.points_per_thread) && !shape_valid(o.block_threads, o.points_per_thread))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad launch shape (threads 128/256, points 2/4)");
  if (per_pass) std::memset(per_pass, 0, sizeof(zef_relabel_pass) * (size_t)max_passes);
  if (passes) *passes = 0;
  if (converged) *converged = 0;
  DeviceGuard g(ctx->device);
  zef_status st = ensure_uploaded(ctx);
  if (st) return st;
  return relabel_run(ctx, nodes, n_nodes, tets, n_tets, node_labels, max_passes, o, per_pass, passes, converged);
}

zef_status zef_taubin_smooth(zef_ctx *ctx, float *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                             const uint8_t *fixed, const zef_smooth_opts *opts, int32_t *iterations) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context");
  if (!opts || n_nodes < 0 || n_tets < 0 || (n_nodes > 0 && !nodes) || (n_tets > 0 && !tets))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad smoothing arguments");
  if (n_nodes > ((int64_t)1 << 31) - 1 || n_tets > ((int64_t)1 << 31) - 1)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "too many nodes or tets (max 2^31-1)");
  if (n_tets > 0 && n_nodes == 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "tets without nodes");
  if (!(opts->lambda >= 0.f && opts->lambda < 1.f) || !(opts->mu >= 0.f && opts->mu < 1.f) ||
      !(opts->xi >= 0.f) || opts->max_iters < 1 || opts->max_iters > 100000)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "smoothing parameters out of range");
  if (iterations) *iterations = 0;
  if (n_nodes == 0) return ZEF_OK;
  DeviceGuard g(ctx->device);
  return taubin_run(ctx, nodes, n_nodes, tets, n_tets, fixed, *opts, iterations);
}

zef_status zef_taubin_smooth_surface(zef_ctx *ctx, float *nodes, int64_t n_nodes, const int32_t *tets,
                                     int64_t n_tets, const int32_t *elem_labels, const zef_smooth_opts *opts,
                                     int32_t *iterations, int64_t *boundary_faces) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context");
  if (!opts || n_nodes < 0 || n_tets < 0 || (n_nodes > 0 && !nodes) || (n_tets > 0 && (!tets || !elem_labels)))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad smoothing arguments");
  if (n_nodes > ((int64_t)1 << 31) - 1 || n_tets > ((int64_t)1 << 31) - 1)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "too many nodes or tets (max 2^31-1)");
  if (n_tets > 0 && n_nodes == 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "tets without nodes");
  if (!(opts->lambda >= 0.f && opts->lambda < 1.f) || !(opts->mu >= 0.f && opts->mu < 1.f) ||
      !(opts->xi >= 0.f) || opts->max_iters < 1 || opts->max_iters > 100000)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "smoothing parameters out of range");
  if (iterations) *iterations = 0;
  if (boundary_faces) *boundary_faces = 0;
  if (n_nodes == 0) return ZEF_OK;
  DeviceGuard g(ctx->device);
  return taubin_surface_run(ctx, nodes, n_nodes, tets, n_tets, elem_labels, *opts, iterations, boundary_faces);
}

zef_status zef_inflate(zef_ctx *ctx, float *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                       int32_t compartment_id, float zeta, int64_t *moved) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->comps.empty()) return fail(ctx, ZEF_ERR_NOT_READY, "no compartment registered");
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context");
  if (n_nodes < 0 || n_tets < 0 || (n_nodes > 0 && !nodes) || (n_tets > 0 && !tets))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad inflation arguments");
  if (n_nodes > ((int64_t)1 << 31) - 1 || n_tets > ((int64_t)1 << 31) - 1)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "too many nodes or tets (max 2^31-1)");
  if (n_tets > 0 && n_nodes == 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "tets without nodes");
  if (!(zeta >= 0.f && zeta < 1.f)) return fail(ctx, ZEF_ERR_INVALID_ARG, "zeta must be in [0, 1)");
  if (moved) *moved = 0;
  if (n_nodes == 0) return ZEF_OK;
  DeviceGuard g(ctx->device);
  zef_status st = ensure_uploaded(ctx);
  if (st) return st;
  return inflate_run(ctx, nodes, n_nodes, tets, n_tets, compartment_id, zeta, moved);
}

zef_status zef_refine_and_relabel(zef_ctx *ctx, zef_mesh *mesh, int32_t levels, const zef_label_opts *opts,
                                  zef_level_stats *per_level) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->comps.empty()) return fail(ctx, ZEF_ERR_NOT_READY, "no compartment registered");
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context cannot refine");
  if (!mesh || levels < 0 || levels > 32) return fail(ctx, ZEF_ERR_INVALID_ARG, "bad mesh/levels");
  if (!mesh->nodes || !mesh->tets || !mesh->node_labels || mesh->num_nodes < 0 || mesh->num_tets < 0 ||
      mesh->num_nodes > mesh->node_capacity || mesh->num_tets > mesh->tet_capacity ||
      mesh->node_capacity >= ((int64_t)1 << 31) || mesh->tet_capacity >= ((int64_t)1 << 31))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad mesh arrays or capacities");
  if (mesh->flags & ~(int32_t)ZEF_REFINE_CONFORMING) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown mesh flags");
  zef_label_opts o;
  if (opts) o = *opts; else std::memset(&o, 0, sizeof(o));
  fill_default_opts(&o);
  if (o.precision < 0 || o.precision > 2 || o.kernel < 0 || o.kernel > 2)
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad precision or kernel");
  if (o.flags & ~kLabelFlagsAll) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown label flags");
  if ((o.block_threads || o.points_per_thread) && !shape_valid(o.block_threads, o.points_per_thread))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "bad launch shape (threads 128/256, points 2/4)");
  DeviceGuard g(ctx->device);
  zef_status st = ensure_uploaded(ctx);
  if (st) return st;
  return refine_run(ctx, mesh, levels, o, per_level);
}

}  // extern "C"

namespace zef {

template <class T>
zef_status ensure_buffer(zef_ctx *ctx, T **p, int64_t *cap, int64_t need) {
  if (*p && *cap >= need) return ZEF_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cudaError_t e = cudaMalloc((void **)p, (size_t)std::max<int64_t>(need, 1) * sizeof(T));
  if (e != cudaSuccess) {
    *cap = 0;
    return cuda_fail(ctx, e, "cudaMalloc");
  }
  *cap = need;
  return ZEF_OK;
}
template zef_status ensure_buffer<float>(zef_ctx *, float **, int64_t *, int64_t);
template zef_status ensure_buffer<int32_t>(zef_ctx *, int32_t **, int64_t *, int64_t);
template zef_status ensure_buffer<unsigned long long>(zef_ctx *, unsigned long long **, int64_t *, int64_t);

zef_status ensure_uploaded(zef_ctx *ctx) {
  if (ctx->device == ZEF_HOST_ONLY) return ZEF_OK;
  if (!ctx->dirty) return ZEF_OK;
  const int C = (int)ctx->comps.size();
  if (C == 0) return ZEF_OK;
  int64_t ne = (int64_t)ctx->h_entries.size();
  int64_t ntv = (int64_t)ctx->h_tris.size();
  if (ctx->d_entries_cap < ne) {
    if (ctx->d_entries) cudaFree(ctx->d_entries);
    ctx->d_entries = nullptr;
    CK(cudaMalloc(&ctx->d_entries, ne * sizeof(Entry)), "cudaMalloc(entries)");
    ctx->d_entries_cap = ne;
  }
  if (ctx->d_tris_cap < ntv) {
    if (ctx->d_tris) cudaFree(ctx->d_tris);
    ctx->d_tris = nullptr;
    CK(cudaMalloc(&ctx->d_tris, ntv * sizeof(float4)), "cudaMalloc(tris)");
    ctx->d_tris_cap = ntv;
  }
  if (!ctx->d_comps) {
    CK(cudaMalloc(&ctx->d_comps, ZEF_MAX_COMPARTMENTS * sizeof(DevComp)), "cudaMalloc(comps)");
    CK(cudaMalloc(&ctx->d_row_ids, ZEF_MAX_COMPARTMENTS * sizeof(int32_t)), "cudaMalloc(rows)");
    CK(cudaMalloc(&ctx->d_lpt, ZEF_MAX_COMPARTMENTS * sizeof(int32_t)), "cudaMalloc(lpt)");
    CK(cudaMalloc(&ctx->d_dop, ZEF_MAX_COMPARTMENTS * kDop * sizeof(float)), "cudaMalloc(dop)");
  }
  // power-of-two scale: the largest |coordinate| of the surfaces -> [32, 64)
  float m = 0.f;
  for (const CompHost &h : ctx->comps)
    for (int k = 0; k < 3; ++k) m = std::max(m, std::max(std::fabs(h.lo[k]), std::fabs(h.hi[k])));
  int ex = 0;
  std::frexp(m, &ex);  // m = f 2^ex, f in [0.5, 1)
  const float s = (m > 0.f) ? std::ldexp(1.f, 6 - ex) : 1.f;
  const float s2 = s * s;
  ctx->scale = s;
  std::vector<Entry> es(ctx->h_entries);
  for (Entry &e : es) {
    e.v.x *= s; e.v.y *= s; e.v.z *= s;
    e.n.x *= s2; e.n.y *= s2; e.n.z *= s2; e.n.w *= s2;
  }
  std::vector<float4> ts(ctx->h_tris);
  for (float4 &t : ts) {
    t.x *= s; t.y *= s; t.z *= s;
  }
  // cap trees: vertices scale by s, normals and kappa |n| by s^2 (exact)
  std::vector<CapNode> ns(ctx->h_nodes);
  for (CapNode &nd : ns)
    for (int k = 0; k < 3; ++k) {
      nd.lo[k] *= s;
      nd.hi[k] *= s;
    }
  if (ctx->d_nodes_cap < (int64_t)ns.size()) {
    if (ctx->d_nodes) cudaFree(ctx->d_nodes);
    ctx->d_nodes = nullptr;
    CK(cudaMalloc(&ctx->d_nodes, std::max<size_t>(ns.size(), 1) * sizeof(CapNode)), "cudaMalloc(cap nodes)");
    ctx->d_nodes_cap = (int64_t)ns.size();
  }
  if (!ns.empty()) CK(cudaMemcpy(ctx->d_nodes, ns.data(), ns.size() * sizeof(CapNode), cudaMemcpyHostToDevice), "upload cap nodes");
  std::vector<Entry> gs(ctx->h_cseg);
  for (Entry &e : gs) {
    e.v.x *= s; e.v.y *= s; e.v.z *= s;
    e.n.x *= s2; e.n.y *= s2; e.n.z *= s2; e.n.w *= s2;
  }
  if (ctx->d_cseg_cap < (int64_t)gs.size()) {
    if (ctx->d_cseg) cudaFree(ctx->d_cseg);
    ctx->d_cseg = nullptr;
    CK(cudaMalloc(&ctx->d_cseg, std::max<size_t>(gs.size(), 1) * sizeof(Entry)), "cudaMalloc(cap segments)");
    ctx->d_cseg_cap = (int64_t)gs.size();
  }
  if (!gs.empty()) CK(cudaMemcpy(ctx->d_cseg, gs.data(), gs.size() * sizeof(Entry), cudaMemcpyHostToDevice), "upload cap segments");
  if (ctx->d_ctidx_cap < (int64_t)ctx->h_ctidx.size()) {
    if (ctx->d_ctidx) cudaFree(ctx->d_ctidx);
    ctx->d_ctidx = nullptr;
    CK(cudaMalloc(&ctx->d_ctidx, std::max<size_t>(ctx->h_ctidx.size(), 1) * sizeof(int32_t)),
       "cudaMalloc(cap-tree triangle order)");
    ctx->d_ctidx_cap = (int64_t)ctx->h_ctidx.size();
  }
  if (!ctx->h_ctidx.empty())
    CK(cudaMemcpy(ctx->d_ctidx, ctx->h_ctidx.data(), ctx->h_ctidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice),
       "upload cap-tree triangle order");
  // union box of the surfaces in the caller's coordinates: the binning keys'
  // range (a point outside it is outside every compartment's box)
  UnionBox ub;
  for (int k = 0; k < 3; ++k) {
    ub.lo[k] = std::numeric_limits<float>::infinity();
    ub.hi[k] = -std::numeric_limits<float>::infinity();
  }
  for (const CompHost &h : ctx->comps)
    for (int k = 0; k < 3; ++k) {
      ub.lo[k] = std::min(ub.lo[k], h.lo[k]);
      ub.hi[k] = std::max(ub.hi[k], h.hi[k]);
    }
  // cubic Morton cells: the scale of the box's longest side on every axis
  float ext = 0.f;
  for (int k = 0; k < 3; ++k) ext = std::max(ext, ub.hi[k] - ub.lo[k]);
  for (int k = 0; k < 3; ++k) ub.sc[k] = ext > 0.f ? (float)(1 << kMortonBits) / ext : 0.f;
  ctx->ubox = ub;
  std::vector<DevComp> dc(C);
  std::vector<int32_t> rows(C), lpt(C);
  for (int i = 0; i < C; ++i) {
    const CompHost &h = ctx->comps[i];
    DevComp &d = dc[i];
    for (int k = 0; k < 3; ++k) {
      d.lo[k] = h.lo[k] * s;
      d.hi[k] = h.hi[k] * s;
    }
    d.entry_off = (int32_t)h.entry_off;
    d.entry_cnt = (int32_t)h.entry_cnt;
    d.tri_off = (int32_t)h.tri_off;
    d.tri_cnt = (int32_t)h.nt;
    d.cap_root = h.cap_root;
    d.cseg_off = (int32_t)h.cseg_off;
    d.cseg_leaf = (int32_t)h.cseg_leaf;
    d.pad_ = 0;
    d.id = h.id;
    d.row = -1;
    for (int r = 0; r < C; ++r)
      if (ctx->priority[r] == h.id) d.row = r;
    rows[d.row] = h.id;
  }
  // hull bounds in scaled coordinates: h s (exact power-of-two scaling) plus a
  // margin that covers the float evaluation of d . p for |p| <= 1000 (scaled
  // units; every surface lies within 64), rounded up to float
  std::vector<float> dop((size_t)C * kDop);
  for (int i = 0; i < C; ++i)
    for (int k = 0; k < kDop; ++k) {
      const double thr = ctx->comps[i].dop[k] * s + 6.4e-4;
      float f = (float)thr;
      if ((double)f < thr) f = std::nextafter(f, std::numeric_limits<float>::infinity());
      dop[(size_t)i * kDop + k] = f;
    }
  std::iota(lpt.begin(), lpt.end(), 0);
  std::stable_sort(lpt.begin(), lpt.end(),
                   [&](int a, int b) { return ctx->comps[a].nt > ctx->comps[b].nt; });
  CK(cudaMemcpy(ctx->d_dop, dop.data(), dop.size() * sizeof(float), cudaMemcpyHostToDevice), "upload dop");
  CK(cudaMemcpy(ctx->d_entries, es.data(), ne * sizeof(Entry), cudaMemcpyHostToDevice), "upload entries");
  CK(cudaMemcpy(ctx->d_tris, ts.data(), ntv * sizeof(float4), cudaMemcpyHostToDevice), "upload tris");
  CK(cudaMemcpy(ctx->d_comps, dc.data(), C * sizeof(DevComp), cudaMemcpyHostToDevice), "upload comps");
  CK(cudaMemcpy(ctx->d_row_ids, rows.data(), C * sizeof(int32_t), cudaMemcpyHostToDevice), "upload rows");
  CK(cudaMemcpy(ctx->d_lpt, lpt.data(), C * sizeof(int32_t), cudaMemcpyHostToDevice), "upload lpt");
  ctx->dirty = false;
  ++ctx->gen;
  return ZEF_OK;
}

}  // namespace zef

// Copy of compartment `index`'s strip stream (8 floats per entry: vertex
// x, y, z, weight, normal x, y, z, kappa) for host-side checks; returns the
// entry count in *count and copies min(count, cap) entries.
extern "C" zef_status zef_debug_strip_entries(const zef_ctx *ctx, int32_t index, float *out, int64_t cap,
                                              int64_t *count) {
  if (!ctx || index < 0 || index >= (int32_t)ctx->comps.size() || !count) return ZEF_ERR_INVALID_ARG;
  const CompHost &c = ctx->comps[index];
  *count = c.entry_cnt;
  if (out) {
    const int64_t m = std::min(cap, c.entry_cnt);
    std::memcpy(out, ctx->h_entries.data() + c.entry_off, (size_t)m * sizeof(Entry));
  }
  return ZEF_OK;
}

// Strip statistics for diagnostics (not part of the public header's promises):
// number of stream entries and strips of compartment `index`.
extern "C" zef_status zef_debug_strip_stats(const zef_ctx *ctx, int32_t index, int64_t *entries,
                                            int64_t *strips) {
  if (!ctx || index < 0 || index >= (int32_t)ctx->comps.size()) return ZEF_ERR_INVALID_ARG;
  if (entries) *entries = ctx->comps[index].entry_cnt;
  if (strips) *strips = ctx->comps[index].nstrips;
  return ZEF_OK;
}

extern "C" zef_status zef_debug_half_angle(zef_ctx *ctx, const float *y, const float *x, float *out,
                                           int64_t n) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context");
  if (n < 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "negative count");
  if (n == 0) return ZEF_OK;
  if (!y || !x || !out) return fail(ctx, ZEF_ERR_INVALID_ARG, "null array");
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(y, ctx->device) || !is_device_ptr(x, ctx->device) || !is_device_ptr(out, ctx->device))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "arrays must be device memory of the context's device");
  zef_status st = launch_debug_half_angle(ctx, y, x, out, n);
  if (st) return st;
  return zef_synchronize(ctx);
}

extern "C" zef_status zef_debug_cap_tree(const zef_ctx *ctx, int32_t index, int64_t *n_nodes, int64_t *n_entries,
                                         float *boxes, int32_t *links, float *entries) {
  if (!ctx || index < 0 || index >= (int32_t)ctx->comps.size() || !n_nodes || !n_entries) return ZEF_ERR_INVALID_ARG;
  const CompHost &c = ctx->comps[(size_t)index];
  const bool last = index + 1 == (int32_t)ctx->comps.size();
  const int64_t node_end = last ? (int64_t)ctx->h_nodes.size() : ctx->comps[(size_t)index + 1].cap_root;
  const int64_t seg_end = last ? (int64_t)ctx->h_cseg.size() : ctx->comps[(size_t)index + 1].cseg_off;
  *n_nodes = node_end - c.cap_root;
  *n_entries = seg_end - c.cseg_off;
  for (int64_t k = 0; k < *n_nodes; ++k) {
    const CapNode &nd = ctx->h_nodes[(size_t)(c.cap_root + k)];
    if (boxes)
      for (int d = 0; d < 3; ++d) {
        boxes[6 * k + d] = nd.lo[d];
        boxes[6 * k + 3 + d] = nd.hi[d];
      }
    if (links) {
      int32_t *l = links + 9 * k;
      l[0] = nd.left < 0 ? -1 : nd.left - c.cap_root;
      l[1] = nd.right < 0 ? -1 : nd.right - c.cap_root;
      l[2] = nd.left < 0 ? nd.leaf_begin - (int32_t)c.cseg_off : 0;
      l[3] = nd.left < 0 ? nd.leaf_cnt : 0;
      l[4] = nd.cap_begin - (int32_t)c.cseg_off;
      l[5] = nd.cap_cnt;
      l[6] = nd.left < 0 ? nd.leaf_tris : 0;
      l[7] = nd.cap_tris;
      l[8] = nd.skip - c.cap_root;
    }
  }
  if (entries)
    std::memcpy(entries, ctx->h_cseg.data() + c.cseg_off, (size_t)*n_entries * sizeof(Entry));
  return ZEF_OK;
}

extern "C" zef_status zef_debug_fma_rate(zef_ctx *ctx, int32_t fp64, double *tflops) {
  if (!ctx || !tflops) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context");
  DeviceGuard g(ctx->device);
  return debug_fma_rate(ctx, fp64 != 0, tflops);
}

extern "C" zef_status zef_debug_wait_probe(zef_ctx *ctx, int64_t limit_ns) {
  if (!ctx) return ZEF_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->device == ZEF_HOST_ONLY) return fail(ctx, ZEF_ERR_NOT_READY, "host-only context");
  if (limit_ns <= 0 || limit_ns > 2000000000LL) return fail(ctx, ZEF_ERR_INVALID_ARG, "limit must be in (0, 2 s]");
  DeviceGuard g(ctx->device);
  zef_status st = launch_wait_probe(ctx, limit_ns);
  if (st) return st;
  return zef_synchronize(ctx);
}
