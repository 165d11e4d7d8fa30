// Refinement and recursive re-labeling (Sec. 2.1.2 and Sec. 2.1.3 item 2).
//
// One level, entirely on the device with device-resident counts:
//   k_rf_flag      tets whose four node labels are not all equal (the tissue
//                  boundary of the labeled mesh) -> flag
//   scan           rank of every flagged tet, count F
//   k_rf_check     capacity checks (tets M + 7F, hash table)
//   k_rf_insert    the six edges of every flagged tet into an open-addressing
//                  table keyed by the sorted node pair; atomicMin keeps the
//                  smallest (rank, local edge) code, i.e. the first appearance
//   k_rf_owner/scan  new node numbers in order of first appearance, count K
//   k_rf_nodes     the K edge midpoints, rounded once to float32
//   label pipeline only the K new nodes are labeled (zef_label.cu)
//   k_rf_children  1 -> 8 split: the slot of the flagged tet receives child 0,
//                  children 1..7 are appended; the octahedron is cut along its
//                  shortest diagonal (float32 squared lengths, ties to the
//                  lower diagonal index)
//   k_rf_advance   per-level statistics, N += K, M += 7F
// The `levels` iterations are captured once into a CUDA graph and launched as
// one unit; no host round trip happens between levels.
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

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kLevelStats = 10;

// local node numbering of a flagged tet: 0..3 corners, 4 = m01, 5 = m02,
// 6 = m03, 7 = m12, 8 = m13, 9 = m23
__constant__ int c_edge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int c_child[3][8][4] = {
    // diagonal m01-m23
    {{0, 4, 5, 6}, {4, 1, 7, 8}, {5, 7, 2, 9}, {6, 8, 9, 3},
     {4, 9, 5, 6}, {4, 9, 6, 8}, {4, 9, 8, 7}, {4, 9, 7, 5}},
    // diagonal m02-m13
    {{0, 4, 5, 6}, {4, 1, 7, 8}, {5, 7, 2, 9}, {6, 8, 9, 3},
     {5, 8, 6, 4}, {5, 8, 9, 6}, {5, 8, 7, 9}, {5, 8, 4, 7}},
    // diagonal m03-m12
    {{0, 4, 5, 6}, {4, 1, 7, 8}, {5, 7, 2, 9}, {6, 8, 9, 3},
     {6, 7, 4, 5}, {6, 7, 5, 9}, {6, 7, 9, 8}, {6, 7, 8, 4}},
};
__constant__ int c_diag[3][2] = {{4, 9}, {5, 8}, {6, 7}};

// Conforming closure (Sec. 2.1.2, Fig. 2 c-e), per 6-bit mask of split
// edges (bit e = local edge e): number of children (0: nothing to split,
// -1: the pattern is split into eight), the children for the two quad
// diagonals of a two-edge pattern (the same twice otherwise) and those two
// diagonals.  Filled on the host by green_tables().
__constant__ int c_gn[64];
__constant__ signed char c_gch[64][2][4][4];
__constant__ signed char c_gdg[64][2][2];
constexpr int kClosureMaxPasses = 4096;

struct RF {
  float *nodes;
  int32_t *tets;
  int32_t *labels;
  int64_t *cnt;
  uint32_t *flags;   // [tet_cap], scanned in place
  uint32_t *owned;   // [6 fmax], scanned in place
  unsigned long long *hkeys;
  uint32_t *hvals;
  int32_t *hids;
  unsigned long long hmask;
  int64_t node_cap, tet_cap, fmax;
  uint32_t *status;
  int64_t *lstats;
  uint8_t *state;    // conforming: 0 not split into eight, 1 red, 2 red with edges not yet inserted
  uint32_t *gx;      // conforming: extra children of each green split, scanned in place
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ unsigned long long edge_key(int32_t a, int32_t b) {
  const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
  return ((unsigned long long)lo << 32) | hi;
}

__device__ __forceinline__ bool is_flagged(const RF &r, int64_t t, int64_t M, uint32_t *rank) {
  const uint32_t s = r.flags[t];
  const uint32_t nx = (t + 1 < M) ? r.flags[t + 1] : (uint32_t)r.cnt[CNT_LEVEL_FLAGGED];
  *rank = s;
  return nx != s;
}

// slot of a key known to be in the table (bounded probe)
__device__ __forceinline__ unsigned long long find_slot(const RF &r, unsigned long long key) {
  unsigned long long h = mix64(key) & r.hmask;
  for (unsigned long long it = 0; it <= r.hmask; ++it) {
    if (r.hkeys[h] == key) return h;
    h = (h + 1) & r.hmask;
  }
  return 0;  // unreachable when the key was inserted
}

__global__ void k_rf_init(int64_t *cnt, int64_t n, int64_t m) {
  if (threadIdx.x == 0) {
    cnt[CNT_NODES] = n;
    cnt[CNT_TETS] = m;
    cnt[CNT_ABORT] = 0;
    cnt[CNT_LEVEL_SEED] = cnt[CNT_CL_CHANGED] = cnt[CNT_CL_ITER] = 0;
    cnt[CNT_CL_GREEN] = cnt[CNT_CL_GEXTRA] = 0;
  }
}

// ---- conforming closure
// true when the key is in the table (bounded probe)
__device__ __forceinline__ bool edge_present(const RF &r, unsigned long long key) {
  unsigned long long h = mix64(key) & r.hmask;
  for (unsigned long long it = 0; it <= r.hmask; ++it) {
    const unsigned long long k = r.hkeys[h];
    if (k == key) return true;
    if (k == kEmpty) return false;
    h = (h + 1) & r.hmask;
  }
  return false;
}

__device__ __forceinline__ int split_mask(const RF &r, const int32_t *v) {
  int m = 0;
#pragma unroll
  for (int e = 0; e < 6; ++e)
    if (edge_present(r, edge_key(v[c_edge[e][0]], v[c_edge[e][1]]))) m |= 1 << e;
  return m;
}

__global__ void k_cl_reset(int64_t *cnt) {
  if (threadIdx.x == 0) {
    cnt[CNT_LEVEL_SEED] = cnt[CNT_CL_CHANGED] = cnt[CNT_CL_ITER] = 0;
    cnt[CNT_CL_GREEN] = cnt[CNT_CL_GEXTRA] = 0;
  }
}

// the tets flagged by their labels start the red set
__global__ void __launch_bounds__(256) k_cl_seed(RF r) {
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < M; t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    const bool f = t < M && r.flags[t] != 0u;
    if (t < M) r.state[t] = f ? 2 : 0;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && b)
      atomicAdd((unsigned long long *)(r.cnt + CNT_LEVEL_SEED), (unsigned long long)__popc(b));
  }
}

// closure pass, part 1: the edges of the tets made red by the last pass
__global__ void __launch_bounds__(256) k_cl_insert(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    if (r.state[t] != 2) continue;
    const int32_t *v = r.tets + 4 * t;
    for (int e = 0; e < 6; ++e) {
      const unsigned long long key = edge_key(v[c_edge[e][0]], v[c_edge[e][1]]);
      unsigned long long h = mix64(key) & r.hmask;
      for (unsigned long long it = 0; it <= r.hmask; ++it) {
        const unsigned long long prev = atomicCAS(r.hkeys + h, kEmpty, key);
        if (prev == kEmpty || prev == key) break;
        h = (h + 1) & r.hmask;
      }
    }
    r.state[t] = 1;
  }
}

// closure pass, part 2: a tet whose split edges form no green pattern turns red
__global__ void __launch_bounds__(256) k_cl_check(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < M; t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    bool promote = false;
    if (t < M && r.state[t] == 0) {
      promote = c_gn[split_mask(r, r.tets + 4 * t)] < 0;
      if (promote) r.state[t] = 2;
    }
    const unsigned b = __ballot_sync(0xffffffffu, promote);
    if ((threadIdx.x & 31) == 0 && b)
      atomicAdd((unsigned long long *)(r.cnt + CNT_CL_CHANGED), (unsigned long long)__popc(b));
  }
}

// closure pass, part 3: loop while a pass promoted a tet (bounded)
__global__ void k_cl_next(RF r, cudaGraphConditionalHandle handle) {
  if (threadIdx.x != 0) return;
  const int64_t changed = r.cnt[CNT_CL_CHANGED];
  r.cnt[CNT_CL_CHANGED] = 0;
  const int64_t it = ++r.cnt[CNT_CL_ITER];
  bool more = changed > 0 && !r.cnt[CNT_ABORT];
  if (more && it >= kClosureMaxPasses) {
    r.cnt[CNT_ABORT] = 1;
    atomicOr(r.status, ST_CAPACITY);
    more = false;
  }
  cudaGraphSetConditional(handle, more ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_cl_red(RF r) {
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x)
    r.flags[t] = r.state[t] != 0 ? 1u : 0u;
}

// extra children of every green split (scanned afterwards into offsets)
__global__ void __launch_bounds__(256) k_cl_gcount(RF r) {
  const int64_t M = r.cnt[CNT_TETS];
  const bool ab = r.cnt[CNT_ABORT] != 0;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < M; t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    int n = 0;
    if (t < M && !ab && r.state[t] == 0) n = c_gn[split_mask(r, r.tets + 4 * t)];
    if (t < M) r.gx[t] = n > 1 ? (uint32_t)(n - 1) : 0u;
    const unsigned b = __ballot_sync(0xffffffffu, n > 1);
    if ((threadIdx.x & 31) == 0 && b)
      atomicAdd((unsigned long long *)(r.cnt + CNT_CL_GREEN), (unsigned long long)__popc(b));
  }
}

// tet capacity including the green children
__global__ void k_cl_check3(RF r) {
  if (threadIdx.x != 0) return;
  const int64_t F = r.cnt[CNT_LEVEL_FLAGGED], M = r.cnt[CNT_TETS], G = r.cnt[CNT_CL_GEXTRA];
  if (!r.cnt[CNT_ABORT] && M + 7 * F + G > r.tet_cap) {
    r.cnt[CNT_ABORT] = 1;
    atomicOr(r.status, ST_CAPACITY);
  }
}


__global__ void __launch_bounds__(256) k_rf_flag(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    const int4 q = reinterpret_cast<const int4 *>(r.tets)[t];
    const int64_t N = r.cnt[CNT_NODES];
    if (q.x < 0 || q.y < 0 || q.z < 0 || q.w < 0 || q.x >= N || q.y >= N || q.z >= N || q.w >= N) {
      // a node index outside [0, num_nodes): stop the refinement, report it
      r.flags[t] = 0u;
      atomicOr(r.status, ST_INVALID);
      atomicExch((unsigned long long *)(r.cnt + CNT_ABORT), 1ull);
      continue;
    }
    const int32_t l0 = r.labels[q.x], l1 = r.labels[q.y], l2 = r.labels[q.z], l3 = r.labels[q.w];
    r.flags[t] = (l0 != l1 || l0 != l2 || l0 != l3) ? 1u : 0u;
  }
}

__global__ void k_rf_check(RF r) {
  if (threadIdx.x != 0) return;
  const int64_t F = r.cnt[CNT_LEVEL_FLAGGED], M = r.cnt[CNT_TETS];
  if (!r.cnt[CNT_ABORT] && (F > r.fmax || M + 7 * F > r.tet_cap)) {
    r.cnt[CNT_ABORT] = 1;
    atomicOr(r.status, ST_CAPACITY);
  }
  r.cnt[CNT_OWN_LEN] = r.cnt[CNT_ABORT] ? 0 : 6 * F;
}

__global__ void __launch_bounds__(256) k_rf_insert(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rank;
    if (!is_flagged(r, t, M, &rank)) continue;
    const int32_t *v = r.tets + 4 * t;
    for (int e = 0; e < 6; ++e) {
      const unsigned long long key = edge_key(v[c_edge[e][0]], v[c_edge[e][1]]);
      const uint32_t code = rank * 6u + (uint32_t)e;
      unsigned long long h = mix64(key) & r.hmask;
      for (unsigned long long it = 0; it <= r.hmask; ++it) {
        const unsigned long long prev = atomicCAS(r.hkeys + h, kEmpty, key);
        if (prev == kEmpty || prev == key) {
          atomicMin(r.hvals + h, code);
          break;
        }
        h = (h + 1) & r.hmask;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_rf_owner(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rank;
    if (!is_flagged(r, t, M, &rank)) continue;
    const int32_t *v = r.tets + 4 * t;
    for (int e = 0; e < 6; ++e) {
      const unsigned long long key = edge_key(v[c_edge[e][0]], v[c_edge[e][1]]);
      const uint32_t code = rank * 6u + (uint32_t)e;
      r.owned[code] = (r.hvals[find_slot(r, key)] == code) ? 1u : 0u;
    }
  }
}

// after the owner scan: node capacity, and the counts of the label pipeline
__global__ void k_rf_check2(RF r) {
  if (threadIdx.x != 0) return;
  const int64_t K = r.cnt[CNT_LEVEL_NEW], N = r.cnt[CNT_NODES];
  if (!r.cnt[CNT_ABORT] && N + K > r.node_cap) {
    r.cnt[CNT_ABORT] = 1;
    atomicOr(r.status, ST_CAPACITY);
  }
  r.cnt[CNT_N] = r.cnt[CNT_ABORT] ? 0 : K;
  r.cnt[CNT_OFF] = N;
}

__global__ void __launch_bounds__(256) k_rf_nodes(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS], N = r.cnt[CNT_NODES];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rank;
    if (!is_flagged(r, t, M, &rank)) continue;
    const int32_t *v = r.tets + 4 * t;
    for (int e = 0; e < 6; ++e) {
      const int32_t a = v[c_edge[e][0]], b = v[c_edge[e][1]];
      const unsigned long long key = edge_key(a, b);
      const uint32_t code = rank * 6u + (uint32_t)e;
      const unsigned long long slot = find_slot(r, key);
      if (r.hvals[slot] != code) continue;
      const int64_t id = N + r.owned[code];
      r.hids[slot] = (int32_t)id;
      const int32_t lo = min(a, b), hi = max(a, b);
      for (int k = 0; k < 3; ++k)
        r.nodes[3 * id + k] = __fmul_rn(__fadd_rn(r.nodes[3 * (int64_t)lo + k], r.nodes[3 * (int64_t)hi + k]), 0.5f);
    }
  }
}

__device__ __forceinline__ float len2_rn(const float *p, const float *q) {
  const float dx = __fsub_rn(p[0], q[0]), dy = __fsub_rn(p[1], q[1]), dz = __fsub_rn(p[2], q[2]);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__global__ void __launch_bounds__(256) k_rf_children(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rank;
    if (!is_flagged(r, t, M, &rank)) continue;
    int32_t loc[10];
    for (int k = 0; k < 4; ++k) loc[k] = r.tets[4 * t + k];
    for (int e = 0; e < 6; ++e)
      loc[4 + e] = r.hids[find_slot(r, edge_key(loc[c_edge[e][0]], loc[c_edge[e][1]]))];
    float l[3];
    for (int d = 0; d < 3; ++d)
      l[d] = len2_rn(r.nodes + 3 * (int64_t)loc[c_diag[d][0]], r.nodes + 3 * (int64_t)loc[c_diag[d][1]]);
    int diag = 0;
    if (l[1] < l[diag]) diag = 1;
    if (l[2] < l[diag]) diag = 2;
    for (int c = 0; c < 8; ++c) {
      const int64_t dst = c == 0 ? t : M + 7 * (int64_t)rank + (c - 1);
      const int4 q = make_int4(loc[c_child[diag][c][0]], loc[c_child[diag][c][1]], loc[c_child[diag][c][2]],
                               loc[c_child[diag][c][3]]);
      reinterpret_cast<int4 *>(r.tets)[dst] = q;
    }
  }
}

// green splits: child 0 into the tet's slot, the others after the red children
__global__ void __launch_bounds__(256) k_cl_children(RF r) {
  if (r.cnt[CNT_ABORT]) return;
  const int64_t M = r.cnt[CNT_TETS], F = r.cnt[CNT_LEVEL_FLAGGED];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
    if (r.state[t] != 0) continue;
    int32_t loc[10];
    for (int k = 0; k < 4; ++k) loc[k] = r.tets[4 * t + k];
    const int mask = split_mask(r, loc);
    const int n = c_gn[mask];
    if (n <= 0) continue;
    for (int e = 0; e < 6; ++e)
      loc[4 + e] = ((mask >> e) & 1) ? r.hids[find_slot(r, edge_key(loc[c_edge[e][0]], loc[c_edge[e][1]]))] : -1;
    int alt = 0;
    if (n == 3) {
      const float d0 = len2_rn(r.nodes + 3 * (int64_t)loc[c_gdg[mask][0][0]], r.nodes + 3 * (int64_t)loc[c_gdg[mask][0][1]]);
      const float d1 = len2_rn(r.nodes + 3 * (int64_t)loc[c_gdg[mask][1][0]], r.nodes + 3 * (int64_t)loc[c_gdg[mask][1][1]]);
      alt = d1 < d0 ? 1 : 0;
    }
    const uint32_t off = r.gx[t];
    for (int c = 0; c < n; ++c) {
      const int64_t dst = c == 0 ? t : M + 7 * F + (int64_t)off + (c - 1);
      const signed char *k = c_gch[mask][alt][c];
      reinterpret_cast<int4 *>(r.tets)[dst] = make_int4(loc[k[0]], loc[k[1]], loc[k[2]], loc[k[3]]);
    }
  }
}

__global__ void k_rf_advance(RF r, int level) {
  if (threadIdx.x != 0) return;
  int64_t *s = r.lstats + (int64_t)level * kLevelStats;
  if (r.cnt[CNT_ABORT]) {
    s[0] = s[1] = s[4] = s[5] = s[7] = s[8] = 0;
    s[2] = r.cnt[CNT_NODES];
    s[3] = r.cnt[CNT_TETS];
    s[6] = 1;
    return;
  }
  const int64_t F = r.cnt[CNT_LEVEL_FLAGGED], K = r.cnt[CNT_LEVEL_NEW];
  r.cnt[CNT_NODES] += K;
  r.cnt[CNT_TETS] += 7 * F + r.cnt[CNT_CL_GEXTRA];
  s[7] = r.state ? r.cnt[CNT_LEVEL_SEED] : F;  // tets flagged by their labels
  s[8] = r.state ? r.cnt[CNT_CL_GREEN] : 0;
  s[0] = F;
  s[1] = K;
  s[2] = r.cnt[CNT_NODES];
  s[3] = r.cnt[CNT_TETS];
  s[4] = r.cnt[CNT_PAIRS_EVAL] + r.cnt[CNT_PAIRS_RESCUE];
  s[5] = r.cnt[CNT_UNC];
  s[6] = 0;
}

bool device_ptr(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

zef_status grow(zef_ctx *ctx, int idx, size_t bytes) {
  if (ctx->rf_buf[idx] && ctx->rf_cap[idx] >= bytes) return ZEF_OK;
  if (ctx->rf_buf[idx]) cudaFree(ctx->rf_buf[idx]);
  ctx->rf_buf[idx] = nullptr;
  ctx->rf_cap[idx] = 0;
  if (ctx->rf_exec) {
    cudaGraphExecDestroy(ctx->rf_exec);
    ctx->rf_exec = nullptr;
  }
  CK(cudaMalloc(&ctx->rf_buf[idx], std::max<size_t>(bytes, 256)), "cudaMalloc(refine)");
  ctx->rf_cap[idx] = bytes;
  return ZEF_OK;
}

uint64_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, sizeof(u));
  return u;
}

uint64_t hash_mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// ---- closure tables
int local_edge(int i, int j) {
  static const int E[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
  return E[i][j];
}

struct GreenTables {
  int n[64];
  signed char ch[64][2][4][4];
  signed char dg[64][2][2];
};

// The parent's corners 0..3 with corner x replaced by local node m for each
// (x, m) pair: replacing a corner by a point of an edge leaving another corner
// of the tet keeps the orientation.
void substitute(signed char out[4], std::initializer_list<std::pair<int, int>> pairs) {
  for (int k = 0; k < 4; ++k) out[k] = (signed char)k;
  for (const auto &pm : pairs) out[pm.first] = (signed char)pm.second;
}

void green_tables(GreenTables &g) {
  static const int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  std::memset(&g, 0, sizeof(g));
  for (int mask = 0; mask < 64; ++mask) {
    int bits[6], nb = 0, used = 0;
    for (int e = 0; e < 6; ++e)
      if ((mask >> e) & 1) {
        bits[nb++] = e;
        used |= (1 << E[e][0]) | (1 << E[e][1]);
      }
    int nv = 0;
    for (int v = 0; v < 4; ++v) nv += (used >> v) & 1;
    signed char(*c)[4] = g.ch[mask][0];
    if (nb == 0) {
      g.n[mask] = 0;
    } else if (nb == 1) {  // one edge (i, j): T[j<-m], T[i<-m]
      const int i = E[bits[0]][0], j = E[bits[0]][1], m = 4 + bits[0];
      substitute(c[0], {{j, m}});
      substitute(c[1], {{i, m}});
      g.n[mask] = 2;
    } else if (nb == 2 && nv == 3) {  // two edges (p, q), (p, r) with a common vertex p
      int p = -1;
      for (int v = 0; v < 4; ++v)
        if ((E[bits[0]][0] == v || E[bits[0]][1] == v) && (E[bits[1]][0] == v || E[bits[1]][1] == v)) p = v;
      int o[2] = {0, 0}, no = 0;  // the two used vertices other than p (nv == 3)
      for (int v = 0; v < 4; ++v)
        if (((used >> v) & 1) && v != p && no < 2) o[no++] = v;
      const int q = o[0], r = o[1];  // q < r
      const int mpq = 4 + local_edge(p, q), mpr = 4 + local_edge(p, r);
      substitute(c[0], {{q, mpq}, {r, mpr}});
      substitute(c[1], {{q, mpq}, {p, mpr}});
      substitute(c[2], {{p, mpq}});
      signed char(*c1)[4] = g.ch[mask][1];
      substitute(c1[0], {{q, mpq}, {r, mpr}});
      substitute(c1[1], {{r, mpr}, {p, mpq}});
      substitute(c1[2], {{p, mpr}});
      g.dg[mask][0][0] = (signed char)mpq;
      g.dg[mask][0][1] = (signed char)r;
      g.dg[mask][1][0] = (signed char)q;
      g.dg[mask][1][1] = (signed char)mpr;
      g.n[mask] = 3;
      continue;
    } else if (nb == 3 && nv == 3) {  // the three edges of face (p, q, r)
      int f[3], nf = 0;
      for (int v = 0; v < 4; ++v)
        if ((used >> v) & 1) f[nf++] = v;
      const int p = f[0], q = f[1], r = f[2];
      const int mpq = 4 + local_edge(p, q), mpr = 4 + local_edge(p, r), mqr = 4 + local_edge(q, r);
      substitute(c[0], {{q, mpq}, {r, mpr}});
      substitute(c[1], {{p, mpq}, {r, mqr}});
      substitute(c[2], {{p, mpr}, {q, mqr}});
      substitute(c[3], {{p, mqr}, {q, mpr}, {r, mpq}});
      g.n[mask] = 4;
    } else {
      g.n[mask] = -1;  // split into eight
    }
    std::memcpy(g.ch[mask][1], g.ch[mask][0], sizeof(g.ch[mask][0]));
  }
}

// Appends to the graph being captured on `cap` a conditional while-node that
// becomes the capture's new dependency, and captures `body(stream, handle)`
// into it on the helper stream `aux`.
template <class F>
zef_status capture_while(zef_ctx *ctx, cudaStream_t cap, cudaStream_t aux, F &&body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &graph, &deps, nullptr, &ndeps), "cudaStreamGetCaptureInfo");
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault), "conditional handle");
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp), "conditional node");
  CK(cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
     "capture dependencies");
  CK(cudaStreamBeginCaptureToGraph(aux, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal),
     "capture loop body");
  body(aux, handle);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(aux, &out);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end of loop body capture");
  return ZEF_OK;
}

}  // namespace

zef_status refine_run(zef_ctx *ctx, zef_mesh *mesh, int32_t levels, const zef_label_opts &opts,
                      zef_level_stats *per_level) {
  NvtxRange nvtx_("zef.refine_and_relabel");
  const int64_t N0 = mesh->num_nodes, M0 = mesh->num_tets;
  const int64_t ncap = mesh->node_capacity, tcap = mesh->tet_capacity;
  const bool dn = device_ptr(mesh->nodes, ctx->device), dt = device_ptr(mesh->tets, ctx->device),
             dl = device_ptr(mesh->node_labels, ctx->device);
  if (!(dn == dt && dt == dl)) return fail(ctx, ZEF_ERR_INVALID_ARG, "mesh arrays must all be host or all device");
  const bool host = !dn;
  const bool conforming = (mesh->flags & ZEF_REFINE_CONFORMING) != 0;
  if (per_level) std::memset(per_level, 0, sizeof(zef_level_stats) * std::max(levels, 0));

  // buffers
  float *nodes = mesh->nodes;
  int32_t *tets = mesh->tets, *labels = mesh->node_labels;
  zef_status st;
  if (host) {
    if ((st = grow(ctx, 5, (size_t)ncap * 3 * sizeof(float)))) return st;
    if ((st = grow(ctx, 6, (size_t)tcap * 4 * sizeof(int32_t)))) return st;
    if ((st = grow(ctx, 7, (size_t)ncap * sizeof(int32_t)))) return st;
    nodes = (float *)ctx->rf_buf[5];
    tets = (int32_t *)ctx->rf_buf[6];
    labels = (int32_t *)ctx->rf_buf[7];
    CK(cudaMemcpyAsync(nodes, mesh->nodes, (size_t)N0 * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
       "copy nodes");
    CK(cudaMemcpyAsync(tets, mesh->tets, (size_t)M0 * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream),
       "copy tets");
    if (mesh->labels_valid)
      CK(cudaMemcpyAsync(labels, mesh->node_labels, (size_t)N0 * sizeof(int32_t), cudaMemcpyHostToDevice,
                         ctx->stream),
         "copy labels");
  } else if ((reinterpret_cast<uintptr_t>(tets) & 15) != 0) {
    return fail(ctx, ZEF_ERR_INVALID_ARG, "device tets must be 16-byte aligned");
  }
  const int64_t fmax = std::max<int64_t>(0, (tcap - M0) / 7);
  int64_t hcap = 1024;
  while (hcap < 12 * fmax) hcap <<= 1;
  const int64_t bs_len = std::max<int64_t>(tcap, 6 * fmax) / 2048 + 2;
  if ((st = grow(ctx, 0, (size_t)std::max<int64_t>(tcap, 1) * sizeof(uint32_t)))) return st;      // flags
  if ((st = grow(ctx, 1, (size_t)std::max<int64_t>(6 * fmax, 1) * sizeof(uint32_t)))) return st;  // owned
  if ((st = grow(ctx, 2, (size_t)hcap * (sizeof(unsigned long long) + 2 * sizeof(uint32_t))))) return st;
  if ((st = grow(ctx, 3, (size_t)bs_len * sizeof(uint32_t)))) return st;
  if ((st = grow(ctx, 4, (size_t)std::max(levels, 1) * kLevelStats * sizeof(int64_t)))) return st;
  if (conforming) {
    if ((st = grow(ctx, 8, (size_t)std::max<int64_t>(tcap, 1)))) return st;                     // state
    if ((st = grow(ctx, 9, (size_t)std::max<int64_t>(tcap, 1) * sizeof(uint32_t)))) return st;  // gx
    static GreenTables gt;
    static bool gt_ready = false;
    if (!gt_ready) {
      green_tables(gt);
      gt_ready = true;
    }
    CK(cudaMemcpyToSymbol(c_gn, gt.n, sizeof(gt.n)), "upload closure table");
    CK(cudaMemcpyToSymbol(c_gch, gt.ch, sizeof(gt.ch)), "upload closure table");
    CK(cudaMemcpyToSymbol(c_gdg, gt.dg, sizeof(gt.dg)), "upload closure table");
  }
  const int64_t new_cap = std::max<int64_t>(1, std::min<int64_t>(6 * fmax, ncap - N0));
  if ((st = label_reserve(ctx, std::max<int64_t>(new_cap, mesh->labels_valid ? 1 : N0)))) return st;
  LabelBuffers &b = ctx->lb;

  LaunchShape shape{256, 2, kernel_variant(opts.kernel)};
  if (opts.precision == ZEF_FP64_PLAIN) shape = LaunchShape{128, 2};
  else if (opts.block_threads) shape = LaunchShape{opts.block_threads, opts.points_per_thread, kernel_variant(opts.kernel)};

  // initial labeling of every node (not graph-captured: host-known count)
  if (!mesh->labels_valid && N0 > 0) {
    LabelPlan p0;
    p0.pts = nodes;
    p0.labels = labels;
    p0.omega = nullptr;
    p0.omega_ld = 0;
    p0.n_cap = N0;
    p0.d_n = b.counters + CNT_N;
    p0.d_off = b.counters + CNT_OFF;
    p0.opts = opts;
    p0.shape = shape;
    p0.timed = false;
    if ((st = label_set_count(ctx, N0, 0))) return st;
    if ((st = label_enqueue(ctx, p0))) return st;
  }

  RF r;
  r.nodes = nodes;
  r.tets = tets;
  r.labels = labels;
  r.cnt = b.counters;
  r.flags = (uint32_t *)ctx->rf_buf[0];
  r.owned = (uint32_t *)ctx->rf_buf[1];
  r.hkeys = (unsigned long long *)ctx->rf_buf[2];
  r.hvals = (uint32_t *)(r.hkeys + hcap);
  r.hids = (int32_t *)(r.hvals + hcap);
  r.hmask = (unsigned long long)(hcap - 1);
  r.node_cap = ncap;
  r.tet_cap = tcap;
  r.fmax = fmax;
  r.status = ctx->d_status;
  r.lstats = (int64_t *)ctx->rf_buf[4];
  r.state = conforming ? (uint8_t *)ctx->rf_buf[8] : nullptr;
  r.gx = conforming ? (uint32_t *)ctx->rf_buf[9] : nullptr;
  uint32_t *bsums = (uint32_t *)ctx->rf_buf[3];

  k_rf_init<<<1, 32, 0, ctx->stream>>>(b.counters, N0, M0);
  CK(cudaGetLastError(), "k_rf_init");

  if (levels > 0) {
    uint64_t key = 0x5eed;
    for (uint64_t v : {(uint64_t)(uintptr_t)nodes, (uint64_t)(uintptr_t)tets, (uint64_t)(uintptr_t)labels,
                       (uint64_t)ncap, (uint64_t)tcap, (uint64_t)fmax, (uint64_t)levels,
                       (uint64_t)(uintptr_t)b.spts, (uint64_t)(uintptr_t)b.flags, (uint64_t)(uintptr_t)b.hist,
                       (uint64_t)(uintptr_t)b.counters, (uint64_t)b.cap_points, (uint64_t)shape.threads,
                       (uint64_t)shape.ppt, (uint64_t)shape.variant, (uint64_t)opts.precision, fbits(opts.margin),
                       fbits(opts.winding_tol), (uint64_t)(uintptr_t)ctx->d_entries, (uint64_t)conforming, ctx->gen,
                       (uint64_t)(uintptr_t)r.state, (uint64_t)(uintptr_t)r.gx})
      key = hash_mix(key, v);
    if (!ctx->rf_exec || ctx->rf_key != key) {
      if (ctx->rf_exec) {
        cudaGraphExecDestroy(ctx->rf_exec);
        ctx->rf_exec = nullptr;
      }
      // capture on a private stream (the caller's may be the legacy default
      // stream, which cannot be captured)
      cudaStream_t cap, aux = nullptr;
      CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate(capture)");
      if (conforming) CK(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking), "cudaStreamCreate(loop body)");
      cudaStream_t user = ctx->stream;
      ctx->stream = cap;
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      st = ZEF_OK;
      if (ce == cudaSuccess) {
        const int g_t = grid_blocks(ctx, tcap, 256);
        for (int lv = 0; lv < levels && st == ZEF_OK; ++lv) {
          k_rf_flag<<<g_t, 256, 0, cap>>>(r);
          if (conforming) {
            // closure: the red set grows until every other tet has a green pattern
            cudaMemsetAsync(r.hkeys, 0xff, (size_t)hcap * sizeof(unsigned long long), cap);
            cudaMemsetAsync(r.hvals, 0xff, (size_t)hcap * sizeof(uint32_t), cap);
            k_cl_reset<<<1, 32, 0, cap>>>(b.counters);
            k_cl_seed<<<g_t, 256, 0, cap>>>(r);
            st = capture_while(ctx, cap, aux, [&](cudaStream_t s, cudaGraphConditionalHandle h) {
              k_cl_insert<<<g_t, 256, 0, s>>>(r);
              k_cl_check<<<g_t, 256, 0, s>>>(r);
              k_cl_next<<<1, 32, 0, s>>>(r, h);
            });
            if (st) break;
            k_cl_red<<<g_t, 256, 0, cap>>>(r);
          }
          st = scan_exclusive(ctx, r.flags, b.counters + CNT_TETS, 1, tcap, b.counters + CNT_LEVEL_FLAGGED, bsums);
          if (st) break;
          k_rf_check<<<1, 32, 0, cap>>>(r);
          if (!conforming) {
            cudaMemsetAsync(r.hkeys, 0xff, (size_t)hcap * sizeof(unsigned long long), cap);
            cudaMemsetAsync(r.hvals, 0xff, (size_t)hcap * sizeof(uint32_t), cap);
          }
          k_rf_insert<<<g_t, 256, 0, cap>>>(r);
          k_rf_owner<<<g_t, 256, 0, cap>>>(r);
          st = scan_exclusive(ctx, r.owned, b.counters + CNT_OWN_LEN, 1, std::max<int64_t>(6 * fmax, 1),
                              b.counters + CNT_LEVEL_NEW, bsums);
          if (st) break;
          k_rf_check2<<<1, 32, 0, cap>>>(r);
          if (conforming) {
            k_cl_gcount<<<g_t, 256, 0, cap>>>(r);
            st = scan_exclusive(ctx, r.gx, b.counters + CNT_TETS, 1, tcap, b.counters + CNT_CL_GEXTRA, bsums);
            if (st) break;
            k_cl_check3<<<1, 32, 0, cap>>>(r);
          }
          k_rf_nodes<<<g_t, 256, 0, cap>>>(r);
          LabelPlan p;
          p.pts = nodes;
          p.labels = labels;
          p.omega = nullptr;
          p.omega_ld = 0;
          p.n_cap = new_cap;
          p.d_n = b.counters + CNT_N;
          p.d_off = b.counters + CNT_OFF;
          p.opts = opts;
          p.shape = shape;
          p.timed = false;
          st = label_enqueue(ctx, p);
          if (st) break;
          k_rf_children<<<g_t, 256, 0, cap>>>(r);
          if (conforming) k_cl_children<<<g_t, 256, 0, cap>>>(r);
          k_rf_advance<<<1, 32, 0, cap>>>(r, lv);
        }
        cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (st == ZEF_OK && ee != cudaSuccess) st = cuda_fail(ctx, ee, "cudaStreamEndCapture");
      } else {
        st = cuda_fail(ctx, ce, "cudaStreamBeginCapture");
      }
      ctx->stream = user;
      cudaStreamDestroy(cap);
      if (aux) cudaStreamDestroy(aux);
      if (st == ZEF_OK) {
        cudaError_t ie = cudaGraphInstantiate(&ctx->rf_exec, graph, 0);
        if (ie != cudaSuccess) st = cuda_fail(ctx, ie, "cudaGraphInstantiate");
        else ctx->rf_key = key;
      }
      if (graph) cudaGraphDestroy(graph);
      if (st) return st;
    }
    CK(cudaGraphLaunch(ctx->rf_exec, ctx->stream), "cudaGraphLaunch");
  }
  // results
  std::vector<int64_t> ls((size_t)std::max(levels, 1) * kLevelStats, 0);
  int64_t cnt[CNT_COUNT_];
  CK(cudaMemcpyAsync(ctx->h_counters, b.counters, CNT_COUNT_ * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
     "read counters");
  if (levels > 0)
    CK(cudaMemcpyAsync(ls.data(), r.lstats, ls.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
       "read level stats");
  st = zef_synchronize(ctx);
  std::memcpy(cnt, ctx->h_counters, sizeof(cnt));
  const int64_t N1 = cnt[CNT_NODES], M1 = cnt[CNT_TETS];
  if (host) {
    CK(cudaMemcpy(mesh->nodes, nodes, (size_t)N1 * 3 * sizeof(float), cudaMemcpyDeviceToHost), "copy nodes back");
    CK(cudaMemcpy(mesh->tets, tets, (size_t)M1 * 4 * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy tets back");
    CK(cudaMemcpy(mesh->node_labels, labels, (size_t)N1 * sizeof(int32_t), cudaMemcpyDeviceToHost),
       "copy labels back");
  }
  mesh->num_nodes = N1;
  mesh->num_tets = M1;
  mesh->labels_valid = 1;
  if (per_level)
    for (int lv = 0; lv < levels; ++lv) {
      const int64_t *s = &ls[(size_t)lv * kLevelStats];
      per_level[lv].new_nodes = s[1];
      per_level[lv].nodes = s[2];
      per_level[lv].tets = s[3];
      per_level[lv].pairs_evaluated = s[4];
      per_level[lv].uncertain_pairs = s[5];
      per_level[lv].flagged_tets = s[7];
      per_level[lv].promoted_tets = s[0] - s[7];
      per_level[lv].green_tets = s[8];
    }
  return st;
}

}  // namespace zef
