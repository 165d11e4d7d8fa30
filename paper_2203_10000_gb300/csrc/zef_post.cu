// zef_post.cu -- post-processing of the labeled mesh (Sec. 2.2): Taubin
// smoothing (Sec. 2.2.1) and inflation towards a compartment surface
// (Sec. 2.2.2).
//
// Both work on the mesh's unique edges, gathered once per call into a CSR
// adjacency: every tet inserts its six edges into an open-addressing table
// (an edge's probe starts in the run of slots of its lower node, so the
// edges of nearby tets, which share nodes with nearby numbers, land in nearby
// slots), the first insertion of a key counts the edge at both nodes, the degrees are
// scanned into row offsets, the table's keys are scattered into the rows and
// each row is sorted, so that every sum over a node's neighbours runs in
// ascending neighbour order (deterministic results).
//
// Smoothing: the iteration loop is one CUDA graph with a conditional
// while-node; its body is the forward step x' = x + lambda L(x), a fixed-order
// reduction of ||x' - x||^2, the backward step x'' = x' - mu L(x'), and a
// one-thread kernel that decides whether to continue, with
// L(x)_i = sum_j (x_j - x_i) / (deg_i + 1) over the edge neighbours j of i
// (node i itself belongs to its neighbourhood and adds nothing to the sum).
//
// Smoothing of the tissue boundaries (surface variant of Sec. 2.2.1): the
// tets' faces go into an open-addressing table keyed by their sorted node
// triple (128-bit compare-and-swap) with the smallest and largest element
// label of the tets that share them; a face whose two labels differ is a
// boundary face, and its three edges build the adjacency of the same
// iteration, so that only the boundary nodes move.
//
// Inflation: the nodes are labeled (inside bits of every compartment); every
// node inside compartment c with an outside neighbour is listed, and one warp
// per listed node intersects each of its crossing edges with c's triangles
// (lanes split the triangles, a warp minimum keeps the intersection nearest
// to the inside node); the node moves by zeta t (x_j - x_i) averaged over its
// crossing edges, t the edge parameter of that intersection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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

constexpr unsigned long long kNoKey = ~0ull;
__constant__ int kEdgeLocal[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
// words of the post-processing statistics (device)
enum PpWord { PP_EDGES = 0, PP_BAD, PP_ITER, PP_STOP, PP_LISTED, PP_FACES, PP_FULL, PP_WORDS };

__device__ __forceinline__ unsigned long long pp_mix(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

struct Adj {
  unsigned long long *keys;  // open-addressing table of edge keys (lo << 32 | hi)
  unsigned long long mask;   // table size - 1
  int shift;                 // log2 of the slots per node (table size >= n << shift)
  uint32_t *deg;             // [n + 1] degrees, scanned into row offsets
  uint32_t *fill;            // [n] scatter cursors
  int32_t *nbr;              // [2 E] neighbours, rows sorted ascending
  int64_t n;
  int64_t *words;            // PpWord
};

// First probe of edge (lo, hi), lo < hi: a slot of lo's run of 2^shift slots,
// picked by a hash of hi (linear probing from there may leave the run).
__device__ __forceinline__ unsigned long long edge_slot(const Adj &g, uint32_t lo, uint32_t hi) {
  return (((unsigned long long)lo << g.shift) | (pp_mix(hi) & ((1ull << g.shift) - 1ull))) & g.mask;
}

// every tet's six edges into the table; the first insertion counts the edge
// in both end nodes' degrees (the edge count is half the degree sum)
__global__ void __launch_bounds__(256) k_pp_edges(Adj g, const int32_t *tets, int64_t m, uint32_t *status) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = tets[4 * t + k];
      bad |= v[k] < 0 || v[k] >= g.n;
    }
    if (bad) {
      atomicOr(status, ST_INVALID);
      atomicExch((unsigned long long *)(g.words + PP_BAD), 1ull);
      continue;
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const uint32_t a = (uint32_t)v[kEdgeLocal[e][0]], b = (uint32_t)v[kEdgeLocal[e][1]];
      if (a == b) continue;
      const unsigned long long key = ((unsigned long long)min(a, b) << 32) | max(a, b);
      unsigned long long h = edge_slot(g, min(a, b), max(a, b));
      for (unsigned long long it = 0; it <= g.mask; ++it) {
        const unsigned long long prev = atomicCAS(g.keys + h, kNoKey, key);
        if (prev == kNoKey) {
          atomicAdd(g.deg + min(a, b), 1u);
          atomicAdd(g.deg + max(a, b), 1u);
          break;
        }
        if (prev == key) break;
        h = (h + 1) & g.mask;
      }
    }
  }
}

// one undirected edge into the table (first insertion counts it at both ends)
__device__ __forceinline__ void insert_edge(const Adj &g, uint32_t a, uint32_t b) {
  if (a == b) return;
  const unsigned long long key = ((unsigned long long)min(a, b) << 32) | max(a, b);
  unsigned long long h = edge_slot(g, min(a, b), max(a, b));
  for (unsigned long long it = 0; it <= g.mask; ++it) {
    const unsigned long long prev = atomicCAS(g.keys + h, kNoKey, key);
    if (prev == kNoKey) {
      atomicAdd(g.deg + min(a, b), 1u);
      atomicAdd(g.deg + max(a, b), 1u);
      return;
    }
    if (prev == key) return;
    h = (h + 1) & g.mask;
  }
  atomicExch((unsigned long long *)(g.words + PP_FULL), 1ull);  // cannot happen at load <= 1/2
}

// ---- tissue-boundary faces
struct FaceTab {
  unsigned long long *keys;  // [2 * (mask + 1)]: (a | b << 32, c) of the sorted triple, all ones when empty
  int32_t *lo, *hi;          // smallest / largest element label of the tets sharing the face
  unsigned long long mask;
};

// 128-bit compare-and-swap (sm_90 and later): returns the previous value
__device__ __forceinline__ void cas128(unsigned long long *p, unsigned long long clo, unsigned long long chi,
                                       unsigned long long vlo, unsigned long long vhi, unsigned long long &olo,
                                       unsigned long long &ohi) {
  asm volatile(
      "{\n\t.reg .b128 d, c, v;\n\tmov.b128 c, {%2, %3};\n\tmov.b128 v, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], c, v;\n\tmov.b128 {%0, %1}, d;\n\t}"
      : "=l"(olo), "=l"(ohi)
      : "l"(clo), "l"(chi), "l"(vlo), "l"(vhi), "l"(p)
      : "memory");
}

__global__ void __launch_bounds__(256) k_sf_clear(FaceTab f) {
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s <= f.mask;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    f.keys[2 * s] = kNoKey;
    f.keys[2 * s + 1] = kNoKey;
    f.lo[s] = INT32_MAX;
    f.hi[s] = INT32_MIN;
  }
}

// every tet's four faces into the table with the tet's element label
__global__ void __launch_bounds__(256) k_sf_faces(FaceTab f, const int32_t *tets, const int32_t *labels, int64_t m,
                                                 int64_t n, int64_t *words, uint32_t *status) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = tets[4 * t + k];
      bad |= v[k] < 0 || v[k] >= n;
    }
    if (bad) {
      atomicOr(status, ST_INVALID);
      atomicExch((unsigned long long *)(words + PP_BAD), 1ull);
      continue;
    }
    const int32_t lab = labels[t];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // face q leaves out vertex 3 - q
      uint32_t a = (uint32_t)v[q == 3 ? 1 : 0], b = (uint32_t)v[q >= 2 ? 2 : 1], c = (uint32_t)v[q >= 1 ? 3 : 2];
      uint32_t lo = min(a, min(b, c)), hi = max(a, max(b, c));
      const uint32_t mid = a ^ b ^ c ^ lo ^ hi;
      a = lo;
      b = mid;
      c = hi;
      const unsigned long long klo = (unsigned long long)a | ((unsigned long long)b << 32), khi = c;
      unsigned long long h = pp_mix(klo ^ pp_mix(khi)) & f.mask;
      bool placed = false;
      for (unsigned long long it = 0; it <= f.mask; ++it) {
        unsigned long long olo, ohi;
        cas128(f.keys + 2 * h, kNoKey, kNoKey, klo, khi, olo, ohi);
        if ((olo == kNoKey && ohi == kNoKey) || (olo == klo && ohi == khi)) {
          atomicMin(f.lo + h, lab);
          atomicMax(f.hi + h, lab);
          placed = true;
          break;
        }
        h = (h + 1) & f.mask;
      }
      if (!placed) atomicExch((unsigned long long *)(words + PP_FULL), 1ull);
    }
  }
}

// the boundary faces (two tets, different labels) and their edges
__global__ void __launch_bounds__(256) k_sf_edges(FaceTab f, Adj g) {
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s <= f.mask;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long klo = f.keys[2 * s];
    if (klo == kNoKey || f.lo[s] == f.hi[s]) continue;
    const uint32_t a = (uint32_t)(klo & 0xffffffffu), b = (uint32_t)(klo >> 32), c = (uint32_t)f.keys[2 * s + 1];
    atomicAdd((unsigned long long *)(g.words + PP_FACES), 1ull);
    insert_edge(g, a, b);
    insert_edge(g, a, c);
    insert_edge(g, b, c);
  }
}

__global__ void __launch_bounds__(256) k_pp_scatter(Adj g) {
  if (g.words[PP_BAD]) return;
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s <= g.mask;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = g.keys[s];
    if (key == kNoKey) continue;
    const uint32_t a = (uint32_t)(key >> 32), b = (uint32_t)(key & 0xffffffffu);
    g.nbr[g.deg[a] + atomicAdd(g.fill + a, 1u)] = (int32_t)b;
    g.nbr[g.deg[b] + atomicAdd(g.fill + b, 1u)] = (int32_t)a;
  }
}

// ascending order inside every row (insertion sort; rows hold a few dozen)
__global__ void __launch_bounds__(256) k_pp_sort_rows(Adj g) {
  if (g.words[PP_BAD]) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t *r = g.nbr + g.deg[i];
    const int cnt = (int)(g.deg[i + 1] - g.deg[i]);
    for (int k = 1; k < cnt; ++k) {
      const int32_t v = r[k];
      int j = k - 1;
      while (j >= 0 && r[j] > v) {
        r[j + 1] = r[j];
        --j;
      }
      r[j + 1] = v;
    }
  }
}

// ---- smoothing
struct Smooth {
  Adj g;
  float *x, *y;            // positions [n][3]: x current, y after the forward step
  const uint8_t *fixed;    // nullable
  float lambda, mu, xi;
  const double *x0;        // ||x^(0)||_2 (device)
  int max_iters;
  double *partial;         // per-block sums of squares of the forward step
  int nblocks;
};

// y = x + lambda L(x) (fixed nodes keep x); block sums of |y - x|^2 in a fixed order
__global__ void __launch_bounds__(256) k_sm_forward(Smooth s) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float xi0 = s.x[3 * i], xi1 = s.x[3 * i + 1], xi2 = s.x[3 * i + 2];
    float o0 = xi0, o1 = xi1, o2 = xi2;
    if (!(s.fixed && s.fixed[i])) {
      const uint32_t b = s.g.deg[i], e = s.g.deg[i + 1];
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      for (uint32_t k = b; k < e; ++k) {
        const int32_t j = s.g.nbr[k];
        a0 += s.x[3 * (int64_t)j] - xi0;
        a1 += s.x[3 * (int64_t)j + 1] - xi1;
        a2 += s.x[3 * (int64_t)j + 2] - xi2;
      }
      const float w = s.lambda / (float)(e - b + 1);
      o0 = fmaf(w, a0, xi0);
      o1 = fmaf(w, a1, xi1);
      o2 = fmaf(w, a2, xi2);
    }
    s.y[3 * i] = o0;
    s.y[3 * i + 1] = o1;
    s.y[3 * i + 2] = o2;
    const double d0 = (double)o0 - xi0, d1 = (double)o1 - xi1, d2 = (double)o2 - xi2;
    acc += d0 * d0 + d1 * d1 + d2 * d2;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) s.partial[blockIdx.x] = red[0];
}

// x = y - mu L(y) (fixed nodes keep y)
__global__ void __launch_bounds__(256) k_sm_backward(Smooth s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float yi0 = s.y[3 * i], yi1 = s.y[3 * i + 1], yi2 = s.y[3 * i + 2];
    float o0 = yi0, o1 = yi1, o2 = yi2;
    if (!(s.fixed && s.fixed[i])) {
      const uint32_t b = s.g.deg[i], e = s.g.deg[i + 1];
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      for (uint32_t k = b; k < e; ++k) {
        const int32_t j = s.g.nbr[k];
        a0 += s.y[3 * (int64_t)j] - yi0;
        a1 += s.y[3 * (int64_t)j + 1] - yi1;
        a2 += s.y[3 * (int64_t)j + 2] - yi2;
      }
      const float w = -s.mu / (float)(e - b + 1);
      o0 = fmaf(w, a0, yi0);
      o1 = fmaf(w, a1, yi1);
      o2 = fmaf(w, a2, yi2);
    }
    s.x[3 * i] = o0;
    s.x[3 * i + 1] = o1;
    s.x[3 * i + 2] = o2;
  }
}

// one thread: the forward step's relative size decides whether to continue
__global__ void k_sm_next(Smooth s, cudaGraphConditionalHandle handle) {
  if (threadIdx.x != 0) return;
  double ss = 0.0;
  for (int b = 0; b < s.nblocks; ++b) ss += s.partial[b];
  const int64_t it = ++s.g.words[PP_ITER];
  const double x0 = *s.x0;
  const bool small = x0 > 0.0 ? sqrt(ss) / x0 <= (double)s.xi : true;
  if (small) s.g.words[PP_STOP] = 1;
  cudaGraphSetConditional(handle, (!small && it < s.max_iters && !s.g.words[PP_BAD]) ? 1u : 0u);
}

// ||x||_2 of the starting positions (with `off`, the CSR row offsets, only of
// the nodes that have a neighbour): block sums in a fixed order, then one
// thread
__global__ void __launch_bounds__(256) k_sm_norm(const float *x, int64_t n, const uint32_t *off, double *partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
    if (!off || off[i / 3 + 1] > off[i / 3]) acc += (double)x[i] * x[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sm_norm_final(const double *partial, int nblocks, double *x0) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[b];
  *x0 = sqrt(s);
}

// listed nodes in index order from their scanned flags
__global__ void __launch_bounds__(256) k_in_list(const uint32_t *off, int64_t n, const int64_t *total, uint32_t *list) {
  const uint32_t tot = (uint32_t)*total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t nx = (i + 1 < n) ? off[i + 1] : tot;
    if (nx != off[i]) list[off[i]] = (uint32_t)i;
  }
}

__global__ void k_pp_words(int64_t *w) {
  if (threadIdx.x < PP_WORDS) w[threadIdx.x] = 0;
}

// ---- inflation
// nodes inside compartment row `row` with a neighbour outside it
__global__ void __launch_bounds__(256) k_in_flag(Adj g, const unsigned long long *mask, int row, uint32_t *flag) {
  const unsigned long long bit = 1ull << row;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t f = 0;
    if (mask[i] & bit)
      for (uint32_t k = g.deg[i]; k < g.deg[i + 1]; ++k)
        if (!(mask[g.nbr[k]] & bit)) {
          f = 1;
          break;
        }
    flag[i] = f;
  }
}

// One warp per listed node: for each crossing edge (ascending neighbour
// order) the nearest intersection with the compartment's triangles
// (Moller-Trumbore in FP32 on the scaled coordinates, inclusive by a
// relative 2^-20 so that an edge through a shared triangle edge still hits),
// then the averaged move.  The candidates are the
// triangles of the cap-tree leaves whose box meets the edge's box grown by
// 2^-10 (lane 0 walks the tree; a triangle the edge meets lies in such a
// leaf, so the minimum is the one over all triangles); more than kInLeaves
// such leaves fall back to every triangle.
constexpr int kInLeaves = 32;

__global__ void __launch_bounds__(256) k_in_move(Adj g, const float *x, float *out, const unsigned long long *mask,
                                                 int row, const uint32_t *pos, const float4 *tris, int tri_cnt,
                                                 const CapNode *nodes, int root, const int32_t *ctidx, float scale,
                                                 float zeta) {
  __shared__ int2 s_leaf[8][kInLeaves];  // per warp: (first position in ctidx, triangles)
  __shared__ int s_nleaf[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t listed = g.words[PP_LISTED];
  const unsigned long long bit = 1ull << row;
  constexpr float kEps = 9.5367431640625e-07f;  // 2^-20
  constexpr float kBoxMargin = 9.765625e-04f;   // 2^-10
  for (int64_t w = warp; w < listed; w += nwarps) {
    const int32_t i = (int32_t)pos[w];
    const float p0 = x[3 * (int64_t)i] * scale, p1 = x[3 * (int64_t)i + 1] * scale, p2 = x[3 * (int64_t)i + 2] * scale;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
    int cnt = 0;
    for (uint32_t k = g.deg[i]; k < g.deg[i + 1]; ++k) {
      const int32_t j = g.nbr[k];
      if (mask[j] & bit) continue;
      const float e0 = x[3 * (int64_t)j] - x[3 * (int64_t)i], e1 = x[3 * (int64_t)j + 1] - x[3 * (int64_t)i + 1],
                  e2 = x[3 * (int64_t)j + 2] - x[3 * (int64_t)i + 2];
      const float d0 = e0 * scale, d1 = e1 * scale, d2 = e2 * scale;
      if (lane == 0) {
        const float lo0 = fminf(p0, p0 + d0) - kBoxMargin, hi0 = fmaxf(p0, p0 + d0) + kBoxMargin;
        const float lo1 = fminf(p1, p1 + d1) - kBoxMargin, hi1 = fmaxf(p1, p1 + d1) + kBoxMargin;
        const float lo2 = fminf(p2, p2 + d2) - kBoxMargin, hi2 = fmaxf(p2, p2 + d2) + kBoxMargin;
        int nl = 0;
        // pre-order walk without a stack: descend to i + 1, or continue at skip
        const int end = nodes[root].skip;
        for (int q = root; q != end;) {
          const CapNode nd = nodes[q];
          if (nd.hi[0] < lo0 || nd.lo[0] > hi0 || nd.hi[1] < lo1 || nd.lo[1] > hi1 || nd.hi[2] < lo2 ||
              nd.lo[2] > hi2) {
            q = nd.skip;
          } else if (nd.left < 0) {
            if (nl < kInLeaves) s_leaf[wid][nl] = make_int2(nd.tri_begin, nd.leaf_tris);
            ++nl;
            q = nd.skip;
          } else {
            ++q;
          }
        }
        s_nleaf[wid] = nl;
      }
      __syncwarp();
      const int nl = s_nleaf[wid];
      const bool all = nl > kInLeaves;
      const int nsrc = all ? 1 : nl;
      float tmin = INFINITY;
      for (int l = 0; l < nsrc; ++l) {
        const int2 L = all ? make_int2(0, tri_cnt) : s_leaf[wid][l];
        for (int q = lane; q < L.y; q += 32) {
          const int t = all ? q : ctidx[L.x + q];
          const float4 A = tris[3 * t], B = tris[3 * t + 1], C = tris[3 * t + 2];
          const float ax = B.x - A.x, ay = B.y - A.y, az = B.z - A.z;   // edge 1
          const float bx = C.x - A.x, by = C.y - A.y, bz = C.z - A.z;   // edge 2
          const float px = d1 * bz - d2 * by, py = d2 * bx - d0 * bz, pz = d0 * by - d1 * bx;
          const float det = ax * px + ay * py + az * pz;
          if (det == 0.f) continue;
          const float inv = 1.f / det;
          const float tx = p0 - A.x, ty = p1 - A.y, tz = p2 - A.z;
          const float u = (tx * px + ty * py + tz * pz) * inv;
          if (u < -kEps || u > 1.f + kEps) continue;
          const float qx = ty * az - tz * ay, qy = tz * ax - tx * az, qz = tx * ay - ty * ax;
          const float v = (d0 * qx + d1 * qy + d2 * qz) * inv;
          if (v < -kEps || u + v > 1.f + kEps) continue;
          const float tt = (bx * qx + by * qy + bz * qz) * inv;
          if (tt >= 0.f && tt <= 1.f + kEps) tmin = fminf(tmin, tt);
        }
      }
      __syncwarp();  // lane 0 rewrites the leaf list for the next edge
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
      if (tmin < INFINITY) {
        const float tc = fminf(tmin, 1.f);
        m0 = fmaf(zeta * tc, e0, m0);
        m1 = fmaf(zeta * tc, e1, m1);
        m2 = fmaf(zeta * tc, e2, m2);
        ++cnt;
      }
    }
    if (lane == 0 && cnt > 0) {
      out[3 * (int64_t)i] = x[3 * (int64_t)i] + m0 / (float)cnt;
      out[3 * (int64_t)i + 1] = x[3 * (int64_t)i + 1] + m1 / (float)cnt;
      out[3 * (int64_t)i + 2] = x[3 * (int64_t)i + 2] + m2 / (float)cnt;
      atomicAdd((unsigned long long *)(g.words + PP_STOP), 1ull);  // moved nodes
    }
  }
}

bool on_dev(const void *p, int device) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

// post-processing scratch: grow-only device buffers of the context
zef_status pp_grow(zef_ctx *ctx, int idx, size_t bytes) {
  if (ctx->pp_buf[idx] && ctx->pp_cap[idx] >= bytes) return ZEF_OK;
  if (ctx->pp_buf[idx]) cudaFree(ctx->pp_buf[idx]);
  ctx->pp_buf[idx] = nullptr;
  ctx->pp_cap[idx] = 0;
  CK(cudaMalloc(&ctx->pp_buf[idx], std::max<size_t>(bytes, 256)), "cudaMalloc(post-processing)");
  ctx->pp_cap[idx] = bytes;
  return ZEF_OK;
}

// log2 of the table slots per node: the largest s with n 2^s <= cap
int slot_shift(int64_t cap, int64_t n) {
  int sh = 0;
  while (sh < 40 && (std::max<int64_t>(n, 1) << (sh + 1)) <= cap) ++sh;
  return sh;
}

// Unique-edge CSR of the tets (buffers 0-4 of pp_buf); synchronizes.
zef_status build_adjacency(zef_ctx *ctx, const int32_t *tets, int64_t m, int64_t n, Adj *out, int64_t *edges) {
  int64_t cap = 1024;
  while (cap < 12 * std::max<int64_t>(m, 1)) cap <<= 1;  // 6 m edge slots, load <= 1/2
  zef_status st;
  if ((st = pp_grow(ctx, 0, (size_t)cap * sizeof(unsigned long long)))) return st;
  if ((st = pp_grow(ctx, 1, (size_t)(n + 1) * sizeof(uint32_t)))) return st;
  if ((st = pp_grow(ctx, 2, (size_t)std::max<int64_t>(n, 1) * sizeof(uint32_t)))) return st;
  if ((st = pp_grow(ctx, 4, (size_t)PP_WORDS * sizeof(int64_t)))) return st;
  if ((st = pp_grow(ctx, 5, (size_t)((n + 1) / 2048 + 2) * sizeof(uint32_t)))) return st;
  Adj g;
  g.keys = (unsigned long long *)ctx->pp_buf[0];
  g.mask = (unsigned long long)(cap - 1);
  g.shift = slot_shift(cap, n);
  g.deg = (uint32_t *)ctx->pp_buf[1];
  g.fill = (uint32_t *)ctx->pp_buf[2];
  g.n = n;
  g.words = (int64_t *)ctx->pp_buf[4];
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(g.keys, 0xff, (size_t)cap * sizeof(unsigned long long), s), "clear edge table");
  CK(cudaMemsetAsync(g.deg, 0, (size_t)(n + 1) * sizeof(uint32_t), s), "clear degrees");
  CK(cudaMemsetAsync(g.fill, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(uint32_t), s), "clear cursors");
  k_pp_words<<<1, 32, 0, s>>>(g.words);
  if (m > 0) k_pp_edges<<<grid_blocks(ctx, m, 256), 256, 0, s>>>(g, tets, m, ctx->d_status);
  st = scan_exclusive(ctx, g.deg, nullptr, 1, n + 1, nullptr, (uint32_t *)ctx->pp_buf[5]);
  if (st) return st;
  int64_t words[PP_WORDS];
  uint32_t deg_sum = 0;  // 2 x edges: the scanned degrees' last entry
  CK(cudaMemcpyAsync(words, g.words, sizeof(words), cudaMemcpyDeviceToHost, s), "read adjacency status");
  CK(cudaMemcpyAsync(&deg_sum, g.deg + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read edge count");
  CK(cudaStreamSynchronize(s), "build adjacency");
  if (words[PP_BAD]) {
    zef_synchronize(ctx);  // clears the recorded status
    return fail(ctx, ZEF_ERR_INVALID_ARG, "a tet references a node index outside [0, num_nodes)");
  }
  *edges = (int64_t)deg_sum / 2;
  if ((st = pp_grow(ctx, 3, (size_t)std::max<int64_t>((int64_t)deg_sum, 1) * sizeof(int32_t)))) return st;
  g.nbr = (int32_t *)ctx->pp_buf[3];
  k_pp_scatter<<<grid_blocks(ctx, cap, 256), 256, 0, s>>>(g);
  k_pp_sort_rows<<<grid_blocks(ctx, n, 256), 256, 0, s>>>(g);
  CK(cudaGetLastError(), "adjacency kernels");
  *out = g;
  return ZEF_OK;
}

}  // namespace

namespace {

// The Taubin iteration loop over the adjacency g (one graph with a
// conditional while-node), on device positions x; with `boundary_norm` the
// starting norm runs over the nodes that have a neighbour.  Writes the
// iterations run; the caller synchronizes and copies back.
zef_status smooth_loop(zef_ctx *ctx, float *x, int64_t n, const Adj &g, const uint8_t *fx, const zef_smooth_opts &o,
                       bool boundary_norm, int64_t *words) {
  cudaStream_t s = ctx->stream;
  zef_status st;
  const int threads = 256;
  const int nblocks = grid_blocks(ctx, 3 * n, threads);
  if ((st = pp_grow(ctx, 9, (size_t)n * 3 * sizeof(float)))) return st;
  if ((st = pp_grow(ctx, 10, (size_t)(nblocks + 1) * sizeof(double)))) return st;
  double *partial = (double *)ctx->pp_buf[10];
  k_sm_norm<<<nblocks, threads, 0, s>>>(x, n, boundary_norm ? g.deg : nullptr, partial);
  k_sm_norm_final<<<1, 32, 0, s>>>(partial, nblocks, partial + nblocks);
  Smooth sm;
  sm.g = g;
  sm.x = x;
  sm.y = (float *)ctx->pp_buf[9];
  sm.fixed = fx;
  sm.lambda = o.lambda;
  sm.mu = o.mu;
  sm.xi = o.xi;
  sm.x0 = partial + nblocks;
  sm.max_iters = o.max_iters;
  sm.partial = partial;
  sm.nblocks = nblocks;
  // the iteration loop: one graph, one conditional while-node (built per call)
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
  cudaGraphExec_t exec = nullptr;
  if (ce == cudaSuccess) {
    cudaStream_t cap;
    ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (ce == cudaSuccess) {
      ce = cudaStreamBeginCaptureToGraph(cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        k_sm_forward<<<nblocks, threads, 0, cap>>>(sm);
        k_sm_backward<<<nblocks, threads, 0, cap>>>(sm);
        k_sm_next<<<1, 32, 0, cap>>>(sm, handle);
        cudaGraph_t body = nullptr;
        ce = cudaStreamEndCapture(cap, &body);
      }
      cudaStreamDestroy(cap);
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
  }
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "smoothing graph");
  ce = cudaGraphLaunch(exec, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(words, g.words, PP_WORDS * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  cudaGraphExecDestroy(exec);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "smoothing");
  return ZEF_OK;
}

// CSR adjacency of the tissue-boundary faces' edges (buffers 0-5 as
// build_adjacency, 14-16 for the face table); synchronizes.
zef_status build_surface_adjacency(zef_ctx *ctx, const int32_t *tets, const int32_t *labels, int64_t m, int64_t n,
                                   Adj *out, int64_t *faces) {
  int64_t fcap = 1024;
  while (fcap < 8 * std::max<int64_t>(m, 1)) fcap <<= 1;  // 4 m face slots, load <= 1/2
  int64_t cap = 1024;
  while (cap < 12 * std::max<int64_t>(m, 1)) cap <<= 1;   // boundary edges: far fewer than the tets' 6 m
  zef_status st;
  if ((st = pp_grow(ctx, 14, (size_t)fcap * 2 * sizeof(unsigned long long)))) return st;
  if ((st = pp_grow(ctx, 15, (size_t)fcap * sizeof(int32_t)))) return st;
  if ((st = pp_grow(ctx, 16, (size_t)fcap * sizeof(int32_t)))) return st;
  if ((st = pp_grow(ctx, 0, (size_t)cap * sizeof(unsigned long long)))) return st;
  if ((st = pp_grow(ctx, 1, (size_t)(n + 1) * sizeof(uint32_t)))) return st;
  if ((st = pp_grow(ctx, 2, (size_t)std::max<int64_t>(n, 1) * sizeof(uint32_t)))) return st;
  if ((st = pp_grow(ctx, 4, (size_t)PP_WORDS * sizeof(int64_t)))) return st;
  if ((st = pp_grow(ctx, 5, (size_t)((n + 1) / 2048 + 2) * sizeof(uint32_t)))) return st;
  FaceTab f;
  f.keys = (unsigned long long *)ctx->pp_buf[14];
  f.lo = (int32_t *)ctx->pp_buf[15];
  f.hi = (int32_t *)ctx->pp_buf[16];
  f.mask = (unsigned long long)(fcap - 1);
  Adj g;
  g.keys = (unsigned long long *)ctx->pp_buf[0];
  g.mask = (unsigned long long)(cap - 1);
  g.shift = slot_shift(cap, n);
  g.deg = (uint32_t *)ctx->pp_buf[1];
  g.fill = (uint32_t *)ctx->pp_buf[2];
  g.n = n;
  g.words = (int64_t *)ctx->pp_buf[4];
  cudaStream_t s = ctx->stream;
  k_sf_clear<<<grid_blocks(ctx, fcap, 256), 256, 0, s>>>(f);
  CK(cudaMemsetAsync(g.keys, 0xff, (size_t)cap * sizeof(unsigned long long), s), "clear edge table");
  CK(cudaMemsetAsync(g.deg, 0, (size_t)(n + 1) * sizeof(uint32_t), s), "clear degrees");
  CK(cudaMemsetAsync(g.fill, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(uint32_t), s), "clear cursors");
  k_pp_words<<<1, 32, 0, s>>>(g.words);
  if (m > 0) {
    k_sf_faces<<<grid_blocks(ctx, m, 256), 256, 0, s>>>(f, tets, labels, m, n, g.words, ctx->d_status);
    k_sf_edges<<<grid_blocks(ctx, fcap, 256), 256, 0, s>>>(f, g);
  }
  st = scan_exclusive(ctx, g.deg, nullptr, 1, n + 1, nullptr, (uint32_t *)ctx->pp_buf[5]);
  if (st) return st;
  int64_t words[PP_WORDS];
  uint32_t deg_sum = 0;
  CK(cudaMemcpyAsync(words, g.words, sizeof(words), cudaMemcpyDeviceToHost, s), "read adjacency status");
  CK(cudaMemcpyAsync(&deg_sum, g.deg + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read edge count");
  CK(cudaStreamSynchronize(s), "build boundary adjacency");
  if (words[PP_BAD]) {
    zef_synchronize(ctx);  // clears the recorded status
    return fail(ctx, ZEF_ERR_INVALID_ARG, "a tet references a node index outside [0, num_nodes)");
  }
  if (words[PP_FULL]) return fail(ctx, ZEF_ERR_CUDA, "internal: face or edge table full");
  *faces = words[PP_FACES];
  if ((st = pp_grow(ctx, 3, (size_t)std::max<int64_t>((int64_t)deg_sum, 1) * sizeof(int32_t)))) return st;
  g.nbr = (int32_t *)ctx->pp_buf[3];
  k_pp_scatter<<<grid_blocks(ctx, cap, 256), 256, 0, s>>>(g);
  k_pp_sort_rows<<<grid_blocks(ctx, n, 256), 256, 0, s>>>(g);
  CK(cudaGetLastError(), "boundary adjacency kernels");
  *out = g;
  return ZEF_OK;
}

}  // namespace

zef_status taubin_run(zef_ctx *ctx, float *nodes, int64_t n, const int32_t *tets, int64_t m, const uint8_t *fixed,
                      const zef_smooth_opts &o, int32_t *iters_out) {
  NvtxRange nvtx_("zef.taubin_smooth");
  const bool dn = on_dev(nodes, ctx->device);
  const bool dt = m == 0 ? dn : on_dev(tets, ctx->device);
  const bool df = fixed ? on_dev(fixed, ctx->device) : dn;
  if (!(dn == dt && dt == df)) return fail(ctx, ZEF_ERR_INVALID_ARG, "nodes, tets and fixed must all be host or all device");
  zef_status st;
  float *x = nodes;
  const int32_t *tt = tets;
  const uint8_t *fx = fixed;
  cudaStream_t s = ctx->stream;
  if (!dn) {  // stage host arrays (buffers 6: nodes, 7: tets, 8: fixed)
    if ((st = pp_grow(ctx, 6, (size_t)n * 3 * sizeof(float)))) return st;
    if ((st = pp_grow(ctx, 7, (size_t)std::max<int64_t>(m, 1) * 4 * sizeof(int32_t)))) return st;
    x = (float *)ctx->pp_buf[6];
    tt = (const int32_t *)ctx->pp_buf[7];
    CK(cudaMemcpyAsync(x, nodes, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s), "copy nodes");
    if (m > 0) CK(cudaMemcpyAsync((void *)tt, tets, (size_t)m * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy tets");
    if (fixed) {
      if ((st = pp_grow(ctx, 8, (size_t)n))) return st;
      fx = (const uint8_t *)ctx->pp_buf[8];
      CK(cudaMemcpyAsync((void *)fx, fixed, (size_t)n, cudaMemcpyHostToDevice, s), "copy fixed");
    }
  }
  Adj g;
  int64_t edges = 0;
  if ((st = build_adjacency(ctx, tt, m, n, &g, &edges))) return st;  // synchronizes
  int64_t words[PP_WORDS] = {0};
  if ((st = smooth_loop(ctx, x, n, g, fx, o, false, words))) return st;
  if (!dn) CK(cudaMemcpy(nodes, x, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost), "copy nodes back");
  if (iters_out) *iters_out = (int32_t)words[PP_ITER];
  return zef_synchronize(ctx);
}

zef_status taubin_surface_run(zef_ctx *ctx, float *nodes, int64_t n, const int32_t *tets, int64_t m,
                              const int32_t *elem_labels, const zef_smooth_opts &o, int32_t *iters_out,
                              int64_t *faces_out) {
  NvtxRange nvtx_("zef.taubin_smooth_surface");
  const bool dn = on_dev(nodes, ctx->device);
  const bool dt = m == 0 ? dn : on_dev(tets, ctx->device);
  const bool dl = m == 0 ? dn : on_dev(elem_labels, ctx->device);
  if (!(dn == dt && dt == dl))
    return fail(ctx, ZEF_ERR_INVALID_ARG, "nodes, tets and elem_labels must all be host or all device");
  zef_status st;
  float *x = nodes;
  const int32_t *tt = tets;
  const int32_t *lab = elem_labels;
  cudaStream_t s = ctx->stream;
  if (!dn) {  // stage host arrays (buffers 6: nodes, 7: tets, 17: labels)
    if ((st = pp_grow(ctx, 6, (size_t)n * 3 * sizeof(float)))) return st;
    if ((st = pp_grow(ctx, 7, (size_t)std::max<int64_t>(m, 1) * 4 * sizeof(int32_t)))) return st;
    if ((st = pp_grow(ctx, 17, (size_t)std::max<int64_t>(m, 1) * sizeof(int32_t)))) return st;
    x = (float *)ctx->pp_buf[6];
    tt = (const int32_t *)ctx->pp_buf[7];
    lab = (const int32_t *)ctx->pp_buf[17];
    CK(cudaMemcpyAsync(x, nodes, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s), "copy nodes");
    if (m > 0) {
      CK(cudaMemcpyAsync((void *)tt, tets, (size_t)m * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy tets");
      CK(cudaMemcpyAsync((void *)lab, elem_labels, (size_t)m * sizeof(int32_t), cudaMemcpyHostToDevice, s),
         "copy labels");
    }
  }
  Adj g;
  int64_t faces = 0;
  if ((st = build_surface_adjacency(ctx, tt, lab, m, n, &g, &faces))) return st;  // synchronizes
  int64_t words[PP_WORDS] = {0};
  if (faces > 0 && (st = smooth_loop(ctx, x, n, g, nullptr, o, true, words))) return st;
  if (!dn) CK(cudaMemcpy(nodes, x, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost), "copy nodes back");
  if (iters_out) *iters_out = (int32_t)words[PP_ITER];
  if (faces_out) *faces_out = faces;
  return zef_synchronize(ctx);
}

zef_status inflate_run(zef_ctx *ctx, float *nodes, int64_t n, const int32_t *tets, int64_t m, int32_t id,
                       float zeta, int64_t *moved_out) {
  NvtxRange nvtx_("zef.inflate");
  int row = -1, ci = -1;
  for (size_t r = 0; r < ctx->priority.size(); ++r)
    if (ctx->priority[r] == id) row = (int)r;
  for (size_t c = 0; c < ctx->comps.size(); ++c)
    if (ctx->comps[c].id == id) ci = (int)c;
  if (row < 0 || ci < 0) return fail(ctx, ZEF_ERR_INVALID_ARG, "unknown compartment id");
  const bool dn = on_dev(nodes, ctx->device);
  const bool dt = m == 0 ? dn : on_dev(tets, ctx->device);
  if (dn != dt) return fail(ctx, ZEF_ERR_INVALID_ARG, "nodes and tets must both be host or both device");
  zef_status st;
  float *x = nodes;
  const int32_t *tt = tets;
  cudaStream_t s = ctx->stream;
  if (!dn) {
    if ((st = pp_grow(ctx, 6, (size_t)n * 3 * sizeof(float)))) return st;
    if ((st = pp_grow(ctx, 7, (size_t)std::max<int64_t>(m, 1) * 4 * sizeof(int32_t)))) return st;
    x = (float *)ctx->pp_buf[6];
    tt = (const int32_t *)ctx->pp_buf[7];
    CK(cudaMemcpyAsync(x, nodes, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s), "copy nodes");
    if (m > 0) CK(cudaMemcpyAsync((void *)tt, tets, (size_t)m * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy tets");
  }
  // inside bits of every node (every compartment decided)
  if ((st = pp_grow(ctx, 11, (size_t)n * sizeof(unsigned long long)))) return st;
  if ((st = pp_grow(ctx, 12, (size_t)n * sizeof(int32_t)))) return st;
  unsigned long long *mask = (unsigned long long *)ctx->pp_buf[11];
  st = label_points_impl(ctx, x, n, (int32_t *)ctx->pp_buf[12], nullptr, nullptr, nullptr, mask, true);
  if (st) return st;
  Adj g;
  int64_t edges = 0;
  if ((st = build_adjacency(ctx, tt, m, n, &g, &edges))) return st;
  // nodes inside with an outside neighbour, listed in index order
  if ((st = pp_grow(ctx, 13, (size_t)(n + 1) * sizeof(uint32_t)))) return st;
  if ((st = pp_grow(ctx, 9, (size_t)n * 3 * sizeof(float)))) return st;
  uint32_t *flag = (uint32_t *)ctx->pp_buf[13];
  uint32_t *list = (uint32_t *)ctx->pp_buf[2];  // the scatter cursors are free again
  float *out = (float *)ctx->pp_buf[9];
  k_in_flag<<<grid_blocks(ctx, n, 256), 256, 0, s>>>(g, mask, row, flag);
  st = scan_exclusive(ctx, flag, nullptr, 1, n, g.words + PP_LISTED, (uint32_t *)ctx->pp_buf[5]);
  if (st) return st;
  k_in_list<<<grid_blocks(ctx, n, 256), 256, 0, s>>>(flag, n, g.words + PP_LISTED, list);
  CK(cudaMemcpyAsync(out, x, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy positions");
  CK(cudaMemsetAsync(g.words + PP_STOP, 0, sizeof(int64_t), s), "clear moved count");
  const CompHost &c = ctx->comps[(size_t)ci];
  // one warp per listed node; the grid covers the node count at most
  k_in_move<<<grid_blocks(ctx, n * 32, 256), 256, 0, s>>>(g, x, out, mask, row, list, ctx->d_tris + c.tri_off * 3,
                                                          (int)c.nt, ctx->d_nodes, c.cap_root, ctx->d_ctidx,
                                                          ctx->scale, zeta);
  CK(cudaGetLastError(), "k_in_move");
  int64_t words[PP_WORDS];
  CK(cudaMemcpyAsync(x, out, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, s), "write positions");
  if (!dn) CK(cudaMemcpyAsync(nodes, x, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s), "copy nodes back");
  CK(cudaMemcpyAsync(words, g.words, sizeof(words), cudaMemcpyDeviceToHost, s), "read moved count");
  CK(cudaStreamSynchronize(s), "inflation");
  if (moved_out) *moved_out = words[PP_STOP];
  return zef_synchronize(ctx);
}

}  // namespace zef
