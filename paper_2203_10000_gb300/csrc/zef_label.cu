// Labeling kernels of libzef (sm_103a).
//
// Method (Sec. 2.1.3, Eq. 1 and Sec. 2.1): Omega(p) = sum over the triangles
// of a closed compartment surface of the Van Oosterom-Strackee solid angle
// Omega_t = 2 atan2(N, D); p is inside when Omega > 2 pi; the first
// compartment of the priority list that encloses p labels it.
//
// Pipeline of one call (all on the context stream, no host round trip):
//   k_prepare      point count and offset of this call
//   k_reset        counters, work histogram, split-pair completion counts
//   k_keys         binning key of every point: its 21-bit Morton cell in the
//                  union box of the surfaces, or the tail keys of the points
//                  outside that box (outside every compartment: winding
//                  number 0) and of the non-finite points, which it labels
//                  at once; key histogram
//   scan           exclusive scan of the histogram (records where the tails
//                  start and the tile count)
//   k_scatter      the points inside the union box into key order (float4,
//                  scaled) + permutation
//   k_tile_work/k_scan_work/k_tile_scatter
//                  work list of the tiles of sorted points inside the union
//                  box whose box meets some compartment's box and convex-hull
//                  bound, largest estimated work first; a point outside a
//                  closed surface's box or hull has winding number 0, so the
//                  culling is exact (k_tile_box/k_flags/scan/k_emit: the
//                  (tile, compartment) items of the plain FP64 kernel)
//   k_label32      persistent FP32 kernel over the work list (hot loop); the
//                  default form walks each compartment's cap tree for the
//                  tile (far patches replaced by their caps, zef_tree.cpp) and
//                  appends the uncertain (point, compartment) pairs to a list
//   k_rescue64_list (cap-tree form; k_rescue64_caps when the pair list
//                  overflowed) / k_rescue64 (strip forms)
//                  FP64 re-evaluation of the uncertain pairs
//   k_resolve      priority resolve + un-permute of the sorted points
//
// FP32 hot loop.  Surfaces (whole, or the leaves and caps a tile's walk of the
// cap tree lists) are stored as triangle strips (one new vertex per
// triangle), staged into shared memory by 1-D bulk TMA copies
// (cp.async.bulk + mbarrier, double buffered) and broadcast to every thread;
// each thread holds P points in registers.  (The tile representatives' passes
// split the entries over the lanes instead and read them through the
// read-only cache.)  With the window (a, b, c) of the
// strip and R_k = v_k - p:
//     N = R_c . n            (n = (v2 - v1) x (v3 - v1) of the triangle, host
//                             precomputed in FP64; equal to R1 . (R2 x R3))
//     D = r_a r_b r_c + (R_a . R_b) r_c + (R_a . R_c) r_b + (R_b . R_c) r_a
// where R_a, R_b, r_a, r_b and r_a r_b + R_a . R_b are carried from the two
// previous strip steps.  The (D + iN) factors of four consecutive steps are
// multiplied with their 2 pi wraps counted exactly and one atan2 is taken of
// the product (a range-reduced minimax polynomial, see half_angle).  Omega
// is accumulated plainly over groups of 16 entries and the group sums are
// combined with Kahan compensation.
//
// A (point, compartment) pair is sent to the FP64 re-evaluation when
//   |Omega32 - 2 pi| < margin                (the stated margin), or
//   Omega32 is farther than winding_tol (1e-4) from 4 pi Z (the closed-surface
//      invariant; catches FP32 errors of any size except near 4 pi k), or
//   some triangle had max(|N|, D) < kappa |n| r_c: the point lies within a
//      relative distance kappa of that triangle's plane in a position where
//      the sign of N decides the branch of atan2 (an FP32 sign error there
//      changes Omega by almost 4 pi), or the sum is not finite.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "zef_internal.h"

namespace zef {

namespace {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInvTwoPi = 0.159154943091895335769f;
constexpr float kFourPi = 12.5663706143591729539f;

// atan(x) = x (1 + s P(s)), s = x^2, 0 <= x <= 1: minimax fit of the relative
// error with the constant term held at 1 (max relative error 1.9e-8),
// produced by fit_atan.py in this directory.
constexpr float kA1 = -0.333331669656756f;
constexpr float kA2 = 0.19994137196256442f;
constexpr float kA3 = -0.14214209059340627f;
constexpr float kA4 = 0.10678939968964535f;
constexpr float kA5 = -0.07580577411750086f;
constexpr float kA6 = 0.043553530224279755f;
constexpr float kA7 = -0.0165811779740931f;
constexpr float kA8 = 0.0029745887848576756f;

// directions of the convex-hull bound (uploaded once per device): constant
// memory for loops whose lanes read the same direction, a global copy (read
// through the L1) for the warp-split test, whose lanes read different ones
__constant__ float c_dop[kDop][3];
__device__ float g_dop[kDop][3];

constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded mbarrier wait: 2 s

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One elected thread: arm the barrier with the byte count and start the copy.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Arm the barrier with the byte count of several copies (one arrival) ...
__device__ __forceinline__ void tma_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// ... then start each of them.
__device__ __forceinline__ void tma_copy_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}

__device__ __forceinline__ uint32_t spread7(uint32_t v) {
  // 7 bits -> every third bit
  v &= 0x7f;
  v = (v | (v << 8)) & 0x0000f00f;
  v = (v | (v << 4)) & 0x000c30c3;
  v = (v | (v << 2)) & 0x00249249;
  return v;
}

__device__ void record_timeout(uint32_t *status, uint32_t site) {
  atomicOr(status, ST_TIMEOUT);
  atomicExch(status + 1, site);
}

// ------------------------------------------------------------------ FP32 atan2 / 2
// |v| from |v|^2: the square root instruction runs on the MUFU pipe, off the
// FMA pipe that bounds the strip loop (q rsqrt(q) would add a multiply there)
__device__ __forceinline__ float sqrt_mufu(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// atan2(N, D) in [-pi, pi]: x = min/max(|N|, |D|) in [0, 1], the polynomial
// above, then the octant reflections x -> pi/2 - x (|N| > |D|), x -> pi - x
// (D < 0) and the sign of N.  Measured maximum error 2.6 ulp (CUDA documents
// 3 ulp for atan2f).  N = D = 0 (and infinite operands) give NaN, which the
// label kernel treats as an uncertain sum.
__device__ __forceinline__ float half_angle(float N, float D) {
  const float aN = fabsf(N), aD = fabsf(D);
  const float mn = fminf(aN, aD), mx = fmaxf(aN, aD);
  const float x = __fdividef(mn, mx);
  const float s = x * x;
  float p = kA8;
  p = fmaf(p, s, kA7);
  p = fmaf(p, s, kA6);
  p = fmaf(p, s, kA5);
  p = fmaf(p, s, kA4);
  p = fmaf(p, s, kA3);
  p = fmaf(p, s, kA2);
  p = fmaf(p, s, kA1);
  float a = fmaf(x * s, p, x);
  a = (aN > aD) ? (kHalfPi - a) : a;
  a = (D < 0.f) ? (kPi - a) : a;
  return copysignf(a, N);
}

struct PState {
  float px, py, pz;        // the point
  float ax, ay, az;        // R_a
  float bx, by, bz;        // R_b
  float ra, rb, sab;       // |R_a|, |R_b|, r_a r_b + R_a . R_b
  float grp, sum, comp;    // group sum, Kahan sum and compensation (half angles)
  float bad;               // min over triangles of max(|N|, D) - kappa |n| r_c
  uint32_t kp, kn;         // +2 pi / -2 pi wraps of the grouped complex products
};

__device__ __forceinline__ void window_init(PState &s, float4 v0) {
  s.ax = s.bx = v0.x - s.px;
  s.ay = s.by = v0.y - s.py;
  s.az = s.bz = v0.z - s.pz;
  float q = fmaf(s.ax, s.ax, fmaf(s.ay, s.ay, s.az * s.az));
  float r = sqrt_mufu(q);
  s.ra = s.rb = r;
  s.sab = 2.f * q;
}

__device__ __forceinline__ void vos_step(PState &s, const float4 V, const float4 Nn) {
  const float cx = V.x - s.px, cy = V.y - s.py, cz = V.z - s.pz;
  const float qc = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  const float rc = sqrt_mufu(qc);
  const float dac = fmaf(s.ax, cx, fmaf(s.ay, cy, s.az * cz));
  const float dbc = fmaf(s.bx, cx, fmaf(s.by, cy, s.bz * cz));
  const float N = fmaf(Nn.x, cx, fmaf(Nn.y, cy, Nn.z * cz));
  const float D = fmaf(s.sab, rc, fmaf(dac, s.rb, dbc * s.ra));
  const float t = half_angle(N, D);
  s.grp = fmaf(fabsf(V.w), t, s.grp);  // |w| = 1 on triangles, 0 elsewhere
  s.bad = fminf(s.bad, fmaf(-Nn.w, rc, fmaxf(fabsf(N), D)));
  s.sab = fmaf(s.rb, rc, dbc);
  s.ax = s.bx; s.ay = s.by; s.az = s.bz;
  s.bx = cx; s.by = cy; s.bz = cz;
  s.ra = s.rb;
  s.rb = rc;
}

// Geometry of one strip step: (N, D) of the window (a, b, c) and the
// conditioning minimum; the angle is left to the caller.
__device__ __forceinline__ void geom_step(PState &s, const float4 V, const float4 Nn, float &N, float &D) {
  const float cx = V.x - s.px, cy = V.y - s.py, cz = V.z - s.pz;
  const float qc = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  const float rc = sqrt_mufu(qc);
  const float dac = fmaf(s.ax, cx, fmaf(s.ay, cy, s.az * cz));
  const float dbc = fmaf(s.bx, cx, fmaf(s.by, cy, s.bz * cz));
  N = fmaf(Nn.x, cx, fmaf(Nn.y, cy, Nn.z * cz));
  D = fmaf(s.sab, rc, fmaf(dac, s.rb, dbc * s.ra));
  s.bad = fminf(s.bad, fmaf(-Nn.w, rc, fmaxf(fabsf(N), D)));
  s.sab = fmaf(s.rb, rc, dbc);
  s.ax = s.bx; s.ay = s.by; s.az = s.bz;
  s.bx = cx; s.by = cy; s.bz = cz;
  s.ra = s.rb;
  s.rb = rc;
}

// (cr, ci) = (ar + i ai)(br + i bi); the principal argument of the product
// loses 2 pi when both factors lie in the upper half plane (sign bits of ai
// and bi clear) and the product falls in the lower one, and gains 2 pi in the
// mirrored case: kp / kn count those wraps (IEEE signed zeros keep +-0 and
// +-pi consistent with atan2).
__device__ __forceinline__ void cmul_wrap(float ar, float ai, float br, float bi, float &cr, float &ci,
                                          uint32_t &kp, uint32_t &kn) {
  cr = fmaf(ar, br, -(ai * bi));
  ci = fmaf(ar, bi, ai * br);
  const uint32_t x = __float_as_uint(ai), y = __float_as_uint(bi), z = __float_as_uint(ci);
  kp += (~x & ~y & z) >> 31;
  kn += (x & y & ~z) >> 31;
}

__device__ __forceinline__ void kahan_flush(PState &s) {
  const float y = s.grp - s.comp;
  const float t = s.sum + y;
  s.comp = (t - s.sum) - y;
  s.sum = t;
  s.grp = 0.f;
}

// ------------------------------------------------------------------ two points per instruction
// sm_100 and later execute packed f32x2 add / mul / fma: one instruction does
// the IEEE fp32 operation (same rounding, flush to zero as the rest of this
// file) on two values, so the strip arithmetic of a lane's two points takes
// half the issue slots of two scalar streams.  A pair lives in one 64-bit
// register pair; lo() and hi() are its halves.
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo(f2 a) { return __uint_as_float((uint32_t)a.v); }
__device__ __forceinline__ float hi(f2 a) { return __uint_as_float((uint32_t)(a.v >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// The strip state of a lane's two points (PState, each field a pair).
struct PState2 {
  f2 px, py, pz;
  f2 ax, ay, az, bx, by, bz;
  f2 ra, rb, sab;
  float bad0, bad1;
};

__device__ __forceinline__ void window_init2(PState2 &s, float4 v0) {
  const f2 vx = pk(v0.x, v0.x), vy = pk(v0.y, v0.y), vz = pk(v0.z, v0.z);
  s.ax = s.bx = sub2(vx, s.px);
  s.ay = s.by = sub2(vy, s.py);
  s.az = s.bz = sub2(vz, s.pz);
  const f2 q = fma2(s.ax, s.ax, fma2(s.ay, s.ay, mul2(s.az, s.az)));
  const f2 r = pk(sqrt_mufu(lo(q)), sqrt_mufu(hi(q)));
  s.ra = s.rb = r;
  s.sab = add2(q, q);
}

// geom_step for both points: the same operations in the same order
__device__ __forceinline__ void geom_step2(PState2 &s, const float4 V, const float4 Nn, f2 &N, f2 &D) {
  const f2 cx = sub2(pk(V.x, V.x), s.px), cy = sub2(pk(V.y, V.y), s.py), cz = sub2(pk(V.z, V.z), s.pz);
  const f2 qc = fma2(cx, cx, fma2(cy, cy, mul2(cz, cz)));
  const f2 rc = pk(sqrt_mufu(lo(qc)), sqrt_mufu(hi(qc)));
  const f2 dac = fma2(s.ax, cx, fma2(s.ay, cy, mul2(s.az, cz)));
  const f2 dbc = fma2(s.bx, cx, fma2(s.by, cy, mul2(s.bz, cz)));
  N = fma2(pk(Nn.x, Nn.x), cx, fma2(pk(Nn.y, Nn.y), cy, mul2(pk(Nn.z, Nn.z), cz)));
  D = fma2(s.sab, rc, fma2(dac, s.rb, mul2(dbc, s.ra)));
  s.bad0 = fminf(s.bad0, fmaf(-Nn.w, lo(rc), fmaxf(fabsf(lo(N)), lo(D))));
  s.bad1 = fminf(s.bad1, fmaf(-Nn.w, hi(rc), fmaxf(fabsf(hi(N)), hi(D))));
  s.sab = fma2(s.rb, rc, dbc);
  s.ax = s.bx; s.ay = s.by; s.az = s.bz;
  s.bx = cx; s.by = cy; s.bz = cz;
  s.ra = s.rb;
  s.rb = rc;
}

// cmul_wrap for both points.  The real part a_r b_r - a_i b_i takes the
// product a_i b_i, negated (0 - x: exact; only the sign of a zero can
// differ from the scalar form, which neither the wraps nor the atan2 read),
// into one fused multiply-add, as the scalar form does.
__device__ __forceinline__ void cmul_wrap2(f2 ar, f2 ai, f2 br, f2 bi, f2 &cr, f2 &ci, uint32_t &kp0, uint32_t &kn0,
                                           uint32_t &kp1, uint32_t &kn1) {
  cr = fma2(ar, br, sub2(pk(0.f, 0.f), mul2(ai, bi)));
  ci = fma2(ar, bi, mul2(ai, br));
  const uint32_t x0 = __float_as_uint(lo(ai)), y0 = __float_as_uint(lo(bi)), z0 = __float_as_uint(lo(ci));
  const uint32_t x1 = __float_as_uint(hi(ai)), y1 = __float_as_uint(hi(bi)), z1 = __float_as_uint(hi(ci));
  kp0 += (~x0 & ~y0 & z0) >> 31;
  kn0 += (x0 & y0 & ~z0) >> 31;
  kp1 += (~x1 & ~y1 & z1) >> 31;
  kn1 += (x1 & y1 & ~z1) >> 31;
}

struct LabelArgs {
  const Entry *entries;
  const float4 *tris;
  const DevComp *comps;
  const float4 *spts;
  const int32_t *perm;
  const int2 *items;
  const float *tile_box;
  const float *dop;  // [C][kDop] hull bounds
  unsigned long long *in_mask;
  unsigned long long *unc_mask;
  float *omega;
  int64_t omega_ld;
  int64_t *counters;
  uint32_t *status;
  float margin;
  float winding_tol;
  int ncomp;
  int fp32_only;
  int coherence;  // tile representatives allowed
  int early;      // priority early exit: a point certainly inside needs no later compartment
  int lane_walk;  // kernel form 2 (cap trees): 0 = every point walks the tree for itself
  int omega_raw;  // diagnostics: certified pairs report their FP32 sum, not 4 pi k
  unsigned long long *masks_out;  // nullable: inside bits per point in the caller's order
  const CapNode *nodes;  // cap trees
  const Entry *cseg;     // cap-tree strip segments
  int2 *unc_list;        // uncertain (sorted point, row) pairs of the cap-tree re-evaluation
  int64_t unc_cap;
  double *unc_part;      // [kSplitPairs][kMaxParts] partial half-angle sums of split pairs
  uint32_t *unc_done;    // [kSplitPairs] parts finished
  int64_t n_nodes;       // cap-tree nodes and segment entries (debug-build index checks)
  int64_t n_cseg;
};

// True when the box b (lo x, y, z, hi x, y, z) misses the compartment's box.
__device__ __forceinline__ bool box_misses(const float *b, const DevComp *cp) {
  return b[3] < __ldg(&cp->lo[0]) || b[0] > __ldg(&cp->hi[0]) || b[4] < __ldg(&cp->lo[1]) ||
         b[1] > __ldg(&cp->hi[1]) || b[5] < __ldg(&cp->lo[2]) || b[2] > __ldg(&cp->hi[2]);
}

// Convex-hull bound (kDop half-spaces d_k . x <= thr_k, thr from the host with
// a conservative margin).  A box lies outside when its smallest d_k . x,
// taken at the corner (d_k >= 0 ? lo : hi), exceeds one bound; the winding
// number of every point in it is then 0.
__device__ __forceinline__ bool dop_box_misses(const float *b, const float *thr) {
#pragma unroll 4
  for (int k = 0; k < kDop; ++k) {
    const float dx = c_dop[k][0], dy = c_dop[k][1], dz = c_dop[k][2];
    const float t = fmaf(dx, dx >= 0.f ? b[0] : b[3], fmaf(dy, dy >= 0.f ? b[1] : b[4], dz * (dz >= 0.f ? b[2] : b[5])));
    if (t > __ldg(thr + k)) return true;
  }
  return false;
}

// The same test with the directions split over the lanes of a warp (three
// per lane); every lane of the warp must call it with the same box.
__device__ __forceinline__ bool dop_box_misses_warp(const float *b, const float *thr, int lane) {
  bool miss = false;
#pragma unroll
  for (int k = lane; k < kDop; k += 32) {
    const float dx = __ldg(&g_dop[k][0]), dy = __ldg(&g_dop[k][1]), dz = __ldg(&g_dop[k][2]);
    const float t = fmaf(dx, dx >= 0.f ? b[0] : b[3], fmaf(dy, dy >= 0.f ? b[1] : b[4], dz * (dz >= 0.f ? b[2] : b[5])));
    miss |= t > __ldg(thr + k);
  }
  return __any_sync(0xffffffffu, miss);
}
static_assert(kDop % 32 == 0, "whole directions per lane");

__device__ __forceinline__ bool dop_point_outside(float x, float y, float z, const float *thr) {
#pragma unroll 4
  for (int k = 0; k < kDop; ++k)
    if (fmaf(c_dop[k][0], x, fmaf(c_dop[k][1], y, c_dop[k][2] * z)) > __ldg(thr + k)) return true;
  return false;
}

// Classification of one (point, compartment) pair after the FP32 sum:
// Omega / 2 = half + 2 pi K (K the net count of 2 pi wraps).  Returns true
// when the point is certainly inside the compartment.
__device__ __forceinline__ bool classify_store(const LabelArgs &a, const DevComp &c, const float *thr, int64_t i,
                                               float px, float py, float pz, float half, int K, float bad) {
  if (!ZEF_BOUNDS_OK(i >= 0 && i < a.counters[CNT_NIN], a.status, 14)) return false;
  float omega = 2.f * fmaf(kTwoPi, (float)K, half);
  bool inside = false;
  const unsigned long long bit = 1ull << c.row;
  if (!finite3(px, py, pz)) {
    omega = __int_as_float(0x7fc00000);
  } else {
    // distance of Omega to 4 pi Z, from the small half angle (K drops out)
    const float k = rintf(half * kInvTwoPi);
    const float dist = 2.f * fabsf(fmaf(-kTwoPi, k, half));
    const bool unc = !(bad > 0.f) || !(dist <= a.winding_tol) || !(fabsf(omega - kTwoPi) >= a.margin);
    if (unc && (px < c.lo[0] || px > c.hi[0] || py < c.lo[1] || py > c.hi[1] || pz < c.lo[2] ||
                pz > c.hi[2] || dop_point_outside(px, py, pz, thr))) {
      // outside the box or the hull bound the winding number is 0 whatever
      // the sum says: Omega is exactly 0 (tested only here, where it decides)
      omega = 0.f;
    } else if (unc && !a.fp32_only) {
      atomicOr(a.unc_mask + i, bit);
      if (a.unc_list) {  // the cap-tree re-evaluation's pair list (may overflow: counted beyond its capacity)
        const unsigned long long slot = atomicAdd((unsigned long long *)(a.counters + CNT_UNC_LIST), 1ull);
        if ((int64_t)slot < a.unc_cap) a.unc_list[slot] = make_int2((int)i, c.row);
      }
    } else {
      // a certified winding number K + k: Omega is exactly 4 pi (K + k)
      if (!unc && !a.omega_raw) omega = kFourPi * ((float)K + k);
      if (omega > kTwoPi) {
        atomicOr(a.in_mask + i, bit);
        inside = true;
      }
    }
  }
  if (a.omega) a.omega[(int64_t)c.row * a.omega_ld + a.perm[i]] = omega;
  return inside;
}

// Classification of a point of a coherent tile or group: Omega = 4 pi k
// exactly, k the winding number of the tile's or group's representative.  No
// triangle of the surface meets the box of those points, so the winding
// number is k at every one of them -- 0 in particular wherever a point lies
// outside the compartment's box or hull, which therefore needs no test here.
__device__ __forceinline__ bool classify_coherent(const LabelArgs &a, const DevComp &c, int64_t i, float px,
                                                  float py, float pz, int k) {
  if (!ZEF_BOUNDS_OK(i >= 0 && i < a.counters[CNT_NIN], a.status, 15)) return false;
  float omega;
  bool inside = false;
  if (!finite3(px, py, pz)) {
    omega = __int_as_float(0x7fc00000);
  } else {
    omega = kFourPi * (float)k;
    if (k >= 1) {
      atomicOr(a.in_mask + i, 1ull << c.row);
      inside = true;
    }
  }
  if (a.omega) a.omega[(int64_t)c.row * a.omega_ld + a.perm[i]] = omega;
  return inside;
}

// (s, e) += (b, f): compensated sum of two (value, error) pairs (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float &s, float &e, float b, float f) {
  const float t = s + b;
  const float bb = t - s;
  const float err = (s - (t - bb)) + (b - bb);
  s = t;
  e = e + f + err;
}

// Plain FP32 Van Oosterom-Strackee half angle of triangle (A, B, C) seen
// from r; bad = min(bad, max(|N|, D) - kappa r1 r2 r3).
__device__ __forceinline__ void vos_term(float rx, float ry, float rz, float4 A, float4 B, float4 C, float &term,
                                         float &bad) {
  const float x1 = A.x - rx, y1 = A.y - ry, z1 = A.z - rz;
  const float x2 = B.x - rx, y2 = B.y - ry, z2 = B.z - rz;
  const float x3 = C.x - rx, y3 = C.y - ry, z3 = C.z - rz;
  const float q1 = fmaf(x1, x1, fmaf(y1, y1, z1 * z1));
  const float q2 = fmaf(x2, x2, fmaf(y2, y2, z2 * z2));
  const float q3 = fmaf(x3, x3, fmaf(y3, y3, z3 * z3));
  const float r1 = sqrt_mufu(q1), r2 = sqrt_mufu(q2), r3 = sqrt_mufu(q3);
  const float cx = fmaf(y2, z3, -z2 * y3), cy = fmaf(z2, x3, -x2 * z3), cz = fmaf(x2, y3, -y2 * x3);
  const float N = fmaf(x1, cx, fmaf(y1, cy, z1 * cz));
  const float d12 = fmaf(x1, x2, fmaf(y1, y2, z1 * z2));
  const float d13 = fmaf(x1, x3, fmaf(y1, y3, z1 * z3));
  const float d23 = fmaf(x2, x3, fmaf(y2, y3, z2 * z3));
  const float r123 = r1 * r2 * r3;
  const float D = fmaf(d12, r3, fmaf(d13, r2, fmaf(d23, r1, r123)));
  term = half_angle(N, D);
  bad = fminf(bad, fmaf(-kKappa, r123, fmaxf(fabsf(N), D)));
}

// Certainty of a representative's FP32 sum after the lanes' compensated
// partials (h, he) and conditioning minima are combined by a butterfly
// (every lane ends with the same value: IEEE addition is commutative).
// True with the winding number in *k when certain (the tests of
// classify_store).
__device__ __forceinline__ bool rep_certain(const LabelArgs &a, float h, float he, float bad, int *k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ph = __shfl_xor_sync(0xffffffffu, h, o);
    const float pe = __shfl_xor_sync(0xffffffffu, he, o);
    two_sum_acc(h, he, ph, pe);
    bad = fminf(bad, __shfl_xor_sync(0xffffffffu, bad, o));
  }
  h += he;
  const float om = 2.f * h;
  const float kf = rintf(h * kInvTwoPi);
  const float dist = 2.f * fabsf(fmaf(-kTwoPi, kf, h));
  const bool unc = !isfinite(om) || !(bad > 0.f) || !(dist <= a.winding_tol) || !(fabsf(om - kTwoPi) >= a.margin);
  if (unc) return false;
  *k = (int)kf;
  return true;
}

// One pass over compartment cp's triangles (lane l takes triangles l, l + 32,
// ...) summing the plain FP32 Van Oosterom-Strackee half angles of the point
// (rx, ry, rz).  With a box wb (non-null) the pass also tests every triangle's
// box against wb and stops at the first chunk of 32 triangles in which one
// meets it, returning that chunk's first index in *t_hit (otherwise -1).
// Returns true with the winding number in *k when the pass completed and the
// point's Omega is certain (the tests of classify_store, with the conditioning
// bound scaled by r1 r2 r3).
__device__ __forceinline__ bool rep_pass(const LabelArgs &a, const DevComp *cp, const float *wb, float rx,
                                         float ry, float rz, int lane, int *k, int *t_hit) {
  const int tri_cnt = __ldg(&cp->tri_cnt);
  const float4 *T = a.tris + (int64_t)__ldg(&cp->tri_off) * 3;
  float lx = 0.f, ly = 0.f, lz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
  if (wb) {
    lx = wb[0]; ly = wb[1]; lz = wb[2]; hx = wb[3]; hy = wb[4]; hz = wb[5];
  }
  *t_hit = -1;
  float sum = 0.f, comp = 0.f, bad = __int_as_float(0x7f800000);
  for (int t0 = 0; t0 < tri_cnt; t0 += 32) {
    const int t = t0 + lane;
    bool ov = false;
    float term = 0.f;
    if (t < tri_cnt) {
      const float4 A = T[3 * t], B = T[3 * t + 1], C = T[3 * t + 2];
      if (wb)
        ov = !(fmaxf(A.x, fmaxf(B.x, C.x)) < lx || fminf(A.x, fminf(B.x, C.x)) > hx ||
               fmaxf(A.y, fmaxf(B.y, C.y)) < ly || fminf(A.y, fminf(B.y, C.y)) > hy ||
               fmaxf(A.z, fmaxf(B.z, C.z)) < lz || fminf(A.z, fminf(B.z, C.z)) > hz);
      vos_term(rx, ry, rz, A, B, C, term, bad);
    }
    if (wb && __any_sync(0xffffffffu, ov)) {
      *t_hit = t0;
      return false;
    }
    const float y = term - comp;
    const float tt = sum + y;
    comp = (tt - sum) - y;
    sum = tt;
  }
  return rep_certain(a, sum, -comp, bad, k);
}

// Representatives of several groups (coordinates rp[g], groups in u) in one
// pass over cp's triangles: each triangle is loaded once for all of them.
// Returns the groups whose representative is certain; their winding numbers
// go to k[g].
template <int NG>
__device__ __forceinline__ uint32_t group_reps(const LabelArgs &a, const DevComp *cp, uint32_t u,
                                               const float (*rp)[3], int lane, int (&k)[NG]) {
  const int tri_cnt = __ldg(&cp->tri_cnt);
  const float4 *T = a.tris + (int64_t)__ldg(&cp->tri_off) * 3;
  float sum[NG], comp[NG], bad[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    sum[g] = comp[g] = 0.f;
    bad[g] = __int_as_float(0x7f800000);
  }
  for (int t = lane; t < tri_cnt; t += 32) {
    const float4 A = T[3 * t], B = T[3 * t + 1], C = T[3 * t + 2];
#pragma unroll
    for (int g = 0; g < NG; ++g)
      if ((u >> g) & 1u) {
        float term;
        vos_term(rp[g][0], rp[g][1], rp[g][2], A, B, C, term, bad[g]);
        const float y = term - comp[g];
        const float tt = sum[g] + y;
        comp[g] = (tt - sum[g]) - y;
        sum[g] = tt;
      }
  }
  uint32_t certain = 0;
#pragma unroll
  for (int g = 0; g < NG; ++g)
    if (((u >> g) & 1u) && rep_certain(a, sum[g], -comp[g], bad[g], &k[g])) certain |= 1u << g;
  return certain;
}

// Groups of a tile (16 consecutive points each, boxes gb[g]) whose box meets
// the box of some triangle of cp, from triangle t_begin on (the earlier ones
// miss the whole tile box wb).  Only the groups in `need` are tested; the
// pass ends once all of them are hit.
template <int NG>
__device__ __forceinline__ uint32_t touched_groups(const LabelArgs &a, const DevComp *cp, const float *wb,
                                                   const float (*gb)[6], uint32_t need, int t_begin, int lane) {
  const int tri_cnt = __ldg(&cp->tri_cnt);
  const float4 *T = a.tris + (int64_t)__ldg(&cp->tri_off) * 3;
  uint32_t hit = 0;
  for (int t0 = t_begin; t0 < tri_cnt; t0 += 32) {
    const int t = t0 + lane;
    if (t < tri_cnt) {
      const float4 A = T[3 * t], B = T[3 * t + 1], C = T[3 * t + 2];
      const float ux = fmaxf(A.x, fmaxf(B.x, C.x)), lx = fminf(A.x, fminf(B.x, C.x));
      const float uy = fmaxf(A.y, fmaxf(B.y, C.y)), ly = fminf(A.y, fminf(B.y, C.y));
      const float uz = fmaxf(A.z, fmaxf(B.z, C.z)), lz = fminf(A.z, fminf(B.z, C.z));
      if (!(ux < wb[0] || lx > wb[3] || uy < wb[1] || ly > wb[4] || uz < wb[2] || lz > wb[5])) {
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (((need >> g) & 1u) && !(ux < gb[g][0] || lx > gb[g][3] || uy < gb[g][1] || ly > gb[g][4] ||
                                      uz < gb[g][2] || lz > gb[g][5]))
            hit |= 1u << g;
      }
    }
    hit = __reduce_or_sync(0xffffffffu, hit);
    if (hit == need) break;
  }
  return hit;
}

// ------------------------------------------------------------------ FP32 persistent kernel
// Every warp is an independent persistent worker: it takes a tile of 32 x P
// consecutive Morton-ordered points from the work list, walks the
// compartments whose boxes meet the tile's box in priority order, and streams
// each compartment's strip entries through its own double buffer in shared
// memory (1-D bulk TMA copies issued by lane 0, one mbarrier per buffer).
// There is no block-wide barrier on the hot path, so a warp that finishes a
// tile early moves straight on to the next one.  Without Omega output a point
// that is certainly inside a compartment needs no lower-priority one (Sec. 2.1:
// the first compartment of the hierarchy wins): groups whose points are all
// decided skip the later compartments, and the warp leaves the tile once all
// its points are decided.
// V = 0: one atan2 per group of four strip steps, on the product of their
//        (D + i N) factors with wrap counting (the default);
// V = 1: one atan2 per triangle.
constexpr int kWChunk = 128;  // strip entries per warp buffer (4 KB)

// Streams compartment cp's strip entries through the warp's double buffer and
// accumulates the FP32 sums of the NA point slots of every lane.  Returns
// false when a bounded wait expired.
template <int NA, int V>
__device__ __forceinline__ bool stream_sums(const LabelArgs &a, const DevComp *cp, Entry *wbuf, uint64_t *bar,
                                            uint32_t &ph0, uint32_t &ph1, int lane, PState (&st)[NA]) {
  const int entry_cnt = __ldg(&cp->entry_cnt);
  const Entry *gsrc = a.entries + __ldg(&cp->entry_off);
  const int nchunks = (entry_cnt + kWChunk - 1) / kWChunk;
  if (lane == 0) {
    tma_load_1d(wbuf, gsrc, min(kWChunk, entry_cnt) * (uint32_t)sizeof(Entry), &bar[0]);
    if (nchunks > 1)
      tma_load_1d(wbuf + kWChunk, gsrc + kWChunk, min(kWChunk, entry_cnt - kWChunk) * (uint32_t)sizeof(Entry),
                  &bar[1]);
  }
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    st[q].grp = st[q].sum = st[q].comp = 0.f;
    st[q].bad = __int_as_float(0x7f800000);
    st[q].kp = st[q].kn = 0u;
  }
  for (int ch = 0; ch < nchunks; ++ch) {
    const int b = ch & 1;
    const bool ok = mbar_wait(&bar[b], b ? ph1 : ph0);
    if (__any_sync(0xffffffffu, !ok)) return false;
    if (b) ph1 ^= 1; else ph0 ^= 1;
    const Entry *E = wbuf + b * kWChunk;
    const int cnt = min(kWChunk, entry_cnt - ch * kWChunk);
    if (ch == 0) {
      const float4 v0 = E[0].v;
#pragma unroll
      for (int q = 0; q < NA; ++q) window_init(st[q], v0);
    }
    for (int g = 0; g < cnt; g += kGroup) {
      if constexpr (V == 0) {
#pragma unroll 1
        for (int j = 0; j < kGroup; j += 4) {
          const Entry *e = E + g + j;
          const float4 v0 = e[0].v, n0 = e[0].n, v1 = e[1].v, n1 = e[1].n;
          const float4 v2 = e[2].v, n2 = e[2].n, v3 = e[3].v, n3 = e[3].n;
#pragma unroll
          for (int q = 0; q < NA; ++q) {
            float N0, D0, N1, D1, r01, i01, r23, i23, R, I;
            geom_step(st[q], v0, n0, N0, D0);
            geom_step(st[q], v1, n1, N1, D1);
            cmul_wrap(D0, N0, D1, N1, r01, i01, st[q].kp, st[q].kn);
            geom_step(st[q], v2, n2, N0, D0);
            geom_step(st[q], v3, n3, N1, D1);
            cmul_wrap(D0, N0, D1, N1, r23, i23, st[q].kp, st[q].kn);
            cmul_wrap(r01, i01, r23, i23, R, I, st[q].kp, st[q].kn);
            st[q].grp += half_angle(I, R);
          }
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < kGroup; ++j) {
          const float4 Vv = E[g + j].v;
          const float4 Nn = E[g + j].n;
#pragma unroll
          for (int q = 0; q < NA; ++q) vos_step(st[q], Vv, Nn);
        }
      }
#pragma unroll
      for (int q = 0; q < NA; ++q) kahan_flush(st[q]);
    }
    __syncwarp();  // every lane is done with buffer b before it is refilled
    if (lane == 0 && ch + 2 < nchunks)
      tma_load_1d(wbuf + b * kWChunk, gsrc + (int64_t)(ch + 2) * kWChunk,
                  min(kWChunk, entry_cnt - (ch + 2) * kWChunk) * (uint32_t)sizeof(Entry), &bar[b]);
  }
  return true;
}

// ------------------------------------------------------------------ cap trees (kernel form 2)
// For a box of points, the strip segments that stand for a compartment's
// surface: a depth-first walk of its cap tree emits the cap of every node
// whose box misses the point box (outside that box the cap subtends the
// node's patch exactly) and the strips of every leaf whose box meets it.
// The result is a list of entry ranges of the cap-tree segment array
// (contiguous segments merged) with *total entries holding *tris triangles;
// more than kMaxRanges ranges return -1, or with `all_leaves` fall back to
// every leaf segment.
constexpr int kMaxRanges = 192;
// A tile's walk takes a node's cap only when the tile's box misses the node's
// box grown by kCapMargin times the box's longest side: a cap triangle spans
// its patch's boundary, and one that passes within a small fraction of its
// own size from a point carries the largest FP32 rounding (measured on the
// full head: with no margin about 3 % of the certified sums were more than
// 1e-5 from their winding number's 4 pi k, with 1/64 about 0.03 %, for 3 %
// more evaluated pairs).
constexpr float kCapMargin = 1.f / 64.f;

// With `lout` (non-null) the walk also lists the leaf segments alone (the
// only ones whose triangles can meet the box: a cap lies in its node's box,
// which misses it): *lcnt ranges holding *ltot entries, or *lcnt = -1 when
// they exceed kMaxLeafRanges.
constexpr int kMaxLeafRanges = 64;

__device__ int cap_ranges(const LabelArgs &a, const DevComp *cp, const float *wb, int2 *out, int *total,
                          int *tris, bool all_leaves, float margin = 0.f, int2 *lout = nullptr,
                          int *lcnt = nullptr, int *ltot = nullptr) {
  int n = 0, tot = 0, nt = 0, nl = 0, lt = 0;
  // pre-order walk without a stack: descend to i + 1, or continue at skip
  const int root = __ldg(&cp->cap_root);
  const int end = __ldg(&a.nodes[root].skip);
  for (int i = root; i != end;) {
    if (!ZEF_BOUNDS_OK(i >= 0 && i < a.n_nodes, a.status, 10)) {
      n = 0;
      tot = nt = nl = lt = 0;
      break;
    }
    const CapNode nd = a.nodes[i];
    const float m = margin * fmaxf(nd.hi[0] - nd.lo[0], fmaxf(nd.hi[1] - nd.lo[1], nd.hi[2] - nd.lo[2]));
    const bool far = nd.hi[0] + m < wb[0] || nd.lo[0] - m > wb[3] || nd.hi[1] + m < wb[1] || nd.lo[1] - m > wb[4] ||
                     nd.hi[2] + m < wb[2] || nd.lo[2] - m > wb[5];
    int b, c, t;
    if (far) {
      b = nd.cap_begin;
      c = nd.cap_cnt;
      t = nd.cap_tris;
    } else if (nd.left < 0) {
      b = nd.leaf_begin;
      c = nd.leaf_cnt;
      t = nd.leaf_tris;
    } else {
      ++i;
      continue;
    }
    i = nd.skip;
    if (c <= 0) continue;
    if (!ZEF_BOUNDS_OK(b >= 0 && (int64_t)b + c <= a.n_cseg, a.status, 11)) continue;
    tot += c;
    nt += t;
    if (n > 0 && out[n - 1].x + out[n - 1].y == b) {
      out[n - 1].y += c;
    } else if (n < kMaxRanges) {
      out[n++] = make_int2(b, c);
    } else {
      n = -1;
      break;
    }
    if (lout && !far && nl >= 0) {
      lt += c;
      if (nl > 0 && lout[nl - 1].x + lout[nl - 1].y == b) lout[nl - 1].y += c;
      else if (nl < kMaxLeafRanges) lout[nl++] = make_int2(b, c);
      else nl = -1;
    }
  }
  if (n < 0 && all_leaves) {  // every leaf segment: the compartment's own triangles
    out[0] = make_int2(__ldg(&cp->cseg_off), __ldg(&cp->cseg_leaf));
    n = 1;
    tot = out[0].y;
    nt = __ldg(&cp->tri_cnt);
  }
  *total = tot;
  *tris = nt;
  if (lout) {
    *lcnt = nl;
    *ltot = nl < 0 ? 0 : lt;
  }
  return n;
}

// Position of flattened entry j of a range list; the cursor (range r, first
// flattened index of r) only moves forward.
__device__ __forceinline__ int range_pos(const int2 *rng, int &r, int &rb, int j) {
  while (j >= rb + rng[r].y) {
    rb += rng[r].y;
    ++r;
  }
  return rng[r].x + (j - rb);
}

// The triangle closed by segment entry `pos` (its window: the two entries
// before it, which lie in the same segment), with the stored oriented
// normal and kappa |n| in nn.w; false for a window that is not a triangle.
__device__ __forceinline__ bool seg_tri(const Entry *E, int pos, float4 &A, float4 &B, float4 &C, float4 &nn) {
  C = E[pos].v;
  if (fabsf(C.w) != 1.f) return false;
  A = E[pos - 2].v;
  B = E[pos - 1].v;
  nn = E[pos].n;
  return true;
}


// Groups of a tile (16 consecutive points each, boxes gb[g]) whose box
// meets the box of some triangle of the leaf ranges (the surface's own
// triangles near the tile); *tile_hit reports whether any triangle box meets
// the tile's box wb.  Only the groups in `need` are tested; the pass ends
// once all of them are hit.
template <int NG>
__device__ __forceinline__ uint32_t touched_leaves(const LabelArgs &a, const int2 *lrng, int ltot, const float *wb,
                                                   const float (*gb)[6], uint32_t need, int lane, bool *tile_hit) {
  uint32_t hit = 0;
  bool th = false;
  int r = 0, rb = 0;
  for (int t0 = 0; t0 < ltot; t0 += 32) {
    const int j = t0 + lane;
    float4 A, B, C, nn;
    if (j < ltot && seg_tri(a.cseg, range_pos(lrng, r, rb, j), A, B, C, nn)) {
      const float ux = fmaxf(A.x, fmaxf(B.x, C.x)), lx = fminf(A.x, fminf(B.x, C.x));
      const float uy = fmaxf(A.y, fmaxf(B.y, C.y)), ly = fminf(A.y, fminf(B.y, C.y));
      const float uz = fmaxf(A.z, fmaxf(B.z, C.z)), lz = fminf(A.z, fminf(B.z, C.z));
      if (!(ux < wb[0] || lx > wb[3] || uy < wb[1] || ly > wb[4] || uz < wb[2] || lz > wb[5])) {
        th = true;
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (((need >> g) & 1u) && !(ux < gb[g][0] || lx > gb[g][3] || uy < gb[g][1] || ly > gb[g][4] ||
                                      uz < gb[g][2] || lz > gb[g][5]))
            hit |= 1u << g;
      }
    }
    hit = __reduce_or_sync(0xffffffffu, hit);
    th = __any_sync(0xffffffffu, th);
    if (hit == need) break;
  }
  *tile_hit = th;
  return hit;
}

// Window of a strip group opened from the two entries before it (A, B): the
// state the sequential stream holds after those two steps, computed with the
// same operations (so the group's factors are the stream's own).
__device__ __forceinline__ void window_prime(PState &s, float4 A, float4 B) {
  s.ax = A.x - s.px;
  s.ay = A.y - s.py;
  s.az = A.z - s.pz;
  s.bx = B.x - s.px;
  s.by = B.y - s.py;
  s.bz = B.z - s.pz;
  const float qa = fmaf(s.ax, s.ax, fmaf(s.ay, s.ay, s.az * s.az));
  const float qb = fmaf(s.bx, s.bx, fmaf(s.by, s.by, s.bz * s.bz));
  s.ra = sqrt_mufu(qa);
  s.rb = sqrt_mufu(qb);
  s.sab = fmaf(s.ra, s.rb, fmaf(s.ax, s.bx, fmaf(s.ay, s.by, s.az * s.bz)));
}

// Sums of nr <= NR representative points over a range list of strip
// segments, the entries split over the lanes instead of the points: lane l
// takes the group of four entries [4 l, 4 l + 4) of each run of kWChunk
// entries of the flattened list.  A group lies inside one segment (segments
// hold whole groups of four), contiguous in memory, and opens its window from
// the two entries before it in that segment or restarts at a reset entry, so
// its four (D + i N) factors are those the sequential stream forms; one
// atan2 per group, wraps counted as in the point-by-point sums, a Kahan sum
// per lane.  Each lane reads its own entries through the read-only cache
// (its cursor over the ranges moves forward only): a warp finishes a run of
// kWChunk entries about 32 times sooner than in the point-by-point sums, too
// soon for the warp's double-buffered bulk copies to keep ahead of it (the
// passes spent most of their time waiting on them).  The lanes' sums, wraps and conditioning minima are
// then combined and each representative is certified by the tests of
// classify_store: bit r of *certain (r < nr) marks a certified
// representative, its winding number in k[r].
template <int NR>
__device__ __noinline__ void rep_stream(const LabelArgs &a, const int2 *rng, int total, int lane,
                                        const float (*rp)[3], int nr, uint32_t *certain, int (&k)[NR]) {
  const int nruns = (total + kWChunk - 1) / kWChunk;
  int cr = 0, cb = 0;  // the lane's cursor: range, and the range's first flattened entry
  float sum[NR], comp[NR], bad[NR];
  int wr[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    sum[r] = comp[r] = 0.f;
    bad[r] = __int_as_float(0x7f800000);
    wr[r] = 0;
  }
  for (int ch = 0; ch < nruns; ++ch) {
    const int j = ch * kWChunk + 4 * lane;
    if (j >= total) continue;
    const int g = range_pos(rng, cr, cb, j);
    if (!ZEF_BOUNDS_OK(g >= 0 && (int64_t)g + 4 <= a.n_cseg, a.status, 21)) continue;
    const Entry *E = a.cseg + g;
    const float4 v0 = __ldg(&E[0].v), n0 = __ldg(&E[0].n), v1 = __ldg(&E[1].v), n1 = __ldg(&E[1].n);
    const float4 v2 = __ldg(&E[2].v), n2 = __ldg(&E[2].n), v3 = __ldg(&E[3].v), n3 = __ldg(&E[3].n);
    float4 A = v0, B = v0;
    if (v0.w != 2.f) {
      A = __ldg(&E[-2].v);
      B = __ldg(&E[-1].v);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r >= nr) break;
      PState st;
      st.px = rp[r][0];
      st.py = rp[r][1];
      st.pz = rp[r][2];
      st.bad = __int_as_float(0x7f800000);
      st.kp = st.kn = 0u;
      if (v0.w == 2.f) window_init(st, v0);
      else window_prime(st, A, B);
      float N0, D0, N1, D1, r01, i01, r23, i23, R, I;
      geom_step(st, v0, n0, N0, D0);
      geom_step(st, v1, n1, N1, D1);
      cmul_wrap(D0, N0, D1, N1, r01, i01, st.kp, st.kn);
      geom_step(st, v2, n2, N0, D0);
      geom_step(st, v3, n3, N1, D1);
      cmul_wrap(D0, N0, D1, N1, r23, i23, st.kp, st.kn);
      cmul_wrap(r01, i01, r23, i23, R, I, st.kp, st.kn);
      const float y = half_angle(I, R) - comp[r];
      const float t = sum[r] + y;
      comp[r] = (t - sum[r]) - y;
      sum[r] = t;
      wr[r] += (int)st.kp - (int)st.kn;
      bad[r] = fminf(bad[r], st.bad);
    }
  }
  uint32_t cert = 0;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r >= nr) break;
    float h = sum[r], he = -comp[r], bd = bad[r];
    int w = wr[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ph = __shfl_xor_sync(0xffffffffu, h, o);
      const float pe = __shfl_xor_sync(0xffffffffu, he, o);
      two_sum_acc(h, he, ph, pe);
      bd = fminf(bd, __shfl_xor_sync(0xffffffffu, bd, o));
      w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    h += he;
    // Omega / 2 = h + 2 pi w; the distance to 4 pi Z from h alone (w drops out)
    const float kf = rintf(h * kInvTwoPi);
    const float dist = 2.f * fabsf(fmaf(-kTwoPi, kf, h));
    const float om = 2.f * fmaf(kTwoPi, (float)w, h);
    const bool unc = !isfinite(om) || !(bd > 0.f) || !(dist <= a.winding_tol) || !(fabsf(om - kTwoPi) >= a.margin);
    if (!unc) {
      cert |= 1u << r;
      k[r] = w + (int)kf;
    }
  }
  *certain = cert;
}

// Point-by-point sums over a range list of strip segments: chunks of
// kWChunk entries (4 KB) gathered into the warp's double buffer by one or
// more bulk copies on one mbarrier (one range piece per lane, issued by the
// lanes together); every lane steps its points' windows
// through the entries, multiplies the (D + i N) factors of four consecutive
// windows with wrap counting and takes one atan2 per four, the group sums
// Kahan-compensated every kGroup entries.  A segment opens with a reset
// entry at a multiple of four (every segment holds whole groups of four),
// which restarts the windows at its vertex.
template <int NA>
__device__ __forceinline__ bool stream_sums_caps(const LabelArgs &a, const int2 *rng, int total, int nrng,
                                                 Entry *wbuf, uint64_t *bar, uint32_t &ph0, uint32_t &ph1, int lane,
                                                 PState (&st)[NA]) {
  const int nchunks = (total + kWChunk - 1) / kWChunk;
  int fr = 0, fb = 0;  // the warp's cursor over the ranges: range, its first flattened entry (every lane)
  // Bulk copies of the flattened entries [j0, j1) into buffer b, issued by
  // the lanes together: lane l copies its share of range fr + l (the flattened
  // starts of 32 ranges at a time from a warp prefix sum of their lengths).
  auto fill = [&](int ch, int b) {
    const int j0 = ch * kWChunk, j1 = min(total, j0 + kWChunk);
    if (lane == 0) tma_expect(&bar[b], (uint32_t)(j1 - j0) * (uint32_t)sizeof(Entry));
    __syncwarp();
    for (;;) {
      const int r = fr + lane;
      const int c = r < nrng ? rng[r].y : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int beg = fb + incl - c, end = beg + c;
      const int s0 = max(beg, j0), s1 = min(end, j1);
      if (s1 > s0)
        tma_copy_1d(wbuf + b * kWChunk + (s0 - j0), a.cseg + (rng[r].x + (s0 - beg)),
                    (uint32_t)(s1 - s0) * (uint32_t)sizeof(Entry), &bar[b]);
      const uint32_t past = __ballot_sync(0xffffffffu, end > j1);
      if (past) {  // the range holding entry j1 opens the next chunk
        const int L = __ffs(past) - 1;
        fb = __shfl_sync(0xffffffffu, beg, L);
        fr += L;
        break;
      }
      fb = __shfl_sync(0xffffffffu, end, 31);
      fr += 32;
      if (fb >= j1 || fr >= nrng) break;
    }
  };
  if (nchunks > 0) fill(0, 0);
  if (nchunks > 1) fill(1, 1);
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    st[q].grp = st[q].sum = st[q].comp = 0.f;
    st[q].bad = __int_as_float(0x7f800000);
    st[q].kp = st[q].kn = 0u;
  }
  PState2 st2;  // NA == 2: both slots' points and windows as pairs
  if constexpr (NA == 2) {
    st2.px = pk(st[0].px, st[1].px);
    st2.py = pk(st[0].py, st[1].py);
    st2.pz = pk(st[0].pz, st[1].pz);
    st2.ax = st2.ay = st2.az = st2.bx = st2.by = st2.bz = st2.ra = st2.rb = st2.sab = pk(0.f, 0.f);
    st2.bad0 = st2.bad1 = __int_as_float(0x7f800000);
  }
  for (int ch = 0; ch < nchunks; ++ch) {
    const int b = ch & 1;
    const bool ok = mbar_wait(&bar[b], b ? ph1 : ph0);
    if (__any_sync(0xffffffffu, !ok)) return false;
    if (b) ph1 ^= 1; else ph0 ^= 1;
    const Entry *E = wbuf + b * kWChunk;
    const int cnt = min(kWChunk, total - ch * kWChunk);  // a multiple of four
    if constexpr (NA == 2) {
      // both slots at once on packed pairs; the windows are carried across
      // chunks in st2
      for (int g = 0; g < cnt; g += kGroup) {
#pragma unroll 1
        for (int j = g; j < min(cnt, g + kGroup); j += 4) {
          const Entry *e = E + j;
          const float4 v0 = e[0].v, n0 = e[0].n, v1 = e[1].v, n1 = e[1].n;
          const float4 v2 = e[2].v, n2 = e[2].n, v3 = e[3].v, n3 = e[3].n;
          if (v0.w == 2.f) window_init2(st2, v0);
          f2 N0, D0, N1, D1, r01, i01, r23, i23, R, I;
          geom_step2(st2, v0, n0, N0, D0);
          geom_step2(st2, v1, n1, N1, D1);
          cmul_wrap2(D0, N0, D1, N1, r01, i01, st[0].kp, st[0].kn, st[1].kp, st[1].kn);
          geom_step2(st2, v2, n2, N0, D0);
          geom_step2(st2, v3, n3, N1, D1);
          cmul_wrap2(D0, N0, D1, N1, r23, i23, st[0].kp, st[0].kn, st[1].kp, st[1].kn);
          cmul_wrap2(r01, i01, r23, i23, R, I, st[0].kp, st[0].kn, st[1].kp, st[1].kn);
          st[0].grp += half_angle(lo(I), lo(R));
          st[1].grp += half_angle(hi(I), hi(R));
        }
        kahan_flush(st[0]);
        kahan_flush(st[1]);
      }
    } else {
    for (int g = 0; g < cnt; g += kGroup) {
#pragma unroll 1
      for (int j = g; j < min(cnt, g + kGroup); j += 4) {
        const Entry *e = E + j;
        const float4 v0 = e[0].v, n0 = e[0].n, v1 = e[1].v, n1 = e[1].n;
        const float4 v2 = e[2].v, n2 = e[2].n, v3 = e[3].v, n3 = e[3].n;
        if (v0.w == 2.f) {
#pragma unroll
          for (int q = 0; q < NA; ++q) window_init(st[q], v0);
        }
#pragma unroll
        for (int q = 0; q < NA; ++q) {
          float N0, D0, N1, D1, r01, i01, r23, i23, R, I;
          geom_step(st[q], v0, n0, N0, D0);
          geom_step(st[q], v1, n1, N1, D1);
          cmul_wrap(D0, N0, D1, N1, r01, i01, st[q].kp, st[q].kn);
          geom_step(st[q], v2, n2, N0, D0);
          geom_step(st[q], v3, n3, N1, D1);
          cmul_wrap(D0, N0, D1, N1, r23, i23, st[q].kp, st[q].kn);
          cmul_wrap(r01, i01, r23, i23, R, I, st[q].kp, st[q].kn);
          st[q].grp += half_angle(I, R);
        }
      }
#pragma unroll
      for (int q = 0; q < NA; ++q) kahan_flush(st[q]);
    }
    }
    __syncwarp();  // every lane is done with buffer b before it is refilled
    if (ch + 2 < nchunks) fill(ch + 2, b);
  }
  if constexpr (NA == 2) {
    st[0].bad = st2.bad0;
    st[1].bad = st2.bad1;
  }
  return true;
}

// Per-lane evaluation, for a tile whose shared range list is long (its box
// covers far more of the surface than any of its points needs, as when its
// Morton-consecutive points straddle a jump of the curve): every lane walks
// the cap tree for each of its own points in `todo` and streams that walk's
// segments from global memory four entries at a time, with the same
// products, wrap counting and compensation as the shared stream.  A node is
// far from a point when the point lies outside the node's box grown by a
// quarter of the box's longest side on every side (exact outside the box;
// the margin keeps the cap's triangles at a distance from the point that is
// a fixed fraction of their size, as the tile's own extent does for the
// shared lists).  Returns the bits q of the points certainly inside; *pairs
// receives the triangles evaluated.
constexpr int kLaneWalkFloor = 4096;  // shared lists up to this long are always kept
constexpr int kLaneWalkRatio = 3;     // longer ones go per lane when > ratio x the longest own walk

__device__ __forceinline__ bool lane_far(const CapNode &nd, float x, float y, float z) {
  const float m = 0.25f * fmaxf(nd.hi[0] - nd.lo[0], fmaxf(nd.hi[1] - nd.lo[1], nd.hi[2] - nd.lo[2]));
  return nd.hi[0] + m < x || nd.lo[0] - m > x || nd.hi[1] + m < y || nd.lo[1] - m > y || nd.hi[2] + m < z ||
         nd.lo[2] - m > z;
}

// Entries of a point's own walk (the same walk as lane_walk_caps).
__device__ __noinline__ int lane_walk_entries(const LabelArgs &a, int root, float x, float y, float z) {
  int tot = 0;
  const int end = __ldg(&a.nodes[root].skip);
  for (int i = root; i != end;) {
    const CapNode nd = a.nodes[i];
    if (lane_far(nd, x, y, z)) {
      tot += nd.cap_cnt;
      i = nd.skip;
    } else if (nd.left < 0) {
      tot += nd.leaf_cnt;
      i = nd.skip;
    } else {
      ++i;
    }
  }
  return tot;
}

template <int P>
__device__ __noinline__ uint32_t lane_walk_caps(const LabelArgs &a, const DevComp *cp, const float *thr, int base,
                                                uint32_t todo, int lane, unsigned long long *pairs) {
  const DevComp c = *cp;
  uint32_t in = 0;
  unsigned long long np = 0;
  for (int q = 0; q < P; ++q) {
    if (!((todo >> q) & 1u)) continue;
    const int i = base + 32 * q + lane;
    const float4 p = a.spts[i];
    PState st;
    st.px = p.x;
    st.py = p.y;
    st.pz = p.z;
    st.grp = st.sum = st.comp = 0.f;
    st.bad = __int_as_float(0x7f800000);
    st.kp = st.kn = 0u;
    int b = 0, e = 0, g = 0;
    int node = c.cap_root;
    const int end = __ldg(&a.nodes[node].skip);
    for (;;) {
      // pre-order walk without a stack to the next segment
      while (b >= e && node != end) {
        if (!ZEF_BOUNDS_OK(node >= 0 && node < a.n_nodes, a.status, 12)) {
          node = end;
          break;
        }
        const CapNode nd = a.nodes[node];
        if (lane_far(nd, p.x, p.y, p.z)) {
          b = nd.cap_begin;
          e = b + nd.cap_cnt;
          np += (unsigned long long)nd.cap_tris;
          node = nd.skip;
        } else if (nd.left < 0) {
          b = nd.leaf_begin;
          e = b + nd.leaf_cnt;
          np += (unsigned long long)nd.leaf_tris;
          node = nd.skip;
        } else {
          ++node;
        }
      }
      if (b >= e) break;
      if (!ZEF_BOUNDS_OK(b >= 0 && (int64_t)b + 4 <= a.n_cseg, a.status, 13)) break;
      const Entry *E = a.cseg + b;
      const float4 v0 = __ldg(&E[0].v), n0 = __ldg(&E[0].n), v1 = __ldg(&E[1].v), n1 = __ldg(&E[1].n);
      const float4 v2 = __ldg(&E[2].v), n2 = __ldg(&E[2].n), v3 = __ldg(&E[3].v), n3 = __ldg(&E[3].n);
      if (v0.w == 2.f) window_init(st, v0);
      float N0, D0, N1, D1, r01, i01, r23, i23, R, I;
      geom_step(st, v0, n0, N0, D0);
      geom_step(st, v1, n1, N1, D1);
      cmul_wrap(D0, N0, D1, N1, r01, i01, st.kp, st.kn);
      geom_step(st, v2, n2, N0, D0);
      geom_step(st, v3, n3, N1, D1);
      cmul_wrap(D0, N0, D1, N1, r23, i23, st.kp, st.kn);
      cmul_wrap(r01, i01, r23, i23, R, I, st.kp, st.kn);
      st.grp += half_angle(I, R);
      b += 4;
      if (++g == kGroup / 4) {
        kahan_flush(st);
        g = 0;
      }
    }
    kahan_flush(st);
    if (classify_store(a, c, thr, i, p.x, p.y, p.z, st.sum - st.comp, (int)st.kp - (int)st.kn, st.bad))
      in |= 1u << q;
  }
  *pairs = np;
  return in;
}

// Point-by-point evaluation of the groups in `act` (m of them), packed two
// per slot of 32 lanes (NA = ceil(m / 2) slots): slot j holds the groups at
// positions 2j (lanes 0-15) and 2j + 1 (lanes 16-31) of the ascending list of
// `act`.  Classifies every evaluated point and sets bit q of `done` for the
// points (in the tile's own layout, point base + 32 q + lane) certainly
// inside.  Returns false when a bounded wait expired.
template <int NA, int V, int P>
__device__ __noinline__ bool eval_groups(const LabelArgs &a, const DevComp *cp, const float *thr, Entry *wbuf,
                                            uint64_t *bar, uint32_t &ph0, uint32_t &ph1, int lane, int base, int n,
                                            uint32_t act, uint32_t list, int m, uint32_t &done, const int2 *rng,
                                            int rtotal, int rtris, int nrng) {
  PState st[NA];
  int idx[NA];
  const int half = lane >> 4;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    const int pos = 2 * j + half;
    const int g = pos < m ? (int)((list >> (4 * pos)) & 15u) : -1;
    const int i = g >= 0 ? base + 16 * g + (lane & 15) : n;
    const bool valid = i < n;
    const float4 p = a.spts[valid ? i : base];
    st[j].px = p.x;
    st[j].py = p.y;
    st[j].pz = p.z;
    idx[j] = (valid && finite3(p.x, p.y, p.z)) ? i : -1;
  }
  if constexpr (V == 2) {
    if (!stream_sums_caps<NA>(a, rng, rtotal, nrng, wbuf, bar, ph0, ph1, lane, st))
      return false;
  } else {
    if (!stream_sums<NA, V>(a, cp, wbuf, bar, ph0, ph1, lane, st)) return false;
  }
  const DevComp c = *cp;
  uint32_t in_bits[NA];
  int evaluated = 0;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    bool inside = false;
    if (idx[j] >= 0)
      inside = classify_store(a, c, thr, idx[j], st[j].px, st[j].py, st[j].pz, st[j].sum - st[j].comp,
                              (int)st[j].kp - (int)st[j].kn, st[j].bad);
    in_bits[j] = __ballot_sync(0xffffffffu, inside);
    evaluated += __popc(__ballot_sync(0xffffffffu, idx[j] >= 0));
  }
  // back to the tile's layout: the group of point (q, lane) is 2 q + half; its
  // position in the packed list is the number of active groups below it
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int g = 2 * q + half;
    if ((act >> g) & 1u) {
      const int pos = __popc(act & ((1u << g) - 1u));
      uint32_t bits = 0;
#pragma unroll
      for (int j = 0; j < NA; ++j)
        if (j == (pos >> 1)) bits = in_bits[j];
      if ((bits >> (16 * (pos & 1) + (lane & 15))) & 1u) done |= 1u << q;
    }
  }
  if (lane == 0)
    atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_EVAL),
              (unsigned long long)evaluated * (V == 2 ? rtris : c.tri_cnt));
  return true;
}

// Register budget: 128 registers (16 warps per SM) with two points per
// thread, which measured fastest; unconstrained with four.
template <int NT, int P>
constexpr int label32_min_blocks() {
  return P == 2 ? 512 / NT : 1;
}

template <int NT, int P, int V>
__global__ void __launch_bounds__(NT, label32_min_blocks<NT, P>()) k_label32(LabelArgs a) {
  constexpr int NW = NT / 32;
  constexpr int TILE = 32 * P;
  constexpr int NG = 2 * P;  // groups of 16 consecutive points
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[NW][2];
  __shared__ int s_rowcomp[ZEF_MAX_COMPARTMENTS];
  __shared__ float s_wbox[NW][6];
  __shared__ float s_gbox[NW][NG][6];
  __shared__ float s_rep[NW][NG][3];
  constexpr int RN = V == 2 ? kMaxRanges : 1;
  __shared__ int2 s_rng[NW][RN];   // form 2: the tile's range list of the compartment
  constexpr int LN = V == 2 ? kMaxLeafRanges : 1;
  __shared__ int2 s_lrng[NW][LN];  // form 2: its leaf ranges alone
  __shared__ int s_rtot[NW][5];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, half = lane >> 4;
  Entry *wbuf = reinterpret_cast<Entry *>(smem_raw) + wid * 2 * kWChunk;
  uint64_t *bar = bars[wid];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  for (int c = threadIdx.x; c < a.ncomp; c += NT) s_rowcomp[a.comps[c].row] = c;
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;
  const int n = (int)a.counters[CNT_NIN];  // sorted points inside the union box, < 2^31 (checked on the host)
  const int64_t nitems = a.counters[CNT_ITEMS];
  const bool early = a.early;
  for (;;) {
    int64_t item = 0;
    if (lane == 0) item = (int64_t)atomicAdd((unsigned long long *)(a.counters + CNT_WORK), 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int tile = a.items[item].x;
    if (!ZEF_BOUNDS_OK(tile >= 0 && (int64_t)tile * TILE < (int64_t)n, a.status, 20)) continue;
    const int base = tile * TILE;
    uint32_t done = 0;    // bit q: point q is invalid, non-finite or certainly inside an earlier compartment
    uint32_t usable = 0;  // bit q: point q is valid and finite
    float wb[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = base + q * 32 + lane;
      const bool valid = i < n;
      const float4 p = a.spts[valid ? i : base];
      const bool ok = valid && finite3(p.x, p.y, p.z);
      if (!ok) done |= 1u << q;
      else usable |= 1u << q;
      // box of the point's group of 16 (half-warp reduction), then the tile's
      float g[6] = {ok ? p.x : INFINITY, ok ? p.y : INFINITY, ok ? p.z : INFINITY,
                    ok ? p.x : -INFINITY, ok ? p.y : -INFINITY, ok ? p.z : -INFINITY};
#pragma unroll
      for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          g[k] = fminf(g[k], __shfl_xor_sync(0xffffffffu, g[k], o));
          g[3 + k] = fmaxf(g[3 + k], __shfl_xor_sync(0xffffffffu, g[3 + k], o));
        }
      if ((lane & 15) == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) s_gbox[wid][2 * q + half][k] = g[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        wb[k] = fminf(wb[k], g[k]);
        wb[3 + k] = fmaxf(wb[3 + k], g[3 + k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wb[k] = fminf(wb[k], __shfl_xor_sync(0xffffffffu, wb[k], 16));
      wb[3 + k] = fmaxf(wb[3 + k], __shfl_xor_sync(0xffffffffu, wb[3 + k], 16));
    }
    // the tile's box lives in shared memory while the compartments are walked
    if (lane == 0)
      for (int k = 0; k < 6; ++k) s_wbox[wid][k] = wb[k];
    __syncwarp();
    bool timed_out = false;
    for (int r = 0; r < a.ncomp; ++r) {
      // the compartment record is re-read where needed (read-only, cached)
      // rather than held in registers across the hot loop
      const DevComp *cp = a.comps + s_rowcomp[r];
      const float *thr = a.dop + (int64_t)s_rowcomp[r] * kDop;
      // winding number 0 for every point of the tile
      if (box_misses(s_wbox[wid], cp) || dop_box_misses_warp(s_wbox[wid], thr, lane)) continue;
      // groups with a point that still needs this compartment
      uint32_t need = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const uint32_t b = __ballot_sync(0xffffffffu, ((usable >> q) & 1u) && !(early && ((done >> q) & 1u)));
        need |= ((b & 0xffffu) ? 1u : 0u) << (2 * q);
        need |= ((b >> 16) ? 1u : 0u) << (2 * q + 1);
      }
      if (!need) {
        if (early) break;  // every point decided: no later compartment matters
        continue;          // no usable point in the tile
      }
      // form 2: the strip entries (and their triangles) standing for the
      // surface near this tile
      int rtotal = 0, rtris = 0, nrng = 0;
      if constexpr (V == 2) {
        if (lane == 0) {
          int tot = 0, nt = 0, nl = 0, lt = 0;
          const int nr = cap_ranges(a, cp, s_wbox[wid], s_rng[wid], &tot, &nt, false, kCapMargin, s_lrng[wid], &nl,
                                    &lt);
          s_rtot[wid][0] = nr < 0 ? -1 : tot;
          s_rtot[wid][1] = nt;
          s_rtot[wid][2] = nl;
          s_rtot[wid][3] = lt;
          s_rtot[wid][4] = nr;
        }
        __syncwarp();
        rtotal = s_rtot[wid][0];
        rtris = s_rtot[wid][1];
        nrng = s_rtot[wid][4];
        uint32_t todo = 0;
#pragma unroll
        for (int q = 0; q < P; ++q)
          if (((usable >> q) & 1u) && !(early && ((done >> q) & 1u))) todo |= 1u << q;
        bool per_lane = rtotal < 0 || !a.lane_walk;
        if (!per_lane && rtotal > kLaneWalkFloor) {
          // the longest own walk of one point per lane (the lanes walk in
          // parallel) decides
          int own = 0;
          if (todo) {
            const int q = __ffs(todo) - 1;
            const float4 p = a.spts[base + 32 * q + lane];
            own = lane_walk_entries(a, __ldg(&cp->cap_root), p.x, p.y, p.z);
          }
          own = __reduce_max_sync(0xffffffffu, own);
          per_lane = (long long)rtotal > (long long)kLaneWalkRatio * own;
        }
        if (per_lane) {
          unsigned long long pairs = 0;
          done |= lane_walk_caps<P>(a, cp, thr, base, todo, lane, &pairs);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
          if (lane == 0) {
            atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_EVAL), pairs);
            atomicAdd((unsigned long long *)(a.counters + CNT_LANE_TILES), 1ull);
          }
          continue;
        }
      }
      const unsigned long long surf = V == 2 ? (unsigned long long)rtris : (unsigned long long)__ldg(&cp->tri_cnt);
      uint32_t coh = 0;  // groups whose points take a representative's winding number
      int kg[NG];
#pragma unroll
      for (int g = 0; g < NG; ++g) kg[g] = 0;
      if (a.coherence && V == 2) {
        // Coherence (cap-tree form): where no triangle's box meets a box of
        // points, the surface does not cross that box (convex, hence
        // connected), so all its points have the winding number of any one of
        // them.  Only the leaf triangles of the tile's list can meet the
        // tile's box (a cap lies in its node's box, which misses it), so the
        // box tests run over the leaf ranges alone; then one representative
        // (the tile's first usable point) when no triangle box meets the
        // tile's box, else one per group of 16 points that no triangle box
        // meets.  The representatives' sums run over the whole list with the
        // entries split over the lanes (rep_stream).
        const int nl = s_rtot[wid][2], ltot = s_rtot[wid][3];
        bool tile_hit = false;
        uint32_t touched = 0;
        if (nl < 0)  // leaf ranges overflowed: every entry of the list (caps never hit)
          touched = touched_leaves<NG>(a, s_rng[wid], rtotal, s_wbox[wid], s_gbox[wid], need, lane, &tile_hit);
        else if (ltot > 0)
          touched = touched_leaves<NG>(a, s_lrng[wid], ltot, s_wbox[wid], s_gbox[wid], need, lane, &tile_hit);
        uint32_t untouched = need & ~touched;
        // an odd number of touched groups leaves half a slot of lanes free:
        // one untouched group is evaluated there instead of by its
        // representative
        if (tile_hit && (__popc(need & ~untouched) & 1) && untouched) untouched &= untouched - 1u;
        int nrep = 0;
        if (untouched) {
          // representatives in shared memory: the tile's first usable point,
          // or each untouched group's
          uint32_t ub[P];
#pragma unroll
          for (int q = 0; q < P; ++q) ub[q] = __ballot_sync(0xffffffffu, (usable >> q) & 1u);
          if (lane == 0) {
#pragma unroll
            for (int g = 0; g < NG; ++g) {
              const uint32_t gl = (ub[g >> 1] >> (16 * (g & 1))) & 0xffffu;
              const bool take = tile_hit ? ((untouched >> g) & 1u) != 0u : (nrep == 0 && gl != 0u);
              if (take) {
                const float4 gp = a.spts[base + 32 * (g >> 1) + 16 * (g & 1) + __ffs(gl) - 1];
                s_rep[wid][nrep][0] = gp.x;
                s_rep[wid][nrep][1] = gp.y;
                s_rep[wid][nrep][2] = gp.z;
                ++nrep;
              }
            }
          }
          nrep = __shfl_sync(0xffffffffu, nrep, 0);
          __syncwarp();
          uint32_t rep_cert = 0;
          int rk[NG];
#pragma unroll
          for (int g = 0; g < NG; ++g) rk[g] = 0;
          for (int r0 = 0; r0 < nrep; r0 += 2) {
            uint32_t c2 = 0;
            int k2[2] = {0, 0};
            rep_stream<2>(a, s_rng[wid], rtotal, lane, s_rep[wid] + r0, min(2, nrep - r0), &c2, k2);
#pragma unroll
            for (int g = 0; g < NG; ++g) {
              if (g == r0 && (c2 & 1u)) rk[g] = k2[0];
              if (g == r0 + 1 && (c2 & 2u)) rk[g] = k2[1];
            }
            rep_cert |= c2 << r0;
          }
          if (!tile_hit) {
            if (rep_cert & 1u) {
              coh = need;
#pragma unroll
              for (int g = 0; g < NG; ++g) kg[g] = rk[0];
            }
          } else {
            // representative r stands for the r-th group of `untouched`
            int r = 0;
#pragma unroll
            for (int g = 0; g < NG; ++g)
              if ((untouched >> g) & 1u) {
                int kr = 0;
#pragma unroll
                for (int q = 0; q < NG; ++q)
                  if (q == r) kr = rk[q];
                if ((rep_cert >> r) & 1u) {
                  coh |= 1u << g;
                  kg[g] = kr;
                }
                ++r;
              }
          }
          __syncwarp();
        }
        const unsigned long long reps = (unsigned long long)nrep * surf;
        if (coh) {
          const DevComp c = *cp;
          int assigned = 0;
#pragma unroll
          for (int q = 0; q < P; ++q) {
            const int g = 2 * q + half;
            const bool mine = ((coh >> g) & 1u) && ((usable >> q) & 1u);
            if (mine) {
              const int i = base + q * 32 + lane;
              const float4 p = a.spts[i];
              if (classify_coherent(a, c, i, p.x, p.y, p.z, half ? kg[2 * q + 1] : kg[2 * q]))
                done |= 1u << q;
            }
            assigned += __popc(__ballot_sync(0xffffffffu, mine));
          }
          if (lane == 0)
            atomicAdd((unsigned long long *)(a.counters + CNT_COHERENT), (unsigned long long)assigned);
        }
        if (lane == 0 && reps) {
          atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_EVAL), reps);
          atomicAdd((unsigned long long *)(a.counters + CNT_REP_PAIRS), reps);
        }
      } else if (a.coherence) {
        // Coherence (strip forms): where no triangle's box meets a box of
        // points, the surface does not cross that box (convex, hence
        // connected), so all its points have the winding number of any one of
        // them.  First the whole tile (representative: its first usable
        // point), then, if some triangle box meets the tile, each group of 16
        // points.  The tile's first usable point (positions are re-read from
        // memory, not held in registers across the hot loop):
        int first = -1;
#pragma unroll
        for (int q = P - 1; q >= 0; --q) {
          const uint32_t b = __ballot_sync(0xffffffffu, (usable >> q) & 1u);
          if (b) first = base + 32 * q + __ffs(b) - 1;
        }
        const float4 rp = a.spts[first];
        const float rx = rp.x, ry = rp.y, rz = rp.z;
        int k_t = 0, t_hit = -1, scanned = 0;
        unsigned long long reps = 0;
        const bool cert = rep_pass(a, cp, s_wbox[wid], rx, ry, rz, lane, &k_t, &t_hit);
        scanned = t_hit;
        if (cert) {
          coh = need;
#pragma unroll
          for (int g = 0; g < NG; ++g) kg[g] = k_t;
          reps += surf;
        } else if (t_hit < 0) {
          reps += surf;  // completed, but the representative is uncertain
        } else {
          reps += scanned;
          const uint32_t touched = touched_groups<NG>(a, cp, s_wbox[wid], s_gbox[wid], need, t_hit, lane);
          uint32_t untouched = need & ~touched;
          // an odd number of touched groups leaves half a slot of lanes free:
          // one untouched group is evaluated there instead of by its
          // representative
          if ((__popc(need & ~untouched) & 1) && untouched) untouched &= untouched - 1u;
          if (untouched) {
            // each group's first usable point, in shared memory for the pass
            uint32_t ub[P];
#pragma unroll
            for (int q = 0; q < P; ++q) ub[q] = __ballot_sync(0xffffffffu, (usable >> q) & 1u);
            if (lane == 0) {
#pragma unroll
              for (int g = 0; g < NG; ++g)
                if ((untouched >> g) & 1u) {
                  const uint32_t gl = (ub[g >> 1] >> (16 * (g & 1))) & 0xffffu;
                  const float4 gp = a.spts[base + 32 * (g >> 1) + 16 * (g & 1) + __ffs(gl) - 1];
                  s_rep[wid][g][0] = gp.x;
                  s_rep[wid][g][1] = gp.y;
                  s_rep[wid][g][2] = gp.z;
                }
            }
            __syncwarp();
            int kk[NG];
            const uint32_t gcert = group_reps<NG>(a, cp, untouched, s_rep[wid], lane, kk);
            __syncwarp();
#pragma unroll
            for (int g = 0; g < NG; ++g)
              if ((gcert >> g) & 1u) kg[g] = kk[g];
            coh |= gcert;
            reps += (unsigned long long)__popc(untouched) * surf;
          }
        }
        if (coh) {
          const DevComp c = *cp;
          int assigned = 0;
#pragma unroll
          for (int q = 0; q < P; ++q) {
            const int g = 2 * q + half;
            const bool mine = ((coh >> g) & 1u) && ((usable >> q) & 1u);
            if (mine) {
              const int i = base + q * 32 + lane;
              const float4 p = a.spts[i];
              if (classify_coherent(a, c, i, p.x, p.y, p.z, half ? kg[2 * q + 1] : kg[2 * q]))
                done |= 1u << q;
            }
            assigned += __popc(__ballot_sync(0xffffffffu, mine));
          }
          if (lane == 0)
            atomicAdd((unsigned long long *)(a.counters + CNT_COHERENT), (unsigned long long)assigned);
        }
        if (lane == 0 && reps) {
          atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_EVAL), reps);
          atomicAdd((unsigned long long *)(a.counters + CNT_REP_PAIRS), reps);
        }
      }
      const uint32_t act = need & ~coh;
      if (!act) continue;
      uint32_t list = 0;
      int m = 0;
#pragma unroll
      for (int g = 0; g < NG; ++g)
        if ((act >> g) & 1u) list |= (uint32_t)g << (4 * m++);
      bool ok = true;
      switch ((m + 1) >> 1) {
        case 1: ok = eval_groups<1, V, P>(a, cp, thr, wbuf, bar, ph0, ph1, lane, base, n, act, list, m, done, s_rng[wid], rtotal, rtris, nrng); break;
        case 2: ok = eval_groups<(P >= 2 ? 2 : 1), V, P>(a, cp, thr, wbuf, bar, ph0, ph1, lane, base, n, act, list, m, done, s_rng[wid], rtotal, rtris, nrng); break;
        case 3: ok = eval_groups<(P >= 3 ? 3 : 1), V, P>(a, cp, thr, wbuf, bar, ph0, ph1, lane, base, n, act, list, m, done, s_rng[wid], rtotal, rtris, nrng); break;
        default: ok = eval_groups<P, V, P>(a, cp, thr, wbuf, bar, ph0, ph1, lane, base, n, act, list, m, done, s_rng[wid], rtotal, rtris, nrng); break;
      }
      if (!ok) {
        timed_out = true;
        break;
      }
    }
    if (timed_out) {
      if (lane == 0) record_timeout(a.status, 1);
      // let copies still in flight land before the warp exits (bounded)
      mbar_wait(&bar[0], ph0);
      mbar_wait(&bar[1], ph1);
      return;
    }
  }
}

// ------------------------------------------------------------------ FP64 pieces
// Van Oosterom-Strackee half angle in FP64, the plain form of the method.
__device__ __forceinline__ double vos64_half(double px, double py, double pz, float4 A, float4 B, float4 C) {
  const double x1 = (double)A.x - px, y1 = (double)A.y - py, z1 = (double)A.z - pz;
  const double x2 = (double)B.x - px, y2 = (double)B.y - py, z2 = (double)B.z - pz;
  const double x3 = (double)C.x - px, y3 = (double)C.y - py, z3 = (double)C.z - pz;
  const double r1 = sqrt(x1 * x1 + y1 * y1 + z1 * z1);
  const double r2 = sqrt(x2 * x2 + y2 * y2 + z2 * z2);
  const double r3 = sqrt(x3 * x3 + y3 * y3 + z3 * z3);
  const double cx = y2 * z3 - z2 * y3, cy = z2 * x3 - x2 * z3, cz = x2 * y3 - y2 * x3;
  const double N = x1 * cx + y1 * cy + z1 * cz;
  const double d12 = x1 * x2 + y1 * y2 + z1 * z2;
  const double d13 = x1 * x3 + y1 * y3 + z1 * z3;
  const double d23 = x2 * x3 + y2 * y3 + z2 * z3;
  const double D = r1 * r2 * r3 + d12 * r3 + d13 * r2 + d23 * r1;
  return atan2(N, D);
}

// Plain FP64 kernel (the baseline): same work list and culling, triangles
// staged by TMA, every pair in FP64, no rescue needed.
template <int NT, int P>
__global__ void __launch_bounds__(NT) k_label64(LabelArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *sbuf = reinterpret_cast<float4 *>(smem_raw);  // 2 x kTriChunk x 3
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_item;
  const int tid = threadIdx.x;
  constexpr int TILE = NT * P;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;
  const int64_t n = a.counters[CNT_NIN];  // sorted points inside the union box
  const int64_t nitems = a.counters[CNT_ITEMS];
  for (;;) {
    if (tid == 0) s_item = (int64_t)atomicAdd((unsigned long long *)(a.counters + CNT_WORK), 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= nitems) break;
    const int2 w = a.items[item];
    const DevComp c = a.comps[w.y];
    const int64_t base = (int64_t)w.x * TILE;
    const float4 *gsrc = a.tris + (int64_t)c.tri_off * 3;
    const int nchunks = (c.tri_cnt + kTriChunk - 1) / kTriChunk;
    if (tid == 0) {
      int cnt0 = min(kTriChunk, c.tri_cnt);
      tma_load_1d(sbuf, gsrc, cnt0 * 48u, &bar[0]);
      if (nchunks > 1) {
        int cnt1 = min(kTriChunk, c.tri_cnt - kTriChunk);
        tma_load_1d(sbuf + 3 * kTriChunk, gsrc + 3 * kTriChunk, cnt1 * 48u, &bar[1]);
      }
    }
    double px[P], py[P], pz[P], acc[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      int64_t i = base + q * NT + tid;
      float4 p = a.spts[i < n ? i : base];
      px[q] = p.x;
      py[q] = p.y;
      pz[q] = p.z;
      acc[q] = 0.0;
    }
    bool timed_out = false;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int b = ch & 1;
      bool ok = mbar_wait(&bar[b], b ? ph1 : ph0);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      if (b) ph1 ^= 1; else ph0 ^= 1;
      const float4 *T = sbuf + b * 3 * kTriChunk;
      const int cnt = min(kTriChunk, c.tri_cnt - ch * kTriChunk);
      for (int t = 0; t < cnt; ++t) {
        const float4 A = T[3 * t], B = T[3 * t + 1], C = T[3 * t + 2];
#pragma unroll
        for (int q = 0; q < P; ++q) acc[q] += vos64_half(px[q], py[q], pz[q], A, B, C);
      }
      __syncthreads();
      if (tid == 0 && ch + 2 < nchunks) {
        int cnt2 = min(kTriChunk, c.tri_cnt - (ch + 2) * kTriChunk);
        tma_load_1d(sbuf + b * 3 * kTriChunk, gsrc + (int64_t)(ch + 2) * 3 * kTriChunk, cnt2 * 48u, &bar[b]);
      }
    }
    if (timed_out) {
      if (tid == 0) record_timeout(a.status, 2);
      mbar_wait(&bar[0], ph0);
      mbar_wait(&bar[1], ph1);
      return;
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int64_t i = base + q * NT + tid;
      if (i < n) {
        const double om = 2.0 * acc[q];
        const float fx = (float)px[q], fy = (float)py[q], fz = (float)pz[q];
        const bool fin = finite3(fx, fy, fz);
        const bool outside_box = fx < c.lo[0] || fx > c.hi[0] || fy < c.lo[1] || fy > c.hi[1] ||
                                 fz < c.lo[2] || fz > c.hi[2] ||
                                 dop_point_outside(fx, fy, fz, a.dop + (int64_t)w.y * kDop);
        float omf = (float)om;
        if (!fin) {
          omf = __int_as_float(0x7fc00000);
        } else if (outside_box) {
          omf = 0.f;
        } else if (om > 6.283185307179586476925) {
          atomicOr(a.in_mask + i, 1ull << c.row);
        }
        if (a.omega) a.omega[(int64_t)c.row * a.omega_ld + a.perm[i]] = omf;
      }
    }
    if (tid == 0) {
      const int64_t valid = min((int64_t)TILE, n - base);
      atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_EVAL), (unsigned long long)(valid * c.tri_cnt));
    }
  }
}

// FP64 re-evaluation.  Blocks take groups of 256 sorted points from a device
// cursor; the uncertain (point, compartment) pairs of a group are gathered in
// shared memory and each pair is summed by the whole block.  Thread k takes a
// contiguous segment of the compartment's strip stream and rebuilds its
// sliding window from the two entries before the segment, so the block walks
// the strips in parallel: per strip step one FP64 square root and the exact
// triple product N = R_a . (R_b x R_c) in double (the host-rounded normals
// are not used here).  The (D + i N) factors of 8 consecutive steps are
// multiplied with exact 2 pi wrap counting and one FP64 atan2 is taken per
// group; segment sums are reduced in a fixed order, so the result does not
// depend on scheduling.
constexpr int kRescueT = 256;
constexpr int kRescueG = 8;

// (cr, ci) = a b with the 2 pi wraps of the principal argument (sign bits of
// the imaginary parts, as in cmul_wrap)
__device__ __forceinline__ void cmul_wrap64(double ar, double ai, double br, double bi, double &cr, double &ci,
                                            int &k) {
  cr = fma(ar, br, -(ai * bi));
  ci = fma(ar, bi, ai * br);
  const uint32_t x = (uint32_t)(__double_as_longlong(ai) >> 32), y = (uint32_t)(__double_as_longlong(bi) >> 32),
                 z = (uint32_t)(__double_as_longlong(ci) >> 32);
  k += (int)((~x & ~y & z) >> 31) - (int)((x & y & ~z) >> 31);
}

// Omega / 2 over entries [s, e) of a strip stream, for the point (px, py, pz),
// returned as (angle sum, wraps)
__device__ void strip_half_angle64(const Entry *E, int s, int e, double px, double py, double pz, double *sum,
                                   int *wraps) {
  const float4 va = E[max(s - 2, 0)].v, vb = E[max(s - 1, 0)].v;
  double ax = (double)va.x - px, ay = (double)va.y - py, az = (double)va.z - pz;
  double bx = (double)vb.x - px, by = (double)vb.y - py, bz = (double)vb.z - pz;
  double ra = sqrt(ax * ax + ay * ay + az * az), rb = sqrt(bx * bx + by * by + bz * bz);
  double sab = ra * rb + (ax * bx + ay * by + az * bz);
  double acc = 0.0;
  int K = 0;
  for (int g = s; g < e; g += kRescueG) {
    double pr = 1.0, pi = 0.0;
    const int ge = min(g + kRescueG, e);
    for (int j = g; j < ge; ++j) {
      const float4 vc = E[j].v;
      const double cx = (double)vc.x - px, cy = (double)vc.y - py, cz = (double)vc.z - pz;
      const double rc = sqrt(cx * cx + cy * cy + cz * cz);
      const double dac = ax * cx + ay * cy + az * cz;
      const double dbc = bx * cx + by * cy + bz * cz;
      const double ux = by * cz - bz * cy, uy = bz * cx - bx * cz, uz = bx * cy - by * cx;
      // w = +-1: the window order keeps / reverses the triangle's orientation
      double N = (double)vc.w * (ax * ux + ay * uy + az * uz);
      double D = sab * rc + dac * rb + dbc * ra;
      if (vc.w == 0.f) {  // not a triangle of the surface: identity factor
        N = 0.0;
        D = 1.0;
      }
      double nr, ni;
      cmul_wrap64(pr, pi, D, N, nr, ni, K);
      pr = nr;
      pi = ni;
      sab = rb * rc + dbc;
      ax = bx; ay = by; az = bz;
      bx = cx; by = cy; bz = cz;
      ra = rb;
      rb = rc;
    }
    acc += atan2(pi, pr);
  }
  *sum = acc;
  *wraps = K;
}

// FP64 strip evaluation of one group of four cap-tree segment entries
// (positions pos .. pos + 3, a multiple of four: a group never straddles two
// segments) seen from p: the window enters the group as (E[pos-2], E[pos-1])
// (both in the same segment, since a segment starts at a multiple of four
// with its reset entry) or restarts at a reset entry; every window that is a
// triangle contributes the factor D + iN with N = w R_a . (R_b x R_c) (w the
// entry's orientation sign, the exact triple product of the stored
// vertices) and D = r_a r_b r_c + (R_a . R_b) r_c + (R_a . R_c) r_b +
// (R_b . R_c) r_a (Sec. 2.1.3), and the group returns the argument of the
// product with the 2 pi wraps of the partial products counted in *K exactly
// as the FP32 kernel does.
__device__ __forceinline__ bool sign64(double x) { return __double_as_longlong(x) < 0; }

__device__ double group64(const Entry *E, int pos, double px, double py, double pz, int *K) {
  double a[3], b[3], ra, rb;
  const float4 v0 = E[pos].v;
  if (v0.w == 2.f) {
    a[0] = b[0] = (double)v0.x - px;
    a[1] = b[1] = (double)v0.y - py;
    a[2] = b[2] = (double)v0.z - pz;
    ra = rb = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  } else {
    const float4 u = E[pos - 2].v, w = E[pos - 1].v;
    a[0] = (double)u.x - px; a[1] = (double)u.y - py; a[2] = (double)u.z - pz;
    b[0] = (double)w.x - px; b[1] = (double)w.y - py; b[2] = (double)w.z - pz;
    ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  }
  double R = 1.0, I = 0.0;
  bool have = false;
  int k = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = E[pos + q].v;
    const double c[3] = {(double)v.x - px, (double)v.y - py, (double)v.z - pz};
    const double rc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (fabsf(v.w) == 1.f) {
      const double N = (double)v.w * (a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                                      a[2] * (b[0] * c[1] - b[1] * c[0]));
      const double dab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
      const double dac = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
      const double dbc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
      const double D = ra * rb * rc + dab * rc + dac * rb + dbc * ra;
      if (!have) {
        R = D;
        I = N;
        have = true;
      } else {
        const double cr = R * D - I * N, ci = R * N + I * D;
        k += (!sign64(I) && !sign64(N) && sign64(ci)) ? 1 : 0;
        k -= (sign64(I) && sign64(N) && !sign64(ci)) ? 1 : 0;
        R = cr;
        I = ci;
      }
    }
    a[0] = b[0]; a[1] = b[1]; a[2] = b[2];
    b[0] = c[0]; b[1] = c[1]; b[2] = c[2];
    ra = rb;
    rb = rc;
  }
  *K += k;
  return have ? atan2(I, R) : 0.0;
}

// FP64 half-angle sum over the flattened entries [j0, j1) of a range list
// (multiples of four), the block's threads splitting the groups of four
// (fixed assignment and reduction order: deterministic); every thread of the
// block returns the block's total.
__device__ double block_sum64(const LabelArgs &a, const int2 *rng, int j0, int j1, double px, double py, double pz,
                              double *s_red, int *s_kred) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double part = 0.0;
  int K = 0;
  int r = 0, rb = 0;
  for (int j = j0 + 4 * tid; j < j1; j += 4 * kRescueT) part += group64(a.cseg, range_pos(rng, r, rb, j), px, py, pz, &K);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, o);
    K += __shfl_xor_sync(0xffffffffu, K, o);
  }
  if (lane == 0) {
    s_red[wid] = part;
    s_kred[wid] = K;
  }
  __syncthreads();
  double half = 0.0;
  int kt = 0;
#pragma unroll
  for (int w = 0; w < kRescueT / 32; ++w) {
    half += s_red[w];
    kt += s_kred[w];
  }
  __syncthreads();
  return half + 6.283185307179586476925 * (double)kt;
}

// Result of one FP64 re-evaluated pair: Omega, the inside bit, counters.
__device__ __forceinline__ void store64(const LabelArgs &a, int row, int64_t i, double half, int tris) {
  const double om = 2.0 * half;
  if (om > 6.283185307179586476925) atomicOr(a.in_mask + i, 1ull << row);
  if (a.omega) a.omega[(int64_t)row * a.omega_ld + a.perm[i]] = (float)om;
  atomicAdd((unsigned long long *)(a.counters + CNT_UNC), 1ull);
  atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_RESCUE), (unsigned long long)tris);
}

// FP64 re-evaluation over the cap tree by listed pair: the point's own
// range list (the tree walked for the point's zero-size box, so leaves near
// the point and caps of every farther node), group64 over it.  Outside a
// node's box its cap subtends its patch exactly, so the sum is Omega up to
// FP64 rounding.  GB300's FP64 pipe is slow, so when the list holds at most
// kSplitPairs pairs each pair is split into P parts (as many as the grid's
// blocks allow, at most kMaxParts): every part walks the tree, sums its
// share of the groups, and the last part to finish adds the partial sums in
// part order (deterministic) and stores the result.  Runs only when the list
// held every pair.
__global__ void __launch_bounds__(kRescueT) k_rescue64_list(LabelArgs a) {
  __shared__ int s_rowcomp[ZEF_MAX_COMPARTMENTS];
  __shared__ int64_t s_item;
  __shared__ double s_red[kRescueT / 32];
  __shared__ int s_kred[kRescueT / 32];
  __shared__ int2 s_rng[kMaxRanges];
  __shared__ int s_tot, s_tris;
  const int64_t npairs = a.counters[CNT_UNC_LIST];
  if (npairs > a.unc_cap) return;  // k_rescue64_caps takes them all
  int P = 1;
  if (npairs > 0 && npairs <= kSplitPairs) {
    const int64_t fit = (int64_t)gridDim.x / npairs;
    P = fit < 1 ? 1 : (fit > kMaxParts ? kMaxParts : (int)fit);
  }
  const int64_t nitems = npairs * P;
  const int tid = threadIdx.x;
  for (int c = tid; c < a.ncomp; c += blockDim.x) s_rowcomp[a.comps[c].row] = c;
  for (;;) {
    if (tid == 0) {
      const int64_t it = (int64_t)atomicAdd((unsigned long long *)(a.counters + CNT_UNC_WORK), 1ull);
      s_item = it;
      if (it < nitems) {
        const int2 e = a.unc_list[it / P];
        const float4 p = a.spts[e.x];
        const float box[6] = {p.x, p.y, p.z, p.x, p.y, p.z};
        int tot = 0, nt = 0;
        cap_ranges(a, a.comps + s_rowcomp[e.y], box, s_rng, &tot, &nt, true);
        s_tot = tot;
        s_tris = nt;
      }
    }
    __syncthreads();
    if (s_item >= nitems) break;
    const int64_t pair = s_item / P;
    const int part = (int)(s_item - pair * P);
    const int2 e = a.unc_list[pair];
    if (!ZEF_BOUNDS_OK(e.x >= 0 && e.x < a.counters[CNT_NIN] && e.y >= 0 && e.y < a.ncomp, a.status, 16)) {
      __syncthreads();
      continue;
    }
    const float4 p = a.spts[e.x];
    // this part's share of the groups of four
    const int groups = s_tot / 4;
    const int g0 = (int)((int64_t)groups * part / P), g1 = (int)((int64_t)groups * (part + 1) / P);
    const double half = block_sum64(a, s_rng, 4 * g0, 4 * g1, p.x, p.y, p.z, s_red, s_kred);
    if (tid == 0) {
      if (P == 1) {
        store64(a, e.y, e.x, half, s_tris);
      } else {
        a.unc_part[pair * kMaxParts + part] = half;
        __threadfence();
        if (atomicAdd(a.unc_done + pair, 1u) == (uint32_t)(P - 1)) {
          __threadfence();
          double h = 0.0;
          for (int q = 0; q < P; ++q) h += *(volatile double *)(a.unc_part + pair * kMaxParts + q);
          store64(a, e.y, e.x, h, s_tris);
        }
      }
    }
    __syncthreads();
  }
}

// The same re-evaluation by point groups (every uncertain pair of a group of
// kRescueT sorted points in turn), for calls whose uncertain pairs overflow
// the pair list.
__global__ void __launch_bounds__(kRescueT) k_rescue64_caps(LabelArgs a) {
  __shared__ int s_rowcomp[ZEF_MAX_COMPARTMENTS];
  __shared__ int64_t s_group;
  __shared__ int s_cnt;
  __shared__ int s_list[kRescueT];
  __shared__ unsigned long long s_mask[kRescueT];
  __shared__ double s_red[kRescueT / 32];
  __shared__ int s_kred[kRescueT / 32];
  __shared__ int2 s_rng[kMaxRanges];
  __shared__ int s_tot, s_tris;
  if (a.counters[CNT_UNC_LIST] <= a.unc_cap) return;  // k_rescue64_list took them
  const int tid = threadIdx.x;
  for (int c = tid; c < a.ncomp; c += blockDim.x) s_rowcomp[a.comps[c].row] = c;
  const int64_t n = a.counters[CNT_NIN];  // sorted points inside the union box
  const int64_t ngroups = (n + kRescueT - 1) / kRescueT;
  for (;;) {
    if (tid == 0) {
      s_group = (int64_t)atomicAdd((unsigned long long *)(a.counters + CNT_UNC_WORK), 1ull);
      s_cnt = 0;
    }
    __syncthreads();
    const int64_t g = s_group;
    if (g >= ngroups) break;
    const int64_t mine = g * kRescueT + tid;
    const unsigned long long m = mine < n ? a.unc_mask[mine] : 0ull;
    if (m) {
      const int k = atomicAdd(&s_cnt, 1);
      s_list[k] = tid;
      s_mask[k] = m;
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int e = 0; e < cnt; ++e) {
      const int64_t i = g * kRescueT + s_list[e];
      unsigned long long mm = s_mask[e];
      const float4 p = a.spts[i];
      while (mm) {
        const int row = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        if (tid == 0) {
          const float box[6] = {p.x, p.y, p.z, p.x, p.y, p.z};
          int tot = 0, nt = 0;
          cap_ranges(a, a.comps + s_rowcomp[row], box, s_rng, &tot, &nt, true);
          s_tot = tot;
          s_tris = nt;
        }
        __syncthreads();
        const double half = block_sum64(a, s_rng, 0, s_tot, p.x, p.y, p.z, s_red, s_kred);
        if (tid == 0) store64(a, row, i, half, s_tris);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRescueT) k_rescue64(LabelArgs a) {
  __shared__ int s_rowcomp[ZEF_MAX_COMPARTMENTS];
  __shared__ int64_t s_group;
  __shared__ int s_cnt;
  __shared__ int s_list[kRescueT];
  __shared__ unsigned long long s_mask[kRescueT];
  __shared__ double s_red[kRescueT / 32];
  __shared__ int s_kred[kRescueT / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int c = tid; c < a.ncomp; c += blockDim.x) s_rowcomp[a.comps[c].row] = c;
  const int64_t n = a.counters[CNT_NIN];  // sorted points inside the union box
  const int64_t ngroups = (n + kRescueT - 1) / kRescueT;
  for (;;) {
    if (tid == 0) {
      s_group = (int64_t)atomicAdd((unsigned long long *)(a.counters + CNT_UNC_WORK), 1ull);
      s_cnt = 0;
    }
    __syncthreads();
    const int64_t g = s_group;
    if (g >= ngroups) break;
    const int64_t mine = g * kRescueT + tid;
    const unsigned long long m = mine < n ? a.unc_mask[mine] : 0ull;
    if (m) {
      const int k = atomicAdd(&s_cnt, 1);
      s_list[k] = tid;
      s_mask[k] = m;
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int e = 0; e < cnt; ++e) {
      const int64_t i = g * kRescueT + s_list[e];
      unsigned long long mm = s_mask[e];
      const float4 p = a.spts[i];
      const double px = p.x, py = p.y, pz = p.z;
      unsigned long long set_bits = 0ull;
      while (mm) {
        const int row = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        const DevComp c = a.comps[s_rowcomp[row]];
        const Entry *E = a.entries + c.entry_off;
        const int seg = (c.entry_cnt + kRescueT - 1) / kRescueT;
        const int s0 = min(tid * seg, c.entry_cnt), e0 = min(s0 + seg, c.entry_cnt);
        double part = 0.0;
        int wraps = 0;
        if (s0 < e0) strip_half_angle64(E, s0, e0, px, py, pz, &part, &wraps);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          part += __shfl_xor_sync(0xffffffffu, part, o);
          wraps += __shfl_xor_sync(0xffffffffu, wraps, o);
        }
        if (lane == 0) {
          s_red[wid] = part;
          s_kred[wid] = wraps;
        }
        __syncthreads();
        double half = 0.0;
        int K = 0;
#pragma unroll
        for (int w = 0; w < kRescueT / 32; ++w) {
          half += s_red[w];
          K += s_kred[w];
        }
        __syncthreads();
        const double om = 2.0 * (half + 6.283185307179586476925 * K);
        if (om > 6.283185307179586476925) set_bits |= 1ull << row;
        if (tid == 0) {
          if (a.omega) a.omega[(int64_t)row * a.omega_ld + a.perm[i]] = (float)om;
          atomicAdd((unsigned long long *)(a.counters + CNT_UNC), 1ull);
          atomicAdd((unsigned long long *)(a.counters + CNT_PAIRS_RESCUE), (unsigned long long)c.tri_cnt);
        }
      }
      if (tid == 0 && set_bits) atomicOr(a.in_mask + i, set_bits);
    }
    __syncthreads();
  }
}

// Failure-detection probe: every thread waits on an mbarrier that nothing
// arrives on (no copy is issued), so the bounded wait must expire; the block
// records ST_TIMEOUT and returns.
__global__ void k_wait_probe(uint32_t *status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) record_timeout(status, 99);
}

// Element labels (Sec. 2.1.3, a tet belongs to S when its four nodes are
// inside dS; priority order of Sec. 2.1): the AND of the four nodes' inside
// bits (priority rows), first set bit -> id, 0 when none; -1 for a tet with a
// non-finite node, and for an index outside [0, n_nodes), which also records
// ST_INVALID.
__global__ void __launch_bounds__(256) k_elem_labels(const int32_t *tets, int64_t n_tets, int64_t n_nodes,
                                                     const int32_t *node_labels,
                                                     const unsigned long long *masks, const int32_t *row_ids,
                                                     int32_t *elem, uint32_t *status) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets;
       t += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long m = ~0ull;
    bool bad = false, nonfinite = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int32_t v = tets[4 * t + k];
      if (v < 0 || v >= n_nodes) {
        bad = true;
      } else {
        nonfinite |= node_labels[v] < 0;
        m &= masks[v];
      }
    }
    if (bad) atomicOr(status, ST_INVALID);
    elem[t] = (bad || nonfinite) ? -1 : (m ? row_ids[__ffsll((long long)m) - 1] : 0);
  }
}

// FMA throughput microbenchmark: kChains independent dependent-FMA chains
// per thread (enough to cover the pipe latency), `iters` rounds; the result
// is stored only when it equals an impossible value, so nothing is dead code.
template <class T>
__global__ void __launch_bounds__(256) k_debug_fma(int iters, T *sink) {
  constexpr int kChains = 8;
  T x[kChains];
  const T a = (T)0.999999, b = (T)1e-7;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.678) sink[0] = s;
}

// The FP32 atan2 of the label kernel applied elementwise (diagnostics: its
// error is measured against FP64 and CUDA's atan2f).
__global__ void k_debug_half_angle(const float *y, const float *x, float *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = half_angle(y[i], x[i]);
}

// ------------------------------------------------------------------ small kernels
__global__ void k_prepare(int64_t *cnt, int64_t n, int64_t off) {
  if (threadIdx.x == 0) {
    cnt[CNT_N] = n;
    cnt[CNT_OFF] = off;
  }
}

// Counters of one call (the point count and offset are already in place: set
// by k_prepare for host-known counts, by other kernels inside the refinement
// and re-labeling graphs), the work-bucket histogram and the completion
// counts of split FP64 re-evaluation pairs.
__global__ void __launch_bounds__(256) k_reset(int64_t *cnt, uint32_t *work_hist, uint32_t *unc_done) {
  if (threadIdx.x == 0) {
    cnt[CNT_ITEMS] = 0;
    cnt[CNT_WORK] = 0;
    cnt[CNT_UNC] = 0;
    cnt[CNT_UNC_WORK] = 0;
    cnt[CNT_NONFINITE] = 0;
    cnt[CNT_PAIRS_EVAL] = 0;
    cnt[CNT_PAIRS_RESCUE] = 0;
    cnt[CNT_COHERENT] = 0;
    cnt[CNT_REP_PAIRS] = 0;
    cnt[CNT_LANE_TILES] = 0;
    cnt[CNT_UNC_LIST] = 0;
    cnt[CNT_NIN] = 0;
    cnt[CNT_NFIN] = 0;
    cnt[CNT_TILES] = 0;
  }
  for (int j = threadIdx.x; j < kWorkBuckets; j += blockDim.x) work_hist[j] = 0u;
  if (unc_done)
    for (int j = threadIdx.x; j < kSplitPairs; j += blockDim.x) unc_done[j] = 0u;
}

// Warp-aggregated increment of ctr[key]: the lanes with equal keys share one
// atomic (neighbouring points often fall in one bucket); returns the counter
// before the increment plus the lane's rank among them.  Every lane of the
// warp calls it; lanes with valid = false take no part.
__device__ __forceinline__ uint32_t agg_inc(uint32_t *ctr, uint32_t key, bool valid, int lane) {
  const uint32_t k = valid ? key : 0xffffffffu;  // keys are below kHistLen
  const uint32_t peers = __match_any_sync(0xffffffffu, k);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (valid && lane == leader) base = atomicAdd(ctr + key, (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// Binning key of every point: the 21-bit Morton cell of the point in the
// union box of the registered surfaces (7 bits per axis), kKeyOutside for a
// finite point outside that box -- outside every compartment's box, so its
// winding number is 0 for every surface -- and kKeyNonfinite for a point with
// a NaN or infinite coordinate.  The points of the two tails are decided here
// (label 0, or -1 and NaN solid angles for the non-finite ones; zero inside
// bits) and take no further part: the sorted order holds the points inside
// the box alone.  Their counts are summed per block in shared memory and
// added once per block (all of them on one histogram word each: atomics of
// every warp on a few neighbouring words kept one L2 slice busy for most of
// the kernel).  Each warp takes kBinU runs of 32 consecutive points per
// pass, their loads and histogram increments issued together.
constexpr int kBinU = 4;

__global__ void __launch_bounds__(256) k_keys(const float *__restrict__ pts, int64_t *cnt, UnionBox ub,
                                             uint32_t *__restrict__ keys, uint32_t *hist,
                                             int32_t *__restrict__ labels, unsigned long long *masks_out,
                                             float *omega, int64_t omega_ld, int ncomp) {
  __shared__ uint32_t s_tail[2];  // outside the union box, non-finite
  if (threadIdx.x < 2) s_tail[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t n = cnt[CNT_N], off = cnt[CNT_OFF];
  const int lane = threadIdx.x & 31;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * kBinU;
  uint32_t n_out = 0, n_nonfin = 0;  // lane 0: the warp's tail points
  // warp-uniform loop: all lanes take part in the aggregated increments
  for (int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) * kBinU; w0 < n; w0 += step) {
    float v[kBinU][3];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      if (i < n) {
        const float *p = pts + 3 * (off + i);
        v[u][0] = p[0];
        v[u][1] = p[1];
        v[u][2] = p[2];
      }
    }
    uint32_t key[kBinU];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      key[u] = kKeyOutside;
      bool fin = true;
      if (i < n) {
        fin = finite3(v[u][0], v[u][1], v[u][2]);
        if (!fin) {
          key[u] = kKeyNonfinite;
        } else if (!(v[u][0] < ub.lo[0] || v[u][0] > ub.hi[0] || v[u][1] < ub.lo[1] || v[u][1] > ub.hi[1] ||
                     v[u][2] < ub.lo[2] || v[u][2] > ub.hi[2])) {
          uint32_t q[3];
#pragma unroll
          for (int k = 0; k < 3; ++k)
            q[k] = (uint32_t)min((int)((v[u][k] - ub.lo[k]) * ub.sc[k]), (1 << kMortonBits) - 1);
          key[u] = spread7(q[0]) | (spread7(q[1]) << 1) | (spread7(q[2]) << 2);
        }
        keys[i] = key[u];
        if (key[u] >= kKeyOutside) {
          labels[off + i] = fin ? 0 : -1;
          if (masks_out) masks_out[off + i] = 0ull;
          if (!fin && omega)
            for (int r = 0; r < ncomp; ++r) omega[(int64_t)r * omega_ld + i] = __int_as_float(0x7fc00000);
        }
      }
      n_out += __popc(__ballot_sync(0xffffffffu, i < n && fin && key[u] == kKeyOutside));
      n_nonfin += __popc(__ballot_sync(0xffffffffu, i < n && !fin));
    }
#pragma unroll
    for (int u = 0; u < kBinU; ++u) agg_inc(hist, key[u], w0 + 32 * u + lane < n && key[u] < kKeyOutside, lane);
  }
  if (lane == 0) {
    if (n_out) atomicAdd(&s_tail[0], n_out);
    if (n_nonfin) atomicAdd(&s_tail[1], n_nonfin);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_tail[0]) atomicAdd(hist + kKeyOutside, s_tail[0]);
    if (s_tail[1]) atomicAdd(hist + kKeyNonfinite, s_tail[1]);
  }
}

// Points inside the union box in key order, multiplied by the context's
// power-of-two scale (exact), with their permutation (their inside /
// uncertain masks are cleared by the tile pass, in sorted order).
__device__ __forceinline__ float scaled_coord(float x, float s) {
  return fminf(fmaxf(x * s, -3.0e38f), 3.0e38f);
}

__global__ void __launch_bounds__(256) k_scatter(const float *pts, int64_t *cnt, const uint32_t *keys,
                                                uint32_t *cursor, float4 *spts, int32_t *perm, float scale,
                                                uint32_t *status) {
  const int64_t n = cnt[CNT_N], off = cnt[CNT_OFF];
  const int lane = threadIdx.x & 31;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * kBinU;
  for (int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) * kBinU; w0 < n; w0 += step) {
    uint32_t key[kBinU];
    bool in[kBinU];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
      const int64_t i = w0 + 32 * u + lane;
      key[u] = i < n ? keys[i] : kKeyOutside;
      in[u] = key[u] < kKeyOutside;
    }
    float v[kBinU][3];
#pragma unroll
    for (int u = 0; u < kBinU; ++u)
      if (in[u]) {
        const float *p = pts + 3 * (off + w0 + 32 * u + lane);
        v[u][0] = p[0];
        v[u][1] = p[1];
        v[u][2] = p[2];
      }
    uint32_t pos[kBinU];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) pos[u] = agg_inc(cursor, key[u], in[u], lane);
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
      if (!in[u]) continue;
      if (!ZEF_BOUNDS_OK((int64_t)pos[u] < n, status, 17)) continue;
      spts[pos[u]] = make_float4(scaled_coord(v[u][0], scale), scaled_coord(v[u][1], scale),
                                 scaled_coord(v[u][2], scale), 0.f);
      perm[pos[u]] = (int32_t)(w0 + 32 * u + lane);
    }
  }
}

// Box of the points [b, e) of the sorted array, reduced over the warp (every
// lane returns it); empty: (+inf, -inf).  Also clears the points' inside and
// uncertain masks (coalesced, in sorted order).
__device__ __forceinline__ void warp_box(const float4 *spts, int64_t b, int64_t e, int lane, float *lo, float *hi,
                                         unsigned long long *in_mask, unsigned long long *unc_mask) {
  lo[0] = lo[1] = lo[2] = INFINITY;
  hi[0] = hi[1] = hi[2] = -INFINITY;
  for (int64_t i = b + lane; i < e; i += 32) {
    in_mask[i] = 0ull;
    unc_mask[i] = 0ull;
    const float4 p = spts[i];
    lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
}

// Bounding box of every tile of `tile` consecutive sorted points inside the
// union box (the plain FP64 kernel's tiles): one warp per tile.
__global__ void __launch_bounds__(256) k_tile_box(const float4 *spts, int64_t *cnt, float *tile_box, int tile,
                                                 unsigned long long *in_mask, unsigned long long *unc_mask) {
  const int64_t nin = cnt[CNT_NIN];
  const int64_t ntiles = cnt[CNT_TILES];
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles; t += warps) {
    float lo[3], hi[3];
    warp_box(spts, t * tile, min(t * tile + tile, nin), lane, lo, hi, in_mask, unc_mask);
    if (lane < 6) tile_box[t * 6 + lane] = lane < 3 ? lo[lane] : hi[lane - 3];
  }
}

__global__ void __launch_bounds__(256) k_flags(int64_t *cnt, const float *tile_box, const DevComp *comps,
                                              const int32_t *lpt, int ncomp, const float *dop, uint32_t *flags) {
  const int64_t ntiles = cnt[CNT_TILES];
  const int64_t len = ntiles * ncomp;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(j / ntiles);
    const int64_t t = j - (int64_t)r * ntiles;
    const DevComp &c = comps[lpt[r]];
    const float *b = tile_box + t * 6;
    const bool ov = !(b[3] < c.lo[0] || b[0] > c.hi[0] || b[4] < c.lo[1] || b[1] > c.hi[1] || b[5] < c.lo[2] ||
                      b[2] > c.hi[2]) &&
                    !dop_box_misses(b, dop + (int64_t)lpt[r] * kDop);
    flags[j] = ov ? 1u : 0u;
  }
}

__global__ void __launch_bounds__(256) k_emit(int64_t *cnt, const uint32_t *scan, const int32_t *lpt, int ncomp,
                                             int2 *items) {
  const int64_t ntiles = cnt[CNT_TILES];
  const int64_t len = ntiles * ncomp;
  const int64_t total = cnt[CNT_ITEMS];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nxt = (j + 1 < len) ? (int64_t)scan[j + 1] : total;
    if (nxt != (int64_t)scan[j]) {
      const int r = (int)(j / ntiles);
      const int64_t t = j - (int64_t)r * ntiles;
      items[scan[j]] = make_int2((int)t, lpt[r]);
    }
  }
}

// Work list of the FP32 kernel: every tile of `tile` (= 32 P) consecutive
// sorted points inside the union box whose box meets at least one
// compartment's box and convex-hull bound, largest estimated work (the sum of
// the met compartments' triangle counts) first, bucketed on a log scale
// (kWorkBuckets buckets).  One warp per tile: the lanes reduce the tile's box,
// then split the compartments.
constexpr uint32_t kNoWork = 0xffffffffu;

__global__ void __launch_bounds__(256) k_tile_work(const float4 *spts, int64_t *cnt, int tile, const DevComp *comps,
                                                  int ncomp, const float *dop, uint32_t *tile_key, uint32_t *hist,
                                                  unsigned long long *in_mask, unsigned long long *unc_mask) {
  const int64_t nin = cnt[CNT_NIN];
  const int64_t ntiles = cnt[CNT_TILES];
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles; t += warps) {
    float lo[3], hi[3];
    warp_box(spts, t * tile, min(t * tile + tile, nin), lane, lo, hi, in_mask, unc_mask);
    const float b[6] = {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]};
    float est = 0.f;
    for (int c0 = 0; c0 < ncomp; c0 += 32) {
      // box test: one compartment per lane; hull test of the met ones: the
      // whole warp per compartment
      const int c = c0 + lane;
      bool ov = false;
      if (c < ncomp) {
        const DevComp &d = comps[c];
        ov = !(b[3] < d.lo[0] || b[0] > d.hi[0] || b[4] < d.lo[1] || b[1] > d.hi[1] || b[5] < d.lo[2] ||
               b[2] > d.hi[2]);
      }
      uint32_t met = __ballot_sync(0xffffffffu, ov);
      while (met) {
        const int cc = c0 + __ffs(met) - 1;
        met &= met - 1;
        if (!dop_box_misses_warp(b, dop + (int64_t)cc * kDop, lane)) est += (float)__ldg(&comps[cc].tri_cnt);
      }
    }
    if (lane == 0) {
      uint32_t key = kNoWork;
      if (est > 0.f) {
        const int lg = (int)(__log2f(est) * 128.f);
        key = (uint32_t)(kWorkBuckets - 1 - min(kWorkBuckets - 1, max(0, lg)));
        atomicAdd(hist + key, 1u);
      }
      tile_key[t] = key;
    }
  }
}

__global__ void __launch_bounds__(256) k_tile_scatter(int64_t *cnt, const uint32_t *tile_key, uint32_t *cursor,
                                                     int2 *items, uint32_t *status) {
  const int64_t ntiles = cnt[CNT_TILES];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = tile_key[t];
    if (key == kNoWork) continue;
    const uint32_t pos = atomicAdd(cursor + key, 1u);
    if (!ZEF_BOUNDS_OK((int64_t)pos < ntiles, status, 19)) continue;
    items[pos] = make_int2((int)t, (int)key);
  }
}

// Labels in the caller's order of the points inside the union box (the
// sorted points): the first set bit of the priority-ordered inside mask -> id,
// 0 when none.  The points outside the box and the non-finite ones were
// labelled by k_keys.
__global__ void __launch_bounds__(256) k_resolve(LabelArgs a, int32_t *labels, const int32_t *row_ids) {
  const int64_t n = a.counters[CNT_N], off = a.counters[CNT_OFF], nfin = a.counters[CNT_NFIN];
  const int64_t nin = a.counters[CNT_NIN];
  if (blockIdx.x == 0 && threadIdx.x == 0) a.counters[CNT_NONFINITE] = n - nfin;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nin; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = a.perm[i];
    if (!ZEF_BOUNDS_OK(o >= 0 && o < n, a.status, 18)) continue;
    const unsigned long long m = a.in_mask[i];
    if (a.masks_out) a.masks_out[off + o] = m;
    labels[off + o] = m ? row_ids[__ffsll((long long)m) - 1] : 0;
  }
}

// ------------------------------------------------------------------ exclusive scan (uint32, in place)
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
  __shared__ uint32_t ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (wid == 0) {
    uint32_t s = lane < nw ? ws[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) ws[lane] = s;
  }
  __syncthreads();
  const uint32_t before = wid ? ws[wid - 1] : 0u;
  *total = ws[nw - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanT) k_scan_blocks(uint32_t *data, const int64_t *len_ptr, int64_t len_c,
                                                       int64_t len_mul, uint32_t *bsums) {
  const int64_t len = len_ptr ? (*len_ptr) * len_mul : len_c;
  const int64_t b0 = (int64_t)blockIdx.x * kScanB + (int64_t)threadIdx.x * kScanV;
  uint32_t v[kScanV];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanV; ++k) {
    v[k] = (b0 + k < len) ? data[b0 + k] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t pre = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanV; ++k) {
    if (b0 + k < len) data[b0 + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) bsums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t *bsums, const int64_t *len_ptr, int64_t len_c,
                                                   int64_t len_mul, int64_t *total_out) {
  const int64_t len = len_ptr ? (*len_ptr) * len_mul : len_c;
  const int64_t nb = (len + kScanB - 1) / kScanB;
  uint32_t carry = 0;
  for (int64_t b = 0; b < nb; b += blockDim.x) {
    const int64_t j = b + threadIdx.x;
    uint32_t v = j < nb ? bsums[j] : 0u;
    uint32_t tot;
    uint32_t pre = block_excl_scan(v, &tot);
    if (j < nb) bsums[j] = carry + pre;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = (int64_t)carry;
}

__global__ void __launch_bounds__(kScanT) k_scan_add(uint32_t *data, const int64_t *len_ptr, int64_t len_c,
                                                    int64_t len_mul, const uint32_t *bsums) {
  const int64_t len = len_ptr ? (*len_ptr) * len_mul : len_c;
  const int64_t b0 = (int64_t)blockIdx.x * kScanB + (int64_t)threadIdx.x * kScanV;
  const uint32_t add = bsums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanV; ++k)
    if (b0 + k < len) data[b0 + k] += add;
}

// k_scan_add of the key histogram (kHistLen entries), which also records
// where the sorted order's tails start -- the first position of the points
// outside the union box (= the points inside it) and of the non-finite
// points -- and the tile count of the points inside.
__global__ void __launch_bounds__(kScanT) k_scan_add_keys(uint32_t *data, const uint32_t *bsums, int64_t *cnt,
                                                         int tile) {
  const int64_t b0 = (int64_t)blockIdx.x * kScanB + (int64_t)threadIdx.x * kScanV;
  const uint32_t add = bsums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanV; ++k) {
    const int64_t j = b0 + k;
    if (j < kHistLen) {
      const uint32_t v = data[j] + add;
      data[j] = v;
      if (j == (int64_t)kKeyOutside) {
        cnt[CNT_NIN] = v;
        cnt[CNT_TILES] = ((int64_t)v + tile - 1) / tile;
      } else if (j == (int64_t)kKeyNonfinite) {
        cnt[CNT_NFIN] = v;
      }
    }
  }
}

// Exclusive scan of the kWorkBuckets work histogram by one block; the total
// (work items) goes to *total_out.
__global__ void __launch_bounds__(1024) k_scan_work(uint32_t *data, int64_t *total_out) {
  constexpr int V = kWorkBuckets / 1024;
  uint32_t v[V];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    v[k] = data[threadIdx.x * V + k];
    s += v[k];
  }
  uint32_t tot;
  uint32_t pre = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < V; ++k) {
    data[threadIdx.x * V + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) *total_out = (int64_t)tot;
}
static_assert(kWorkBuckets % 1024 == 0, "k_scan_work: whole values per thread");

// ------------------------------------------------------------------ launch helpers
template <int NT, int P, int V>
zef_status launch_label32(zef_ctx *ctx, const LabelArgs &a) {
  const size_t smem = (size_t)(NT / 32) * 2 * kWChunk * sizeof(Entry);
  auto kern = k_label32<NT, P, V>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
  if (occ < 1) occ = 1;
  kern<<<ctx->num_sms * occ, NT, smem, ctx->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_label32 launch");
  return ZEF_OK;
}

template <int NT, int P>
zef_status launch_label64(zef_ctx *ctx, const LabelArgs &a) {
  const size_t smem = 2 * kTriChunk * 3 * sizeof(float4);
  auto kern = k_label64<NT, P>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
  if (occ < 1) occ = 1;
  kern<<<ctx->num_sms * occ, NT, smem, ctx->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_label64 launch");
  return ZEF_OK;
}

template <int V>
zef_status dispatch_variant(zef_ctx *ctx, const LabelArgs &a, LaunchShape s) {
  if (s.threads == 256) return s.ppt == 2 ? launch_label32<256, 2, V>(ctx, a) : launch_label32<256, 4, V>(ctx, a);
  return s.ppt == 2 ? launch_label32<128, 2, V>(ctx, a) : launch_label32<128, 4, V>(ctx, a);
}

zef_status dispatch_label32(zef_ctx *ctx, const LabelArgs &a, LaunchShape s) {
  if (s.variant == 2) return dispatch_variant<2>(ctx, a, s);
  return s.variant == 1 ? dispatch_variant<1>(ctx, a, s) : dispatch_variant<0>(ctx, a, s);
}

int grid_for(zef_ctx *ctx, int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

zef_status scan_inplace(zef_ctx *ctx, uint32_t *data, const int64_t *len_ptr, int64_t len_mul, int64_t len_cap,
                        int64_t *total_out) {
  const int64_t nb = std::max<int64_t>(1, (len_cap + kScanB - 1) / kScanB);
  const int64_t len_c = len_ptr ? 0 : len_cap;
  k_scan_blocks<<<(unsigned)nb, kScanT, 0, ctx->stream>>>(data, len_ptr, len_c, len_mul, ctx->lb.block_sums);
  k_scan_sums<<<1, 1024, 0, ctx->stream>>>(ctx->lb.block_sums, len_ptr, len_c, len_mul, total_out);
  k_scan_add<<<(unsigned)nb, kScanT, 0, ctx->stream>>>(data, len_ptr, len_c, len_mul, ctx->lb.block_sums);
  ctx->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan launch");
  return ZEF_OK;
}

// Exclusive scan of the key histogram, recording the tails of the sorted
// order and the tile count (k_scan_add_keys).
zef_status scan_keys(zef_ctx *ctx, uint32_t *hist, int tile) {
  const int64_t nb = (kHistLen + kScanB - 1) / kScanB;
  k_scan_blocks<<<(unsigned)nb, kScanT, 0, ctx->stream>>>(hist, nullptr, kHistLen, 1, ctx->lb.block_sums);
  k_scan_sums<<<1, 1024, 0, ctx->stream>>>(ctx->lb.block_sums, nullptr, kHistLen, 1, nullptr);
  k_scan_add_keys<<<(unsigned)nb, kScanT, 0, ctx->stream>>>(hist, ctx->lb.block_sums, ctx->lb.counters, tile);
  ctx->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "key scan launch");
  return ZEF_OK;
}

}  // namespace

// ------------------------------------------------------------------ host API of this file
// Exclusive in-place scan of uint32 data (length *len_ptr * len_mul, or
// len_cap when len_ptr is null) using `bsums` (>= len_cap / 2048 + 1 words)
// for the block sums; the total goes to *total_out when non-null.
zef_status scan_exclusive(zef_ctx *ctx, uint32_t *data, const int64_t *len_ptr, int64_t len_mul,
                          int64_t len_cap, int64_t *total_out, uint32_t *bsums) {
  const int64_t nb = std::max<int64_t>(1, (len_cap + kScanB - 1) / kScanB);
  const int64_t len_c = len_ptr ? 0 : len_cap;
  k_scan_blocks<<<(unsigned)nb, kScanT, 0, ctx->stream>>>(data, len_ptr, len_c, len_mul, bsums);
  k_scan_sums<<<1, 1024, 0, ctx->stream>>>(bsums, len_ptr, len_c, len_mul, total_out);
  k_scan_add<<<(unsigned)nb, kScanT, 0, ctx->stream>>>(data, len_ptr, len_c, len_mul, bsums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan launch");
  return ZEF_OK;
}

int grid_blocks(zef_ctx *ctx, int64_t work, int threads) { return grid_for(ctx, work, threads); }

bool shape_valid(int threads, int ppt) {
  return (threads == 128 || threads == 256) && (ppt == 2 || ppt == 4);
}

void fill_default_opts(zef_label_opts *o) {
  if (!(o->margin > 0.f)) o->margin = 1e-3f;
  if (!(o->winding_tol > 0.f)) o->winding_tol = 1e-5f;
}

// ------------------------------------------------------------------ autotuner
// The launch shape trades per-pair efficiency (points per thread, warps per
// SM) against culling (smaller tiles of Morton-ordered points overlap fewer
// compartment boxes), so the best shape depends on the geometry.  The tuner
// times every candidate on a strided sample of the call's own points (at most
// 2^20, so the one-time cost stays a fraction of a full call) and caches the
// winner under a key of (point-count octave, compartments, total triangles,
// precision, kernel form).
namespace {

constexpr LaunchShape kCandidates[] = {{256, 4}, {256, 2}, {128, 4}, {128, 2}};
constexpr int64_t kTunePoints = 1 << 20;

uint64_t tune_key(zef_ctx *ctx, const zef_label_opts &o, int64_t n) {
  int oct = 0;
  while ((int64_t(1) << (oct + 1)) <= n) ++oct;
  int64_t tt = 0;
  for (const CompHost &c : ctx->comps) tt += c.nt;
  uint64_t k = (uint64_t)oct;
  k = k * 131 + ctx->comps.size();
  k = k * 1000003 + (uint64_t)tt;
  k = k * 7 + (uint64_t)o.precision;
  k = k * 3 + (uint64_t)o.kernel;
  return k;
}

__global__ void __launch_bounds__(256) k_gather_stride(const float *pts, int64_t stride, int64_t m, float *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float *p = pts + 3 * i * stride;
    out[3 * i] = p[0];
    out[3 * i + 1] = p[1];
    out[3 * i + 2] = p[2];
  }
}

}  // namespace

LaunchShape choose_shape(zef_ctx *ctx, const zef_label_opts &o, int64_t n, bool *need_tune) {
  *need_tune = false;
  if (o.precision == ZEF_FP64_PLAIN) return LaunchShape{128, 2};
  if (o.block_threads && o.points_per_thread)
    return LaunchShape{o.block_threads, o.points_per_thread, kernel_variant(o.kernel)};
  const uint64_t key = tune_key(ctx, o, n);
  for (const auto &kv : ctx->tune_cache)
    if (kv.first == key) return kv.second;
  *need_tune = n >= 4096;  // small calls: not worth timing
  return LaunchShape{256, 2, kernel_variant(o.kernel)};
}

// plan.pts must be device memory with plan.n_cap points at offset 0.
zef_status autotune(zef_ctx *ctx, const LabelPlan &plan, LaunchShape *best) {
  LabelBuffers &b = ctx->lb;
  const int64_t n = plan.n_cap;
  const int64_t stride = (n + kTunePoints - 1) / kTunePoints;
  const int64_t m = (n + stride - 1) / stride;
  if (!b.tune_pts) {
    cudaError_t ea = cudaMalloc(&b.tune_pts, (size_t)kTunePoints * 3 * sizeof(float));
    if (ea != cudaSuccess) return cuda_fail(ctx, ea, "cudaMalloc(tune sample)");
  }
  k_gather_stride<<<grid_for(ctx, m, 256), 256, 0, ctx->stream>>>(plan.pts, stride, m, b.tune_pts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_gather_stride launch");
  float best_ms = 3.0e38f;
  LaunchShape pick{256, 2, kernel_variant(plan.opts.kernel)};
  for (const LaunchShape &c0 : kCandidates) {
    LaunchShape c = c0;
    c.variant = kernel_variant(plan.opts.kernel);
    LabelPlan p = plan;
    p.pts = b.tune_pts;
    p.labels = b.labels_tmp;
    p.omega = nullptr;
    p.omega_ld = 0;
    p.n_cap = m;
    p.shape = c;
    p.timed = false;
    float ms_min = 3.0e38f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run also loads the kernel
      zef_status st = label_set_count(ctx, m, 0);
      if (st) return st;
      cudaEventRecord(ctx->ev[0], ctx->stream);
      st = label_enqueue(ctx, p);
      if (st) return st;
      cudaEventRecord(ctx->ev[5], ctx->stream);
      e = cudaEventSynchronize(ctx->ev[5]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[5]);
      if (rep > 0) ms_min = std::min(ms_min, ms);
    }
    if (ms_min < best_ms) {
      best_ms = ms_min;
      pick = c;
    }
  }
  ctx->tune_cache.emplace_back(tune_key(ctx, plan.opts, n), pick);
  *best = pick;
  return ZEF_OK;
}

zef_status label_reserve(zef_ctx *ctx, int64_t n_cap) {
  LabelBuffers &b = ctx->lb;
  const int C = (int)ctx->comps.size();
  const int64_t min_tile = 32 * 2;  // smallest tile of any launch shape
  const int64_t tiles = (n_cap + min_tile - 1) / min_tile;
  zef_status st;
  if (b.cap_points < n_cap) {
    int64_t cap = std::max<int64_t>(n_cap, 1024);
    auto realloc = [&](void **p, size_t bytes) -> zef_status {
      if (*p) cudaFree(*p);
      *p = nullptr;
      cudaError_t e = cudaMalloc(p, bytes);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(label buffers)");
      return ZEF_OK;
    };
    if ((st = realloc((void **)&b.spts, cap * sizeof(float4)))) return st;
    if ((st = realloc((void **)&b.perm, cap * sizeof(int32_t)))) return st;
    if ((st = realloc((void **)&b.keys, cap * sizeof(uint32_t)))) return st;
    if ((st = realloc((void **)&b.in_mask, cap * sizeof(unsigned long long)))) return st;
    if ((st = realloc((void **)&b.unc_mask, cap * sizeof(unsigned long long)))) return st;
    if ((st = realloc((void **)&b.labels_tmp, cap * sizeof(int32_t)))) return st;
    if ((st = realloc((void **)&b.pts_tmp, cap * 3 * sizeof(float)))) return st;
    b.cap_points = cap;
  }
  const int64_t need_flags = std::max<int64_t>(tiles * std::max(C, 1), kHistLen);
  if (b.cap_tiles < tiles || b.cap_items < need_flags) {
    if (b.tile_box) cudaFree(b.tile_box);
    if (b.flags) cudaFree(b.flags);
    if (b.items) cudaFree(b.items);
    if (b.block_sums) cudaFree(b.block_sums);
    b.tile_box = nullptr;
    b.flags = nullptr;
    b.items = nullptr;
    b.block_sums = nullptr;
    b.cap_tiles = b.cap_items = 0;
    const int64_t ft = std::max<int64_t>(tiles, 1);
    cudaError_t e;
    if ((e = cudaMalloc(&b.tile_box, ft * 6 * sizeof(float))) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    if ((e = cudaMalloc(&b.flags, need_flags * sizeof(uint32_t))) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    if ((e = cudaMalloc(&b.items, need_flags * sizeof(int2))) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    if ((e = cudaMalloc(&b.block_sums, scan_block_sums(need_flags) * sizeof(uint32_t))) != cudaSuccess)
      return cuda_fail(ctx, e, "cudaMalloc");
    b.cap_tiles = ft;
    b.cap_items = need_flags;
  }
  if (!b.hist) {
    cudaError_t e = cudaMalloc(&b.hist, (size_t)(kHistLen + kWorkBuckets) * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(hist)");
  }
  if (!b.unc_list) {
    cudaError_t e = cudaMalloc(&b.unc_list, kUncBytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(uncertain pairs)");
    b.cap_unc = kUncListCap;
  }
  if (!b.counters) {
    cudaError_t e = cudaMalloc(&b.counters, CNT_COUNT_ * sizeof(int64_t));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(counters)");
    cudaMemset(b.counters, 0, CNT_COUNT_ * sizeof(int64_t));
  }
  return ZEF_OK;
}

// Enqueue the whole labeling pipeline (no host synchronisation).  When
// plan.d_n / plan.d_off point into the counters they must already hold the
// call's values; label_points sets them with k_prepare.
zef_status label_enqueue(zef_ctx *ctx, const LabelPlan &plan) {
  LabelBuffers &b = ctx->lb;
  const int C = (int)ctx->comps.size();
  // FP32: tiles of one warp (32 x P points); plain FP64: tiles of one block
  const int tile = plan.opts.precision == ZEF_FP64_PLAIN ? plan.shape.threads * plan.shape.ppt
                                                         : 32 * plan.shape.ppt;
  cudaStream_t s = ctx->stream;
  uint32_t *work_hist = b.hist + kHistLen;
  double *unc_part = b.unc_list ? reinterpret_cast<double *>(b.unc_list + kUncListCap) : nullptr;
  uint32_t *unc_done = b.unc_list ? reinterpret_cast<uint32_t *>(unc_part + (size_t)kSplitPairs * kMaxParts) : nullptr;
  int64_t launches = 0;
  NvtxRange nvtx_stage("zef.binning");
  if (plan.timed) cudaEventRecord(ctx->ev[0], s);
  k_reset<<<1, 256, 0, s>>>(b.counters, work_hist, unc_done);
  ++launches;
  // Omega of (point, compartment) pairs culled by the bounding boxes is 0
  if (plan.omega) cudaMemsetAsync(plan.omega, 0, (size_t)C * plan.omega_ld * sizeof(float), s);
  const int64_t ncap = plan.n_cap;
  const int g = grid_for(ctx, ncap, 256);
  // binning: keys in the surfaces' union box, key histogram, scan, scatter
  cudaMemsetAsync(b.hist, 0, (size_t)kHistLen * sizeof(uint32_t), s);
  k_keys<<<g, 256, 0, s>>>(plan.pts, b.counters, ctx->ubox, b.keys, b.hist, plan.labels, plan.masks, plan.omega,
                           plan.omega_ld, C);
  ++launches;
  zef_status st = scan_keys(ctx, b.hist, tile);
  if (st) return st;
  k_scatter<<<g, 256, 0, s>>>(plan.pts, b.counters, b.keys, b.hist, b.spts, b.perm, ctx->scale, ctx->d_status);
  ++launches;
  const int64_t tiles_cap = (ncap + tile - 1) / tile;
  const int gt = grid_for(ctx, tiles_cap * 32, 256);  // one warp per tile
  if (plan.opts.precision == ZEF_FP64_PLAIN) {
    // (tile, compartment) items for the plain FP64 kernel
    k_tile_box<<<gt, 256, 0, s>>>(b.spts, b.counters, b.tile_box, tile, b.in_mask, b.unc_mask);
    k_flags<<<grid_for(ctx, tiles_cap * C, 256), 256, 0, s>>>(b.counters, b.tile_box, ctx->d_comps, ctx->d_lpt, C,
                                                               ctx->d_dop, b.flags);
    launches += 2;
    st = scan_inplace(ctx, b.flags, b.counters + CNT_TILES, C, tiles_cap * C, b.counters + CNT_ITEMS);
    if (st) return st;
    k_emit<<<grid_for(ctx, tiles_cap * C, 256), 256, 0, s>>>(b.counters, b.flags, ctx->d_lpt, C, b.items);
    ++launches;
  } else {
    // tile items, largest estimated work first
    k_tile_work<<<gt, 256, 0, s>>>(b.spts, b.counters, tile, ctx->d_comps, C, ctx->d_dop, b.flags, work_hist,
                                   b.in_mask, b.unc_mask);
    k_scan_work<<<1, 1024, 0, s>>>(work_hist, b.counters + CNT_ITEMS);
    k_tile_scatter<<<grid_for(ctx, tiles_cap, 256), 256, 0, s>>>(b.counters, b.flags, work_hist, b.items,
                                                                 ctx->d_status);
    launches += 3;
  }

  LabelArgs a;
  a.entries = ctx->d_entries;
  a.tris = ctx->d_tris;
  a.comps = ctx->d_comps;
  a.spts = b.spts;
  a.perm = b.perm;
  a.items = b.items;
  a.tile_box = b.tile_box;
  a.dop = ctx->d_dop;
  a.in_mask = b.in_mask;
  a.unc_mask = b.unc_mask;
  a.omega = plan.omega;
  a.omega_ld = plan.omega_ld;
  a.counters = b.counters;
  a.status = ctx->d_status;
  a.margin = plan.opts.margin;
  a.winding_tol = plan.opts.winding_tol;
  a.ncomp = C;
  a.fp32_only = plan.opts.precision == ZEF_FP32_ONLY;
  a.coherence = !(plan.opts.flags & ZEF_NO_TILE_COHERENCE);
  a.lane_walk = (plan.opts.flags & ZEF_POINT_WALK) ? 0 : 1;
  a.omega_raw = (plan.opts.flags & ZEF_OMEGA_RAW) ? 1 : 0;
  a.early = plan.omega == nullptr && !plan.full_masks;
  a.nodes = ctx->d_nodes;
  a.cseg = ctx->d_cseg;
  // the pair list serves the cap-tree form's FP64 re-evaluation
  const bool pair_list = plan.shape.variant == 2 && plan.opts.precision == ZEF_FP32_RESCUE && b.unc_list;
  a.unc_list = pair_list ? b.unc_list : nullptr;
  a.unc_cap = pair_list ? b.cap_unc : 0;
  a.unc_part = unc_part;
  a.unc_done = unc_done;
  a.masks_out = plan.masks;
  a.n_nodes = (int64_t)ctx->h_nodes.size();
  a.n_cseg = (int64_t)ctx->h_cseg.size();
  nvtx_stage.next("zef.label_kernel");
  if (plan.timed) cudaEventRecord(ctx->ev[1], s);
  if (plan.opts.precision == ZEF_FP64_PLAIN) {
    // the FP64 kernel's tile is 128 x 2 points (choose_shape guarantees it)
    if (tile != 256) return fail(ctx, ZEF_ERR_INVALID_ARG, "internal: FP64 tile");
    st = launch_label64<128, 2>(ctx, a);
  } else {
    st = dispatch_label32(ctx, a, plan.shape);
  }
  if (st) return st;
  ++launches;
  if (plan.timed) cudaEventRecord(ctx->ev[2], s);
  nvtx_stage.next("zef.rescue64");
  if (plan.timed) cudaEventRecord(ctx->ev[3], s);
  if (plan.opts.precision == ZEF_FP32_RESCUE) {
    if (pair_list) {
      // the pair list when it holds every uncertain pair, else by point groups
      k_rescue64_list<<<ctx->num_sms * 4, kRescueT, 0, s>>>(a);
      k_rescue64_caps<<<ctx->num_sms * 4, kRescueT, 0, s>>>(a);
      launches += 2;
    } else {
      k_rescue64<<<ctx->num_sms * 4, kRescueT, 0, s>>>(a);
      ++launches;
    }
  }
  if (plan.timed) cudaEventRecord(ctx->ev[4], s);
  nvtx_stage.next("zef.resolve");
  k_resolve<<<g, 256, 0, s>>>(a, plan.labels, ctx->d_row_ids);
  ++launches;
  if (plan.timed) cudaEventRecord(ctx->ev[5], s);
  // scan_keys and scan_inplace counted their own launches
  ctx->launches += launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "label pipeline launch");
  return ZEF_OK;
}

zef_status launch_wait_probe(zef_ctx *ctx, int64_t limit_ns) {
  k_wait_probe<<<1, 64, 0, ctx->stream>>>(ctx->d_status, (unsigned long long)limit_ns);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_wait_probe launch");
  return ZEF_OK;
}

zef_status launch_elem_labels(zef_ctx *ctx, const int32_t *tets, int64_t n_tets, int64_t n_nodes,
                              const int32_t *node_labels, const unsigned long long *masks, int32_t *elem) {
  if (n_tets > 0)
    k_elem_labels<<<grid_blocks(ctx, n_tets, 256), 256, 0, ctx->stream>>>(tets, n_tets, n_nodes, node_labels, masks,
                                                                          ctx->d_row_ids, elem, ctx->d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_elem_labels launch");
  return ZEF_OK;
}

zef_status debug_fma_rate(zef_ctx *ctx, int fp64, double *tflops) {
  const int blocks = ctx->num_sms * 8, threads = 256, iters = fp64 ? 256 : 4096;
  void *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, 16);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(sink)");
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    cudaEventRecord(t0, ctx->stream);
    if (fp64) k_debug_fma<double><<<blocks, threads, 0, ctx->stream>>>(iters, (double *)sink);
    else k_debug_fma<float><<<blocks, threads, 0, ctx->stream>>>(iters, (float *)sink);
    cudaEventRecord(t1, ctx->stream);
    e = cudaEventSynchronize(t1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(sink);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_debug_fma");
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return ZEF_OK;
}

zef_status launch_debug_half_angle(zef_ctx *ctx, const float *y, const float *x, float *out, int64_t n) {
  if (n > 0) {
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)(want < 4096 ? want : 4096);
    k_debug_half_angle<<<blocks, 256, 0, ctx->stream>>>(y, x, out, n);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_debug_half_angle launch");
  return ZEF_OK;
}

// Set the point count and offset of a label_points call (host-known values).
zef_status label_set_count(zef_ctx *ctx, int64_t n, int64_t off) {
  k_prepare<<<1, 32, 0, ctx->stream>>>(ctx->lb.counters, n, off);
  ++ctx->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_prepare launch");
  return ZEF_OK;
}

}  // namespace zef

namespace zef {

// Convex-hull bound directions into this device's constant memory (once per
// context, at creation; the device is current).
zef_status upload_dop_directions(zef_ctx *ctx) {
  float dirs[kDop][3];
  dop_directions(dirs);
  cudaError_t e = cudaMemcpyToSymbol(c_dop, dirs, sizeof(dirs));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dop, dirs, sizeof(dirs));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload hull directions");
  return ZEF_OK;
}

}  // namespace zef
