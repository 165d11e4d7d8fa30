/*
 * zef_debug.h -- diagnostic entry points of libzef (same conventions as
 * zef.h).  They expose internal data for tests and tuning; the paper has no
 * counterpart for them.
 */
#ifndef ZEF_DEBUG_H
#define ZEF_DEBUG_H

#include "zef.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Strip stream of registered compartment `index` (registration order).
   Each entry is 8 floats: the vertex entering the sliding triangle window
   (x, y, z), a weight (+1 when the window (a, b, c) is a surface triangle
   in its own orientation, -1 when it is the triangle (a, c, b), 0 when the
   window is not a triangle: the two entries that start the stream, strip
   restarts and padding, whose windows repeat a vertex), that triangle's
   doubled-area normal (x, y, z) with the surface orientation, and
   kappa * |normal| (normal and kappa term are 0 when the weight is 0).  Writes min(count, cap) entries to `out` (host,
   nullable) and the entry count to *count.  Works on host-only contexts. */
zef_status zef_debug_strip_entries(const zef_ctx *ctx, int32_t index, float *out, int64_t cap,
                                   int64_t *count);

/* Entry and strip counts of compartment `index`. */
zef_status zef_debug_strip_stats(const zef_ctx *ctx, int32_t index, int64_t *entries, int64_t *strips);

/* The label kernel's FP32 atan2: out[i] = atan2(y[i], x[i]) in (-pi, pi],
   computed by the same device function the FP32 kernel applies to the
   Van Oosterom-Strackee pair (N, D) of Sec. 2.1.3 (range reduction to
   min/max in [0, 1], a minimax polynomial of degree 8 in x^2, octant
   reflections).  y, x, out: n floats each in device memory of the context's
   device; synchronizes.  Denormal inputs are flushed to zero.  Errors:
   ZEF_ERR_INVALID_ARG (null or host arrays, n < 0), ZEF_ERR_NOT_READY on a
   host-only context. */
zef_status zef_debug_half_angle(zef_ctx *ctx, const float *y, const float *x, float *out, int64_t n);

/* Cap tree of compartment `index` (registration order), unscaled: for each
   node its box (lo x, y, z, hi x, y, z of the patch's vertices) and nine
   int32 (left child, right child (-1 for a leaf), first entry and entry
   count of the leaf's strip segment (0, 0 for an inner node), first entry
   and entry count of the node's cap segment, triangles of the leaf segment,
   triangles of the cap segment, the node after its subtree in pre-order;
   nodes and entries relative to the compartment's block); the block's entries as 8 floats each (vertex x, y, z, weight;
   n x, y, z, kappa |n|), weight 2 opening a segment, +-1 closing a
   triangle window in its own / reversed orientation, 0 for the windows that
   repeat a vertex.  *n_nodes and *n_entries receive the counts; the arrays
   (nullable) must hold them.  The identity the tree serves: outside a
   node's box, the solid angle of the node's leaf triangles equals that of
   its cap triangles.  Works on host-only contexts. */
zef_status zef_debug_cap_tree(const zef_ctx *ctx, int32_t index, int64_t *n_nodes, int64_t *n_entries,
                              float *boxes, int32_t *links, float *entries);

/* Measured fused multiply-add throughput of the context's device in TFLOP/s
   (FMA = 2 flops): float (fp64 = 0) or double (fp64 != 0), 8 independent
   chains per thread on SMs x 8 blocks of 256 threads, best of three timed
   launches after a warm-up.  Synchronizes.  Used to check the FP32 peak the
   label kernel is compared with and to measure the FP64 rate that sets the
   cost of the FP64 re-evaluation and of the plain FP64 kernel. */
zef_status zef_debug_fma_rate(zef_ctx *ctx, int32_t fp64, double *tflops);

/* Failure-detection probe: launches one block whose threads wait on a device
   barrier that is never signalled, with the given limit in nanoseconds
   (0 < limit_ns <= 2e9).  The wait expires, the kernel records the timeout
   in the context's status word and returns; the call synchronizes and must
   return ZEF_ERR_TIMEOUT.  No memory copy is in flight during the wait. */
zef_status zef_debug_wait_probe(zef_ctx *ctx, int64_t limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* ZEF_DEBUG_H */
