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
   (x, y, z), a weight (1 when the window is a surface triangle, 0 on the two
   entries that start a strip and on padding), that triangle's doubled-area
   normal (x, y, z) with the surface orientation, and kappa * |normal| (-inf
   when the weight is 0).  Writes min(count, cap) entries to `out` (host,
   nullable) and the entry count to *count.  Works on host-only contexts. */
zef_status zef_debug_strip_entries(const zef_ctx *ctx, int32_t index, float *out, int64_t cap,
                                   int64_t *count);

/* Entry and strip counts of compartment `index`. */
zef_status zef_debug_strip_stats(const zef_ctx *ctx, int32_t index, int64_t *entries, int64_t *strips);

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
