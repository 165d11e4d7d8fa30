// Refinement kernels (placeholder until the refine path lands).
#include "zef_internal.h"

namespace zef {
zef_status refine_run(zef_ctx *ctx, zef_mesh *mesh, int32_t levels, const zef_label_opts &opts,
                      zef_level_stats *per_level) {
  (void)mesh; (void)levels; (void)opts; (void)per_level;
  return fail(ctx, ZEF_ERR_INVALID_ARG, "refinement not built yet");
}
}  // namespace zef
