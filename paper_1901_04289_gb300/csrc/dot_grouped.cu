// Kernel (a) over the classical items of a grouped batch of products.
#include "dot_src.cuh"

namespace arbgpu {

arbgpu_status launch_grouped_dot(arbgpu_ctx *ctx, const GroupItem *dev_items,
                                 const int64_t *dev_ends, int32_t count, int64_t total_dots,
                                 int prec_max, int64_t k_max, int max_nlimbs,
                                 cudaStream_t stream) {
  GroupedDotSrc s{dev_items, dev_ends, count, total_dots, prec_max, 2 * k_max};
  const int cmax = dot_class_for_problem(prec_max, 2 * k_max + 1, max_nlimbs);
  if (cmax < 0) return ARBGPU_ERR_INVALID;
  return launch_dot_src(ctx, s, total_dots, cmax, dot_group_matrix(), stream);
}

}  // namespace arbgpu
