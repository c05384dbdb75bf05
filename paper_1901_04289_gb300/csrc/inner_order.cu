// Host side of the inner ordering (Section IV-B's suggested inner scaling combined with a
// permutation of the inner index; the kernels and the driver are in block.cu).
#include <algorithm>
#include <utility>

#include "internal.h"

namespace arbgpu {

void inner_order_host(const std::vector<int64_t> &a, const std::vector<int64_t> &b,
                      std::vector<int32_t> &ord, std::vector<int64_t> &g) {
  const int64_t K = (int64_t)a.size();
  std::vector<std::pair<int64_t, int32_t>> live;
  std::vector<int32_t> dead;
  g.assign((size_t)K, 0);
  for (int64_t k = 0; k < K; ++k) {
    if (a[k] == INT64_MIN || b[k] == INT64_MIN) {  // no nonzero midpoint product at k
      dead.push_back((int32_t)k);
      continue;
    }
    const int64_t d = b[k] - a[k];
    g[k] = d >= 0 ? d / 2 : -((-d + 1) / 2);  // floor(d / 2)
    live.push_back({a[k] + b[k], (int32_t)k});
  }
  std::sort(live.begin(), live.end());  // by a_k + b_k, ties by index
  ord.clear();
  for (const auto &v : live) ord.push_back(v.second);
  ord.insert(ord.end(), dead.begin(), dead.end());
}

}  // namespace arbgpu
