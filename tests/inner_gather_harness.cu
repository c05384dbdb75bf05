// Runs gather_inner_entry (the per-entry body of the GPU's reordered, scaled operand copies) on
// the host.  Standard input: "rows K cols nl is_b ld", then the operand's limb planes (nl x count),
// exp, flags, rad_man, rad_exp (count each, count = rows * ld for A or K * ld for B), then ord (K)
// and g (K).  Standard output: the copy's arrays in the same order, then "range <0|1>".
#include <cstdio>
#include <vector>

#include "inner_order.cuh"

using namespace arbgpu;

template <typename T>
static bool read_vec(std::vector<T> &v, size_t n) {  // unsigned types in full 64-bit range
  v.resize(n);
  for (auto &x : v) {
    if ((T)-1 > (T)0) {
      unsigned long long t;
      if (scanf("%llu", &t) != 1) return false;
      x = (T)t;
    } else {
      long long t;
      if (scanf("%lld", &t) != 1) return false;
      x = (T)t;
    }
  }
  return true;
}

template <typename T>
static void put(const char *name, const std::vector<T> &v) {
  printf("%s", name);
  for (const T &x : v) {
    if ((T)-1 > (T)0)
      printf(" %llu", (unsigned long long)x);
    else
      printf(" %lld", (long long)x);
  }
  printf("\n");
}

int main() {
  long long rows, K, cols, nl, is_b, ld;
  if (scanf("%lld %lld %lld %lld %lld %lld", &rows, &K, &cols, &nl, &is_b, &ld) != 6) return 2;
  const size_t count = (size_t)((is_b ? K : rows) * ld);
  const size_t n = (size_t)(is_b ? K * cols : rows * K);
  std::vector<uint64_t> limbs;
  std::vector<int64_t> exp, rexp, g;
  std::vector<uint32_t> flags, rman;
  std::vector<int32_t> ord;
  if (!read_vec(limbs, nl * count) || !read_vec(exp, count) || !read_vec(flags, count) ||
      !read_vec(rman, count) || !read_vec(rexp, count) || !read_vec(ord, K) || !read_vec(g, K))
    return 2;
  const BallsView X{limbs.data(), (int64_t)count, (int32_t)nl, exp.data(), flags.data(),
                    rman.data(), rexp.data()};
  std::vector<uint64_t> ylimbs(nl * n);
  std::vector<int64_t> yexp(n), yrexp(n);
  std::vector<uint32_t> yflags(n), yrman(n);
  const BallsOut Y{ylimbs.data(), (int64_t)n, (int32_t)nl, yexp.data(), yflags.data(),
                   yrman.data(), yrexp.data()};
  bool range = false;
  for (size_t idx = 0; idx < n; ++idx)
    range |= gather_inner_entry(X, ld, is_b != 0, K, cols, ord.data(), g.data(), Y, (int64_t)idx);
  put("limbs", ylimbs);
  put("exp", yexp);
  put("flags", yflags);
  put("rad_man", yrman);
  put("rad_exp", yrexp);
  printf("range %d\n", range ? 1 : 0);
  return 0;
}
