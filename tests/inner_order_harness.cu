// Reads K, then a_0..a_{K-1}, then b_0..b_{K-1} (decimal int64) from standard input and prints
// the inner order ("ord ...") and scaling ("g ...") of inner_order_host, for
// tests/test_inner_order_host.py.  Host only: no CUDA call is made.
#include <cinttypes>
#include <cstdio>

#include "internal.h"

int main() {
  long long K = 0;
  if (scanf("%lld", &K) != 1 || K < 0) return 2;
  std::vector<int64_t> a((size_t)K), b((size_t)K);
  for (auto *v : {&a, &b})
    for (auto &x : *v) {
      long long t;
      if (scanf("%lld", &t) != 1) return 2;
      x = (int64_t)t;
    }
  std::vector<int32_t> ord;
  std::vector<int64_t> g;
  arbgpu::inner_order_host(a, b, ord, g);
  printf("ord");
  for (int32_t k : ord) printf(" %d", k);
  printf("\ng");
  for (int64_t v : g) printf(" %lld", (long long)v);
  printf("\n");
  return 0;
}
