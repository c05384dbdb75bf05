// Prints the multimodular engine's host tables for one modulus count (argv[1]) as text lines
// "name v0 v1 ...", for tests/test_crt_tables.py to check against Python integers.  Host only:
// no CUDA call is made.
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "internal.h"

using namespace arbgpu;

template <typename T>
static void put(const char *name, const std::vector<T> &v) {
  printf("%s", name);
  for (const T &x : v) printf(" %llu", (unsigned long long)x);
  printf("\n");
}

static void put_f(const char *name, const std::vector<float> &v) {
  printf("%s", name);
  for (float x : v) {
    uint32_t u;
    memcpy(&u, &x, 4);
    printf(" %u", u);
  }
  printf("\n");
}

int main(int argc, char **argv) {
  if (argc < 2) return 2;
  const int NM = atoi(argv[1]);
  const CrtPlan *P = crt_plan(NM);
  if (!P) return 1;
  printf("dims %d %d %d %d %d %d %d\n", P->NM, P->NMW, P->NCHP, P->NW32P, P->NPAD, P->NQ, P->NQP);
  printf("bits_for %d %d %d\n", crt_moduli_for_bits(100), crt_moduli_for_bits(600),
         crt_moduli_for_bits(2000));
  put("mods", P->mods);
  put("inv", P->inv);
  put("pow32", P->pow32);
  put("Q32", P->Q32);
  put("M32", P->M32);
  put("y", P->y);
  put_f("rinv", P->rinv);
  put("ztab", P->ztab);
  put("M", P->M);
  put("wtab", P->wtab);
  put("crt_wtab", P->crt_wtab);
  put_f("mbytes", P->mbytes);
  printf("dims8 %d %d\n", P->K8, P->NQ8);
  printf("w8");
  for (int8_t x : P->w8) printf(" %d", (int)x);
  printf("\n");
  put("c32", P->c32);
  printf("dimsr %d %d\n", P->N2, P->KR);
  put("w8r", P->w8r);
  return 0;
}
