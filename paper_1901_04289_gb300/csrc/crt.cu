// Host side of the multimodular integer engine: the moduli (primes just below 2^16), their Barrett
// reciprocals, the tables 2^(32c) mod m_t, and the Chinese-remainder data of M = prod m_t: the
// cofactors Q_t = M / m_t, y_t = Q_t^-1 mod m_t and 1 / m_t, all computed once per modulus count and
// cached.  An integer T with |T| < M / 8 follows from its residues r_t as
//   T = sum_t z_t Q_t - q M,   z_t = r_t y_t mod m_t,   q = round(sum_t z_t / m_t),
// since sum_t z_t Q_t = T (mod M) and sum_t z_t / m_t = q + T / M with |T / M| < 1/8, so a float
// sum fixes q.  (The paper's integer products use FLINT's multimodular algorithm, Section IV.)
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>

#include "internal.h"

namespace arbgpu {

namespace {

// Primes below 2^16 in decreasing order (sieve of Eratosthenes).
const std::vector<uint32_t> &primes_desc() {
  static std::vector<uint32_t> p;
  static std::once_flag once;
  std::call_once(once, []() {
    const uint32_t n = 1u << 16;
    std::vector<char> comp(n, 0);
    for (uint32_t i = 2; i * i < n; ++i)
      if (!comp[i])
        for (uint32_t j = i * i; j < n; j += i) comp[j] = 1;
    for (uint32_t i = n - 1; i >= 3; --i)
      if (!comp[i]) p.push_back(i);
  });
  return p;
}

// little-endian multi-limb helpers
void mul_small(std::vector<uint64_t> &a, uint32_t m) {
  u128 c = 0;
  for (auto &w : a) {
    c += (u128)w * m;
    w = (uint64_t)c;
    c >>= 64;
  }
  if (c) a.push_back((uint64_t)c);
}

int bit_length(const std::vector<uint64_t> &a) {
  for (int k = (int)a.size() - 1; k >= 0; --k)
    if (a[k]) return 64 * k + 64 - __builtin_clzll(a[k]);
  return 0;
}

uint32_t inv_mod(uint32_t a, uint32_t m) {  // a^-1 mod m (gcd(a, m) = 1)
  int64_t t = 0, nt = 1, r = m, nr = a % m;
  while (nr) {
    const int64_t q = r / nr;
    int64_t tmp = t - q * nt;
    t = nt;
    nt = tmp;
    tmp = r - q * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += m;
  return (uint32_t)t;
}

std::mutex g_mu;
std::map<int, std::unique_ptr<CrtPlan>> g_plans;

std::unique_ptr<CrtPlan> build_plan(int NM) {
  const auto &pr = primes_desc();
  auto P = std::make_unique<CrtPlan>();
  P->NM = NM;
  P->mods.assign(pr.begin(), pr.begin() + NM);
  std::vector<uint64_t> M{1};
  for (uint32_t m : P->mods) mul_small(M, m);
  P->NMW = (bit_length(M) + 63) / 64;
  if (P->NMW < 2) P->NMW = 2;
  M.resize(P->NMW, 0);
  P->M = M;
  P->inv.resize(NM);
  P->y.resize(NM);
  P->rinv.resize(NM);
  P->NW32P = (2 * P->NMW + 15) / 16 * 16;
  P->Q32.assign((size_t)NM * P->NW32P, 0);
  P->M32.assign((size_t)P->NW32P, 0);
  for (int k = 0; k < P->NMW; ++k) {
    P->M32[2 * k] = (uint32_t)P->M[k];
    P->M32[2 * k + 1] = (uint32_t)(P->M[k] >> 32);
  }
  for (int t = 0; t < NM; ++t) {
    const uint32_t m = P->mods[t];
    P->inv[t] = ~(uint64_t)0 / m;
    P->rinv[t] = (float)(1.0 / (double)m);
    std::vector<uint64_t> Q{1};
    uint64_t qmod = 1;
    for (int s = 0; s < NM; ++s)
      if (s != t) {
        mul_small(Q, P->mods[s]);
        qmod = qmod * (P->mods[s] % m) % m;
      }
    P->y[t] = inv_mod((uint32_t)qmod, m);
    for (int k = 0; k < P->NMW && k < (int)Q.size(); ++k) {
      P->Q32[(size_t)t * P->NW32P + 2 * k] = (uint32_t)Q[k];
      P->Q32[(size_t)t * P->NW32P + 2 * k + 1] = (uint32_t)(Q[k] >> 32);
    }
  }
  // GEMM item tables for up to three residue products in one batch (the complex product by
  // eq. 2 runs its three real products as items t, NM + t and 2 NM + t of modulus t)
  P->ztab.assign((size_t)4 * 3 * NM, 0);
  for (int t = 0; t < 3 * NM; ++t) {
    const uint32_t m = P->mods[t % NM];
    const float mf = (float)m, rinv = (float)(1.0 / (double)m);
    P->ztab[4 * t] = m;
    memcpy(&P->ztab[4 * t + 1], &mf, 4);    // m as a float (exact: m < 2^16)
    memcpy(&P->ztab[4 * t + 2], &rinv, 4);  // 1 / m rounded to nearest
  }
  for (int t = NM; t < 3 * NM; ++t) P->inv.push_back(P->inv[t - NM]);
  P->NCHP = CRT_MAX_CHUNKS32;
  P->pow32.resize((size_t)NM * P->NCHP);
  for (int t = 0; t < NM; ++t) {
    uint64_t v = 1;
    for (int c = 0; c < P->NCHP; ++c) {
      P->pow32[(size_t)t * P->NCHP + c] = (uint32_t)v;
      v = (v << 32) % P->mods[t];
    }
  }
  // digit weights of the tensor-core residue step (one table per operand side)
  P->NPAD = (2 * NM + 15) / 16 * 16;
  P->wtab.assign((size_t)2 * P->NPAD * 128, 0);
  auto bf16_bits = [](int v) {  // |v| <= 256: exact in BF16, the top half of the float
    const float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
  };
  for (int side = 0; side < 2; ++side)
    for (int t = 0; t < NM; ++t) {
      const uint64_t m = P->mods[t];
      uint64_t v = 1;  // 2^(8d) mod m
      for (int d = 0; d < 128; ++d) {
        int64_t w = (int64_t)(side ? v * P->y[t] % m : v);
        if (w > (int64_t)(m >> 1)) w -= (int64_t)m;
        const int64_t l = ((w + 128) & 255) - 128, hb = (w - l) >> 8;
        uint16_t *row = P->wtab.data() + ((size_t)side * P->NPAD + 2 * t) * 128;
        row[d] = bf16_bits((int)l);
        row[128 + d] = bf16_bits((int)hb);
        v = (v << 8) % m;
      }
    }
  // the same weights as unsigned bytes for the warp-level MMA residue step (every NM): side o,
  // column n = 2t + b holds byte b of 2^(8d) mod m_t (times y_t for side 1) in row d < KR
  P->N2 = (2 * NM + 31) / 32 * 32;
  P->KR = (4 * CRT_MAX_CHUNKS32 + 31) / 32 * 32;
  P->w8r.assign((size_t)2 * P->N2 * P->KR, 0);
  for (int side = 0; side < 2; ++side)
    for (int t = 0; t < NM; ++t) {
      const uint64_t m = P->mods[t];
      uint64_t v = 1;  // 2^(8d) mod m
      for (int d = 0; d < P->KR; ++d) {
        const uint64_t w = side ? v * P->y[t] % m : v;
        uint8_t *col = P->w8r.data() + ((size_t)side * P->N2 + 2 * t) * P->KR;
        col[d] = (uint8_t)(w & 255);
        col[P->KR + d] = (uint8_t)(w >> 8);
        v = (v << 8) % m;
      }
    }
  // reconstruction weights (used when NM <= 64)
  {
    auto balanced_bytes = [](const std::vector<uint64_t> &x, int nb) {
      std::vector<int> d(nb, 0);
      int carry = 0;
      for (int n = 0; n < nb; ++n) {
        const int k = n / 8;
        int v = (k < (int)x.size() ? (int)((x[k] >> (8 * (n % 8))) & 255) : 0) + carry;
        carry = 0;
        if (v >= 128) {
          v -= 256;
          carry = 1;
        }
        d[n] = v;
      }
      return d;
    };
    const int NB = (bit_length(P->M) + 7) / 8 + 1;  // balanced bytes of M (and of each Q_t)
    P->NQ = NB + 1;                                 // the high byte of z shifts Q_t by one
    P->NQP = (P->NQ + 1 + 15) / 16 * 16;
    P->crt_wtab.assign((size_t)P->NQP * 128, 0);
    P->mbytes.assign(P->NQ, 0.f);
    auto bf16_of = [](float f) {  // round to nearest even (exact for the small integers)
      uint32_t u;
      memcpy(&u, &f, 4);
      u += 0x7FFFu + ((u >> 16) & 1u);
      return (uint16_t)(u >> 16);
    };
    // the same bytes as 8-bit integers for the warp-level MMA reconstruction (every NM): row n
    // of w8 [NQ8][K8] holds byte n of Q_t in column 2t and byte n - 1 in column 2t + 1
    P->K8 = (2 * NM + 31) / 32 * 32;
    P->NQ8 = (P->NQ + 31) / 32 * 32;
    P->w8.assign((size_t)P->NQ8 * P->K8, 0);
    // the z bytes enter the MMA offset by -128 (signed): c32 = 32896 sum_t Q_t puts them back
    std::vector<uint64_t> qsum(P->NMW + 1, 0);
    for (int t = 0; t < NM; ++t) {
      std::vector<uint64_t> Q(P->NMW, 0);
      for (int k = 0; k < P->NMW; ++k)
        Q[k] = (uint64_t)P->Q32[(size_t)t * P->NW32P + 2 * k] |
               ((uint64_t)P->Q32[(size_t)t * P->NW32P + 2 * k + 1] << 32);
      u128 cq = 0;
      for (int k = 0; k <= P->NMW; ++k) {
        cq += (u128)qsum[k] + (k < P->NMW ? Q[k] : 0);
        qsum[k] = (uint64_t)cq;
        cq >>= 64;
      }
      const std::vector<int> qb = balanced_bytes(Q, NB);
      for (int n = 0; n < P->NQ; ++n) {
        const int lo = n < NB ? qb[n] : 0, hi = (n >= 1 && n - 1 < NB) ? qb[n - 1] : 0;
        P->w8[(size_t)n * P->K8 + 2 * t] = (int8_t)lo;
        P->w8[(size_t)n * P->K8 + 2 * t + 1] = (int8_t)hi;
        if (NM <= 64) {
          P->crt_wtab[(size_t)n * 128 + 2 * t] = bf16_of((float)lo);
          P->crt_wtab[(size_t)n * 128 + 2 * t + 1] = bf16_of((float)hi);
        }
      }
      if (NM <= 64) {
        P->crt_wtab[(size_t)P->NQ * 128 + 2 * t] = bf16_of((float)(1.0 / (double)P->mods[t]));
        P->crt_wtab[(size_t)P->NQ * 128 + 2 * t + 1] =
            bf16_of((float)(256.0 / (double)P->mods[t]));
      }
    }
    mul_small(qsum, 32896u);
    P->c32.assign((size_t)2 * P->NMW + 2, 0);
    for (int k = 0; k < (int)qsum.size() && 2 * k + 1 < (int)P->c32.size(); ++k) {
      P->c32[2 * k] = (uint32_t)qsum[k];
      P->c32[2 * k + 1] = (uint32_t)(qsum[k] >> 32);
    }
    if (NM <= 64) {
      const std::vector<int> mb = balanced_bytes(P->M, NB);
      for (int n = 0; n < NB; ++n) P->mbytes[n] = (float)mb[n];
    }
  }
  return P;
}

}  // namespace

// Number of moduli whose product M exceeds 2^(bits + 3): signed integers T of `bits` bits, sign
// included, then satisfy |T| < M / 8, as the reconstruction requires.
int crt_moduli_for_bits(int bits) {
  const auto &pr = primes_desc();
  double acc = 0;
  int n = 0;
  while (n < (int)pr.size() && acc < bits + 3.0) acc += std::log2((double)pr[n++]);
  return n < 5 ? 5 : n;
}

arbgpu_status crt_device_tables(arbgpu_ctx *ctx, const CrtPlan *P, CrtDevTables *out) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t oQ = 0, oM = oQ + al(4 * P->Q32.size()), oy = oM + al(4 * P->M32.size());
  const size_t oz = oy + al(4 * P->y.size()), op = oz + al(4 * P->ztab.size());
  const size_t orv = op + al(4 * P->pow32.size()), oi = orv + al(4 * P->rinv.size());
  const size_t ow = oi + al(8 * P->inv.size());
  const size_t ocw = ow + al(2 * P->wtab.size());
  const size_t omb = ocw + al(2 * P->crt_wtab.size());
  const size_t ow8 = omb + al(4 * P->mbytes.size());
  const size_t oc32 = ow8 + al(P->w8.size());
  const size_t ow8r = oc32 + al(4 * P->c32.size());
  const size_t total = ow8r + al(P->w8r.size());
  auto it = ctx->crt_tables.find(P->NM);
  uint8_t *base = nullptr;
  if (it != ctx->crt_tables.end()) {
    base = (uint8_t *)it->second;
  } else {
    if (cudaMalloc(&base, total) != cudaSuccess) return ARBGPU_ERR_CUDA;
    std::vector<uint8_t> h(total, 0);
    memcpy(h.data() + oQ, P->Q32.data(), 4 * P->Q32.size());
    memcpy(h.data() + oM, P->M32.data(), 4 * P->M32.size());
    memcpy(h.data() + oy, P->y.data(), 4 * P->y.size());
    memcpy(h.data() + oz, P->ztab.data(), 4 * P->ztab.size());
    memcpy(h.data() + op, P->pow32.data(), 4 * P->pow32.size());
    memcpy(h.data() + orv, P->rinv.data(), 4 * P->rinv.size());
    memcpy(h.data() + oi, P->inv.data(), 8 * P->inv.size());
    memcpy(h.data() + ow, P->wtab.data(), 2 * P->wtab.size());
    memcpy(h.data() + ocw, P->crt_wtab.data(), 2 * P->crt_wtab.size());
    memcpy(h.data() + omb, P->mbytes.data(), 4 * P->mbytes.size());
    memcpy(h.data() + ow8, P->w8.data(), P->w8.size());
    memcpy(h.data() + oc32, P->c32.data(), 4 * P->c32.size());
    memcpy(h.data() + ow8r, P->w8r.data(), P->w8r.size());
    if (cudaMemcpy(base, h.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(base);
      return ARBGPU_ERR_CUDA;
    }
    ctx->crt_tables[P->NM] = base;
  }
  out->Q32 = (const uint32_t *)(base + oQ);
  out->M32 = (const uint32_t *)(base + oM);
  out->y = (const uint32_t *)(base + oy);
  out->ztab = (const uint32_t *)(base + oz);
  out->pow32 = (const uint32_t *)(base + op);
  out->rinv = (const float *)(base + orv);
  out->inv = (const uint64_t *)(base + oi);
  out->wtab = (const uint16_t *)(base + ow);
  out->crt_wtab = (const uint16_t *)(base + ocw);
  out->mbytes = (const float *)(base + omb);
  out->w8 = (const int8_t *)(base + ow8);
  out->c32 = (const uint32_t *)(base + oc32);
  out->w8r = (const uint8_t *)(base + ow8r);
  return ARBGPU_OK;
}

const CrtPlan *crt_plan(int NM) {
  if (NM < 1 || NM > CRT_MAX_MODULI) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_plans.find(NM);
  if (it != g_plans.end()) return it->second.get();
  auto P = build_plan(NM);
  const CrtPlan *r = P.get();
  g_plans[NM] = std::move(P);
  return r;
}

}  // namespace arbgpu
