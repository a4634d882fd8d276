// pm_params.cpp -- host-side setup for a plan (arxiv 2209.01290, Sec. III-A
// setup and Sec. VI-A: twiddle factors are precomputed on the CPU).
//
//  * NTT-friendly primes: q prime with 2N | q - 1, below a bit bound.
//  * psi: a primitive 2N-th root of unity mod q, chosen by the fixed rule
//    "first x = 2, 3, ... whose power x^((q-1)/2N) has psi^N = -1".
//  * Per-limb tables: Psi_br[i] = psi^br(i) and (psi^-1)^br(i) (times 2^-1
//    when the plan uses per-stage halving), each with its Shoup companion
//    floor(w 2^64 / q); Algorithm 4's mu = floor(2^(2m+1) / q); N^-1 and
//    Psi^-1_br[1] * N^-1 for folding 1/N into the last inverse stage.
#include <cstdint>
#include <vector>

#include "pm_params.h"

namespace pm {
namespace host {

using u128 = unsigned __int128;

static inline uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t q) {
  return (uint64_t)((u128)a * b % q);
}

uint64_t pow_mod(uint64_t base, uint64_t exp, uint64_t q) {
  uint64_t acc = 1 % q;
  base %= q;
  for (; exp; exp >>= 1) {
    if (exp & 1) acc = mul_mod(acc, base, q);
    base = mul_mod(base, base, q);
  }
  return acc;
}

// Strong-probable-prime test to base a (n odd, n > a).
static bool sprp(uint64_t n, uint64_t a) {
  a %= n;
  if (a == 0) return true;
  uint64_t d = n - 1;
  unsigned r = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++r;
  }
  uint64_t x = pow_mod(a, d, n);
  if (x == 1 || x == n - 1) return true;
  for (unsigned i = 1; i < r; ++i) {
    x = mul_mod(x, x, n);
    if (x == n - 1) return true;
  }
  return false;
}

// Deterministic for all 64-bit n: the seven-base set {2, 325, 9375, 28178,
// 450775, 9780504, 1795265022} has no common strong pseudoprime below 2^64.
bool is_prime_u64(uint64_t n) {
  if (n < 2) return false;
  static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47};
  for (uint64_t p : small) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  static const uint64_t bases[] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
  for (uint64_t a : bases)
    if (!sprp(n, a)) return false;
  return true;
}

uint32_t bit_length(uint64_t x) {
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

int largest_ntt_primes(uint32_t log2n, uint32_t qbits, uint32_t count, uint64_t* out) {
  const uint64_t two_n = (uint64_t)2 << log2n;
  const uint64_t bound = (uint64_t)1 << qbits;  // exclusive
  // largest value = 1 (mod 2N) strictly below the bound
  uint64_t c = bound - 1 - ((bound - 2) % two_n);
  int found = 0;
  for (uint64_t steps = 0; found < (int)count && c > two_n && steps < (1ull << 26); ++steps) {
    if (is_prime_u64(c)) out[found++] = c;
    c -= two_n;
  }
  return found;
}

uint64_t default_psi(uint64_t q, uint32_t log2n) {
  const uint64_t two_n = (uint64_t)2 << log2n;
  if ((q - 1) % two_n) return 0;
  const uint64_t e = (q - 1) / two_n;
  for (uint64_t x = 2; x < q && x < 4096; ++x) {
    const uint64_t psi = pow_mod(x, e, q);
    if (pow_mod(psi, (uint64_t)1 << log2n, q) == q - 1) return psi;
  }
  return 0;
}

static inline uint64_t shoup_companion(uint64_t w, uint64_t q) {
  return (uint64_t)(((u128)w << 64) / q);
}

static inline uint32_t reverse_bits(uint32_t x, uint32_t nbits) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < nbits; ++i) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

void build_limb(uint32_t log2n, uint64_t q, uint64_t psi, bool halving, LimbConst* lc,
                TwPair* twf, TwPair* twi) {
  const uint32_t n = 1u << log2n;
  const uint32_t m = bit_length(q);
  lc->q = q;
  lc->two_q = 2 * q;
  lc->half_q1 = (q + 1) / 2;
  lc->mu = (uint64_t)((((u128)1) << (2 * m + 1)) / q);
  lc->m = m;
  lc->sh1 = m - 2;
  lc->sh2 = m + 3;
  lc->halving = halving ? 1 : 0;
  // powers psi^e and psi^-e for e < N
  const uint64_t psi_inv = pow_mod(psi, 2 * (uint64_t)n - 1, q);  // psi^(2N) = 1
  const uint64_t inv2 = (q + 1) / 2;
  std::vector<uint64_t> fw(n), iv(n);
  fw[0] = 1;
  iv[0] = 1;
  for (uint32_t e = 1; e < n; ++e) {
    fw[e] = mul_mod(fw[e - 1], psi, q);
    iv[e] = mul_mod(iv[e - 1], psi_inv, q);
  }
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t r = reverse_bits(i, log2n);
    const uint64_t wf = fw[r];
    const uint64_t wi = halving ? mul_mod(iv[r], inv2, q) : iv[r];
    twf[i].w = wf;
    twf[i].wp = shoup_companion(wf, q);
    twi[i].w = wi;
    twi[i].wp = shoup_companion(wi, q);
  }
  // N^-1 = (2^-1)^log2n; Psi^-1_br[1] = psi^-(N/2) (br(1) = N/2)
  const uint64_t ninv = pow_mod(inv2, log2n, q);
  const uint64_t w1 = n > 1 ? iv[reverse_bits(1, log2n)] : 1;
  lc->ninv = ninv;
  lc->ninv_p = shoup_companion(ninv, q);
  lc->w1ninv = mul_mod(w1, ninv, q);
  lc->w1ninv_p = shoup_companion(lc->w1ninv, q);
}

void fused_limb(const LimbConst& in, LimbConst* out) {
  *out = in;
  const uint64_t q = in.q;
  out->ninv = mul_mod(in.ninv, 2, q);
  out->ninv_p = shoup_companion(out->ninv, q);
  out->w1ninv = mul_mod(in.w1ninv, 2, q);
  out->w1ninv_p = shoup_companion(out->w1ninv, q);
}

// 32-bit words: the same tables with Shoup companions floor(w * 2^32 / q) and
// Algorithm 4's mu = floor(2^(2m+1) / q) for beta = 32 (q < 2^30).
void build_limb32(uint32_t log2n, uint64_t q, uint64_t psi, bool halving, LimbConst32* lc,
                  TwPair32* twf, TwPair32* twi) {
  const uint32_t n = 1u << log2n;
  const uint32_t m = bit_length(q);
  auto companion = [&](uint64_t w) { return (uint32_t)((w << 32) / q); };
  lc->q = (uint32_t)q;
  lc->two_q = (uint32_t)(2 * q);
  lc->half_q1 = (uint32_t)((q + 1) / 2);
  lc->mu = (uint32_t)((((u128)1) << (2 * m + 1)) / q);
  lc->m = m;
  lc->sh1 = m - 2;
  lc->sh2 = m + 3;
  lc->halving = halving ? 1 : 0;
  const uint64_t psi_inv = pow_mod(psi, 2 * (uint64_t)n - 1, q);
  const uint64_t inv2 = (q + 1) / 2;
  std::vector<uint64_t> fw(n), iv(n);
  fw[0] = 1;
  iv[0] = 1;
  for (uint32_t e = 1; e < n; ++e) {
    fw[e] = mul_mod(fw[e - 1], psi, q);
    iv[e] = mul_mod(iv[e - 1], psi_inv, q);
  }
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t r = reverse_bits(i, log2n);
    const uint64_t wf = fw[r];
    const uint64_t wi = halving ? mul_mod(iv[r], inv2, q) : iv[r];
    twf[i] = TwPair32{(uint32_t)wf, companion(wf)};
    twi[i] = TwPair32{(uint32_t)wi, companion(wi)};
  }
  const uint64_t ninv = pow_mod(inv2, log2n, q);
  const uint64_t w1 = n > 1 ? iv[reverse_bits(1, log2n)] : 1;
  const uint64_t w1ninv = mul_mod(w1, ninv, q);
  lc->ninv = (uint32_t)ninv;
  lc->ninv_p = companion(ninv);
  lc->w1ninv = (uint32_t)w1ninv;
  lc->w1ninv_p = companion(w1ninv);
}

void fused_limb32(const LimbConst32& in, LimbConst32* out) {
  *out = in;
  const uint64_t q = in.q;
  const uint64_t ninv = mul_mod(in.ninv, 2, q), w1ninv = mul_mod(in.w1ninv, 2, q);
  out->ninv = (uint32_t)ninv;
  out->ninv_p = (uint32_t)((ninv << 32) / q);
  out->w1ninv = (uint32_t)w1ninv;
  out->w1ninv_p = (uint32_t)((w1ninv << 32) / q);
}

}  // namespace host
}  // namespace pm
