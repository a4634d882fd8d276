// pm_arith.cuh -- device modular arithmetic for 64-bit words and moduli
// q < 2^62 (arxiv 2209.01290, Sec. II).
//
// Value ranges ("lazy" representatives, Harvey-style) used by the butterflies:
//   forward CT butterfly : inputs and outputs in [0, 4q)
//   inverse GS butterfly : inputs and outputs in [0, 2q)
// q < 2^62 keeps 4q < 2^64, so no word ever overflows.  Results that leave
// the library are reduced to the canonical range [0, q).
#pragma once
#include <cstdint>

#include "pm_types.h"

namespace pm {

__device__ __forceinline__ TwPair ld_tw(const TwPair* __restrict__ p) {
  ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
  return TwPair{v.x, v.y};
}

// Two consecutive twiddle pairs p[0], p[1] in one 256-bit read-only load.
// p must be 32-byte aligned: every caller passes an even index into a table
// whose base is 32-byte aligned (cudaMalloc'ed, per-limb offsets N * 16 B).
__device__ __forceinline__ void ld_tw2(const TwPair* __restrict__ p, TwPair& t0, TwPair& t1) {
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(t0.w), "=l"(t0.wp), "=l"(t1.w), "=l"(t1.wp)
      : "l"(p));
}

// w * y mod q up to one multiple of q (Shoup): for w < q and any 64-bit y,
// the result is congruent to w*y and lies in [0, 2q).  Written as
// w*y + qh*(2^64 - q) mod 2^64 so that the subtraction folds into the
// multiply-add chain of the low-word products.
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t y, uint64_t w, uint64_t wp,
                                                   uint64_t q) {
  const uint64_t qh = __umul64hi(wp, y);
  return w * y + qh * (0 - q);
}

// x - m if x >= m else x, for x < 2^63 + m and m <= 2^63 (all lazy values here
// are < 2^62): the sign of x - m decides, one compare on the high word.
__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t m) {
  const uint64_t t = x - m;
  return (int64_t)t < 0 ? x : t;
}

// Merged-CT butterfly (Algorithm 6 body):
//   (x, y) <- (x + w y, x - w y) mod q
// on lazy representatives in [0, 4q).
__device__ __forceinline__ void ct_bfly(uint64_t& x, uint64_t& y, uint64_t w, uint64_t wp,
                                        uint64_t q, uint64_t two_q) {
  const uint64_t a = csub(x, two_q);               // [0, 2q)
  const uint64_t t = mul_shoup_lazy(y, w, wp, q);  // [0, 2q)
  x = a + t;                                       // [0, 4q)
  y = a - t + two_q;                               // (0, 4q)
}

// x/2 mod q for x in [0, 2q): x >> 1 plus (q+1)/2 when x is odd (Sec. III-A).
// Result in [0, 2q).
__device__ __forceinline__ uint64_t half_lazy(uint64_t x, uint64_t half_q1) {
  return (x >> 1) + ((x & 1) ? half_q1 : 0);
}

// Merged-GS butterfly (Algorithm 7 body) with the 1/2 scaling of Eq. 2:
//   (x, y) <- ((x + y)/2, w (x - y)/2) mod q
// w2 = w * 2^-1 mod q is the table entry, so the second output needs no
// separate halving.  Lazy representatives in [0, 2q).
__device__ __forceinline__ void gs_bfly_half(uint64_t& x, uint64_t& y, uint64_t w2,
                                             uint64_t w2p, uint64_t q, uint64_t two_q,
                                             uint64_t half_q1) {
  const uint64_t s = csub(x + y, two_q);           // [0, 2q)
  const uint64_t d = x - y + two_q;                // (0, 4q)
  x = half_lazy(s, half_q1);                       // [0, 2q)
  y = mul_shoup_lazy(d, w2, w2p, q);               // [0, 2q)
}

// Merged-GS butterfly (Algorithm 7 body) without scaling:
//   (x, y) <- (x + y, w (x - y)) mod q
// on lazy representatives in [0, 2q); 1/N is applied by gs_bfly_last.
__device__ __forceinline__ void gs_bfly(uint64_t& x, uint64_t& y, uint64_t w, uint64_t wp,
                                        uint64_t q, uint64_t two_q) {
  const uint64_t s = csub(x + y, two_q);           // [0, 2q)
  const uint64_t d = x - y + two_q;                // (0, 4q)
  x = s;
  y = mul_shoup_lazy(d, w, wp, q);                 // [0, 2q)
}

// The last GS stage (k = N/2, twiddle Psi^-1_br[1]) with 1/N folded in:
//   (x, y) <- ((x + y) / N, w (x - y) / N) mod q, results in [0, 2q).
__device__ __forceinline__ void gs_bfly_last(uint64_t& x, uint64_t& y, const LimbConst& k) {
  const uint64_t s = x + y;                        // [0, 4q)
  const uint64_t d = x - y + k.two_q;              // (0, 4q)
  x = mul_shoup_lazy(s, k.ninv, k.ninv_p, k.q);
  y = mul_shoup_lazy(d, k.w1ninv, k.w1ninv_p, k.q);
}

// One GS butterfly in the plan's scaling mode.
template <bool HALVE>
__device__ __forceinline__ void gs_bfly_mode(uint64_t& x, uint64_t& y, uint64_t w, uint64_t wp,
                                             uint64_t q, uint64_t two_q, uint64_t hq) {
  if constexpr (HALVE)
    gs_bfly_half(x, y, w, wp, q, two_q, hq);
  else
    gs_bfly(x, y, w, wp, q, two_q);
}

// [0, 4q) -> [0, q)
__device__ __forceinline__ uint64_t reduce4(uint64_t x, uint64_t q, uint64_t two_q) {
  return csub(csub(x, two_q), q);
}

// Algorithm 4 (the paper's Barrett variant): x = a*b < 2^(2m) for a, b < q,
//   c = x >> (m-2); quot = (c * mu) >> (m+3); rem = x - quot*q; one correction.
// The 128-bit quantities are kept as (hi, lo) pairs; only the low word of
// quot*q is needed because rem < 2q < 2^64.
__device__ __forceinline__ uint64_t mul_barrett_alg4(uint64_t a, uint64_t b,
                                                     const LimbConst& k) {
  const uint64_t lo = a * b;
  const uint64_t hi = __umul64hi(a, b);
  // c = x >> (m-2); 1 <= m-2 <= 60
  const uint64_t c = (lo >> k.sh1) | (hi << (64 - k.sh1));
  const uint64_t plo = c * k.mu;
  const uint64_t phi = __umul64hi(c, k.mu);
  // quot = (phi:plo) >> (m+3); m+3 ranges over [6, 65]
  uint64_t quot;
  if (k.sh2 >= 64) {
    quot = phi >> (k.sh2 - 64);
  } else {
    quot = (plo >> k.sh2) | (phi << (64 - k.sh2));
  }
  const uint64_t rem = lo - quot * k.q;
  return csub(rem, k.q);
}

}  // namespace pm
