// pm_arith.cuh -- device modular arithmetic (arxiv 2209.01290, Sec. II) for
// two word sizes:
//   64-bit words, moduli q < 2^62 (Algorithm 4 with beta = 64);
//   32-bit words, moduli q < 2^30 (Algorithm 4 with beta = 32).
//
// Value ranges ("lazy" representatives, Harvey-style) used by the butterflies:
//   forward CT butterfly : inputs and outputs in [0, 4q)
//   inverse GS butterfly : inputs and outputs in [0, 2q)
// q < 2^(beta-2) keeps 4q < 2^beta, so no word ever overflows.  Results that
// leave the library are reduced to the canonical range [0, q).
//
// The functions are templates over the word type W (uint64_t or uint32_t);
// WordT<W> names the matching twiddle-pair and limb-constant types.
#pragma once
#include <cstdint>

#include "pm_types.h"

namespace pm {

template <typename W>
struct WordT;
template <>
struct WordT<uint64_t> {
  using Tw = TwPair;
  using LC = LimbConst;
  using SW = int64_t;
};
template <>
struct WordT<uint32_t> {
  using Tw = TwPair32;
  using LC = LimbConst32;
  using SW = int32_t;
};

__device__ __forceinline__ TwPair ld_tw(const TwPair* __restrict__ p) {
  ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
  return TwPair{v.x, v.y};
}

__device__ __forceinline__ TwPair32 ld_tw(const TwPair32* __restrict__ p) {
  uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  return TwPair32{v.x, v.y};
}

// Two consecutive twiddle pairs p[0], p[1] in one read-only load (256 bits
// for 64-bit words, 128 bits for 32-bit words).  p must be aligned to twice
// the pair size: every caller passes an even index into a table whose base
// is so aligned (cudaMalloc'ed, per-limb offsets N pairs).
__device__ __forceinline__ void ld_tw2(const TwPair* __restrict__ p, TwPair& t0, TwPair& t1) {
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(t0.w), "=l"(t0.wp), "=l"(t1.w), "=l"(t1.wp)
      : "l"(p));
}

__device__ __forceinline__ void ld_tw2(const TwPair32* __restrict__ p, TwPair32& t0,
                                       TwPair32& t1) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
  t0 = TwPair32{v.x, v.y};
  t1 = TwPair32{v.z, v.w};
}

__device__ __forceinline__ uint64_t mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }
__device__ __forceinline__ uint32_t mulhi(uint32_t a, uint32_t b) { return __umulhi(a, b); }

// w * y mod q up to one multiple of q (Shoup): for w < q and any word y, the
// result is congruent to w*y and lies in [0, 2q).  Written as
// w*y + qh*(2^beta - q) mod 2^beta so that the subtraction folds into the
// multiply-add chain of the low-word products.
template <typename W>
__device__ __forceinline__ W mul_shoup_lazy(W y, W w, W wp, W q) {
  const W qh = mulhi(wp, y);
  return w * y + qh * (W(0) - q);
}

// The same product for 64-bit words, spelled out as 32-bit multiply-adds
// with explicit carries.  Halves: y = y1:y0, wp = p1:p0, w = w1:w0,
// 2^64 - q = n1:n0.  The quotient qh = floor(wp y / 2^64) is exact: the
// column of weight 2^32 (hi(p0 y0) + lo(p1 y0) + lo(p0 y1)) is summed only
// for its carries into the column of weight 2^64 (hi(p1 y0) + hi(p0 y1) +
// lo(p1 y1)), whose carry goes to the top column (hi(p1 y1)).  The result
// w y + qh (2^64 - q) mod 2^64 needs only the low words of the two
// products.  Same value as the generic form (bit-exact); written this way
// the compiler issues 10 multiplies and no 64-bit addend set-up moves, about
// 17% fewer instructions per butterfly on sm_103a (ncu opcode counts).
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t y, uint64_t w, uint64_t wp,
                                                   uint64_t q) {
  const uint64_t nq = 0 - q;
  uint32_t r0, r1;
  asm("{\n\t"
      ".reg .u32 m1, m2, m3, q0, q1;\n\t"
      "mul.hi.u32      m1, %4, %2;\n\t"      // m1 = hi(p0 y0)
      "mad.lo.cc.u32   m1, %5, %2, m1;\n\t"  // m1 += lo(p1 y0)
      "madc.hi.u32     m2, %5, %2, 0;\n\t"   // m2 = hi(p1 y0) + carry
      "mad.lo.cc.u32   m1, %4, %3, m1;\n\t"  // m1 += lo(p0 y1)
      "madc.hi.cc.u32  m2, %4, %3, m2;\n\t"  // m2 += hi(p0 y1) + carry
      "addc.u32        m3, 0, 0;\n\t"        // m3 = carry
      "mad.lo.cc.u32   q0, %5, %3, m2;\n\t"  // q0 = lo(p1 y1) + m2
      "madc.hi.u32     q1, %5, %3, m3;\n\t"  // q1 = hi(p1 y1) + m3 + carry
      "mul.lo.u32      %0, %6, %2;\n\t"      // r = w y mod 2^64
      "mul.hi.u32      %1, %6, %2;\n\t"
      "mad.lo.u32      %1, %7, %2, %1;\n\t"
      "mad.lo.u32      %1, %6, %3, %1;\n\t"
      "mad.lo.cc.u32   %0, q0, %8, %0;\n\t"  // r += qh (2^64 - q) mod 2^64
      "madc.hi.u32     %1, q0, %8, %1;\n\t"
      "mad.lo.u32      %1, q1, %8, %1;\n\t"
      "mad.lo.u32      %1, q0, %9, %1;\n\t"
      "}"
      : "=&r"(r0), "=&r"(r1)
      : "r"((uint32_t)y), "r"((uint32_t)(y >> 32)), "r"((uint32_t)wp),
        "r"((uint32_t)(wp >> 32)), "r"((uint32_t)w), "r"((uint32_t)(w >> 32)),
        "r"((uint32_t)nq), "r"((uint32_t)(nq >> 32)));
  return ((uint64_t)r1 << 32) | r0;
}

// x - m if x >= m else x, for x < 2^(beta-1) + m and m <= 2^(beta-1) (all
// lazy values here are < 2^(beta-2)): the sign of x - m decides.
template <typename W>
__device__ __forceinline__ W csub(W x, W m) {
  const W t = x - m;
  return (typename WordT<W>::SW)t < 0 ? x : t;
}

// 64-bit words: the borrow of the subtraction's carry chain as a mask and a
// bitwise select (lop3: mask ? x : x - m) instead of a compare and selects.
__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t m) {
  uint32_t lo, hi;
  asm("{\n\t.reg .u32 b, tl, th;\n\t"
      "sub.cc.u32 tl, %2, %4;\n\t"
      "subc.cc.u32 th, %3, %5;\n\t"
      "subc.u32 b, 0, 0;\n\t"
      "lop3.b32 %0, tl, %2, b, 0xD8;\n\t"
      "lop3.b32 %1, th, %3, b, 0xD8;\n\t"
      "}"
      : "=r"(lo), "=r"(hi)
      : "r"((uint32_t)x), "r"((uint32_t)(x >> 32)), "r"((uint32_t)m), "r"((uint32_t)(m >> 32)));
  return ((uint64_t)hi << 32) | lo;
}

// Merged-CT butterfly (Algorithm 6 body):
//   (x, y) <- (x + w y, x - w y) mod q
// on lazy representatives in [0, 4q).
template <typename W>
__device__ __forceinline__ void ct_bfly(W& x, W& y, W w, W wp, W q, W two_q) {
  const W a = csub(x, two_q);               // [0, 2q)
  const W t = mul_shoup_lazy(y, w, wp, q);  // [0, 2q)
  x = a + t;                                // [0, 4q)
  y = a - t + two_q;                        // (0, 4q)
}

// x/2 mod q for x in [0, 2q): x >> 1 plus (q+1)/2 when x is odd (Sec. III-A).
// Result in [0, 2q).
template <typename W>
__device__ __forceinline__ W half_lazy(W x, W half_q1) {
  return (x >> 1) + ((x & 1) ? half_q1 : W(0));
}

// Merged-GS butterfly (Algorithm 7 body) with the 1/2 scaling of Eq. 2:
//   (x, y) <- ((x + y)/2, w (x - y)/2) mod q
// w2 = w * 2^-1 mod q is the table entry, so the second output needs no
// separate halving.  Lazy representatives in [0, 2q).
template <typename W>
__device__ __forceinline__ void gs_bfly_half(W& x, W& y, W w2, W w2p, W q, W two_q, W half_q1) {
  const W s = csub(x + y, two_q);           // [0, 2q)
  const W d = x - y + two_q;                // (0, 4q)
  x = half_lazy(s, half_q1);                // [0, 2q)
  y = mul_shoup_lazy(d, w2, w2p, q);        // [0, 2q)
}

// Merged-GS butterfly (Algorithm 7 body) without scaling:
//   (x, y) <- (x + y, w (x - y)) mod q
// on lazy representatives in [0, 2q); 1/N is applied by gs_bfly_last.
template <typename W>
__device__ __forceinline__ void gs_bfly(W& x, W& y, W w, W wp, W q, W two_q) {
  const W s = csub(x + y, two_q);           // [0, 2q)
  const W d = x - y + two_q;                // (0, 4q)
  x = s;
  y = mul_shoup_lazy(d, w, wp, q);          // [0, 2q)
}

// The last GS stage (k = N/2, twiddle Psi^-1_br[1]) with 1/N folded in:
//   (x, y) <- ((x + y) / N, w (x - y) / N) mod q, results in [0, 2q).
template <typename W, typename LC>
__device__ __forceinline__ void gs_bfly_last(W& x, W& y, const LC& k) {
  const W s = x + y;                        // [0, 4q)
  const W d = x - y + k.two_q;              // (0, 4q)
  x = mul_shoup_lazy(s, k.ninv, k.ninv_p, k.q);
  y = mul_shoup_lazy(d, k.w1ninv, k.w1ninv_p, k.q);
}

// One GS butterfly in the plan's scaling mode.
template <bool HALVE, typename W>
__device__ __forceinline__ void gs_bfly_mode(W& x, W& y, W w, W wp, W q, W two_q, W hq) {
  if constexpr (HALVE)
    gs_bfly_half(x, y, w, wp, q, two_q, hq);
  else
    gs_bfly(x, y, w, wp, q, two_q);
}

// [0, 4q) -> [0, q)
template <typename W>
__device__ __forceinline__ W reduce4(W x, W q, W two_q) {
  return csub(csub(x, two_q), q);
}

// ---------------------------------------------------------------------------
// Wide lazy ranges ("headroom 16"): 64-bit words with q < 2^60, so that every
// value below 16q fits a word.  The kernels of the 1024-word split then let
// values grow instead of reducing at every butterfly:
//   forward CT words stay below 16q; a butterfly whose input bound is B
//   outputs values below B + 2q, and one that first reduces x by 8q
//   (x - 8q if x >= 8q, valid for x < 16q) outputs values below 10q.  From a
//   canonical input, 7 stages need no reduction; afterwards every fourth
//   stage reduces.
//   inverse GS words stay below 8q: the difference is formed as x - y + 8q
//   (positive for y < 8q, below 16q), the sum x + y is reduced by 8q once it
//   can reach 16q, i.e. from the fourth stage on (canonical input: bounds q,
//   2q, 4q, 8q).
// The classic ranges ([0, 4q) forward, [0, 2q) inverse, q < 2^62) are the
// same butterflies with m = 2q and a reduction at every stage.

// Merged-CT butterfly with the reduction constant m and a compile-time
// choice of reducing x first: (x, y) <- (a + w y, a - w y + 2q), a = x or
// csub(x, m).  Shoup's product accepts any y < 2^64.
template <bool RED, typename W>
__device__ __forceinline__ void ct_bfly_m(W& x, W& y, W w, W wp, W q, W two_q, W m) {
  const W a = RED ? csub(x, m) : x;
  const W t = mul_shoup_lazy(y, w, wp, q);  // [0, 2q)
  x = a + t;
  y = a - t + two_q;
}

// Merged-GS butterfly without scaling, with the range constant m (inputs
// below m): (x, y) <- (x + y [reduced by m], w (x - y + m)); the second
// output is in [0, 2q).
template <bool RED, typename W>
__device__ __forceinline__ void gs_bfly_m(W& x, W& y, W w, W wp, W q, W m) {
  const W s = x + y;
  const W d = x - y + m;
  x = RED ? csub(s, m) : s;
  y = mul_shoup_lazy(d, w, wp, q);
}

// The last GS stage with 1/N folded in, inputs below m (m = 2q or 8q):
// both outputs in [0, 2q).
template <typename W, typename LC>
__device__ __forceinline__ void gs_bfly_last_m(W& x, W& y, const LC& k, W m) {
  const W s = x + y;
  const W d = x - y + m;
  x = mul_shoup_lazy(s, k.ninv, k.ninv_p, k.q);
  y = mul_shoup_lazy(d, k.w1ninv, k.w1ninv_p, k.q);
}

// [0, 16q) -> [0, q)
template <typename W>
__device__ __forceinline__ W reduce16(W x, W q, W two_q, W eight_q) {
  return csub(csub(csub(csub(x, eight_q), eight_q >> 1), two_q), q);
}

// Algorithm 4 (the paper's Barrett variant), beta = 64: x = a*b < 2^(2m) for
// a, b < q, c = x >> (m-2); quot = (c * mu) >> (m+3); rem = x - quot*q; one
// correction.  The 128-bit quantities are kept as (hi, lo) pairs; only the
// low word of quot*q is needed because rem < 2q < 2^64.
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

// Algorithm 4 with beta = 32 (m <= 30): x = a*b < 2^(2m) fits one 64-bit
// word, c = x >> (m-2) < 2^(m+2) and c*mu < 2^(2m+4) <= 2^64, so every step
// is a single 64-bit operation; rem < 2q < 2^31 needs only the low words.
__device__ __forceinline__ uint32_t mul_barrett_alg4(uint32_t a, uint32_t b,
                                                     const LimbConst32& k) {
  const uint64_t x = (uint64_t)a * b;
  const uint64_t c = x >> k.sh1;
  const uint64_t quot = (c * k.mu) >> k.sh2;
  const uint32_t rem = (uint32_t)x - (uint32_t)quot * k.q;
  return csub(rem, k.q);
}

}  // namespace pm
