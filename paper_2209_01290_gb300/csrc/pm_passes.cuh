// pm_passes.cuh -- the butterfly passes shared by the kernels (arxiv
// 2209.01290, Algorithms 6 and 7): radix-16 register groups of the merged CT
// and GS transforms, column transforms, and the in-row pipeline that runs the
// 12 in-row stages of a 4096-word row through padded shared memory.
// Everything is a template over the word type W (uint64_t or uint32_t, see
// pm_arith.cuh), deduced from the register arrays.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "pm_arith.cuh"
#include "pm_internal.h"

namespace pm {

constexpr int kRowLog = 12;
constexpr int kRow = 1 << kRowLog;        // 4096 words per row
// Pad words after every 16 words of a row: p(j) = j + P floor(j/16).
// 64-bit words, P = 2: 64-bit shared accesses are served per half-warp and
// 128-bit ones per quarter-warp; layouts 0 and 1 (64-bit, a half-warp reads 16
// consecutive words) and layout 2 (128-bit word pairs, quarter-warp chunks
// 9 th + u/2 are distinct mod 8) are all free of bank conflicts, and every
// layout-2 pair starts on a 16-byte boundary.
// 32-bit words, P = 1: accesses are served per warp (32 banks of 4 bytes);
// layout 2 (17 th) and layout 1 (half-warps 16 banks apart) are conflict-free,
// layout 0 has one 2-way conflict (lanes 0 and 31).
template <typename W>
constexpr int kPadW = sizeof(W) == 8 ? 2 : 1;

// Non-deduced pointer parameter (so that nullptr can be passed for it).
template <typename T>
struct NoDeduce {
  using type = T;
};
template <typename W>
constexpr int kRowPadW = kRow + 256 * kPadW<W>;  // padded row length in words
constexpr int kRowPad = kRowPadW<uint64_t>;

template <typename W = uint64_t>
__device__ __forceinline__ int padj(int j) {
  return j + kPadW<W> * (j >> 4);
}

// ------------------------------------------------------------------ passes

// Four consecutive merged-CT stages (Algorithm 6) on a register group of 16
// words.  Global stages s0..s0+3; the group lies in the (N >> s0)-word block
// number g, its 16 words spaced N >> (s0+4) apart.  Stage s0+st pairs
// (u, u + 8 >> st) with twiddle Psi_br[2^(s0+st) + g 2^st + (u >> (4-st))].
// (Stages are template parameters so every register index is a constant.)
template <int ST, typename W>
__device__ __forceinline__ void ct16_stage1(W (&v)[16], const typename WordT<W>::Tw* __restrict__ tw,
                                            uint32_t s0, uint32_t g, W q, W two_q) {
  using Tw = typename WordT<W>::Tw;
  constexpr int h = 8 >> ST;
  const uint32_t base = (1u << (s0 + ST)) + (g << ST);  // even for ST >= 1
  if constexpr (ST == 0) {
    const Tw t = ld_tw(tw + base);
#pragma unroll
    for (int u0 = 0; u0 < 8; u0++) ct_bfly(v[u0], v[u0 + 8], t.w, t.wp, q, two_q);
  } else {
#pragma unroll
    for (int blk = 0; blk < (1 << ST); blk += 2) {
      Tw t[2];
      ld_tw2(tw + base + blk, t[0], t[1]);
#pragma unroll
      for (int e = 0; e < 2; e++)
#pragma unroll
        for (int u0 = 0; u0 < h; u0++)
          ct_bfly(v[(blk + e) * 2 * h + u0], v[(blk + e) * 2 * h + u0 + h], t[e].w, t[e].wp, q,
                  two_q);
    }
  }
}

// The same four stages on two operands that share the twiddles (a and b of
// one product): each twiddle pair is loaded once and used twice.
template <int ST, typename W>
__device__ __forceinline__ void ct16_stage2(W (&va)[16], W (&vb)[16],
                                            const typename WordT<W>::Tw* __restrict__ tw,
                                            uint32_t s0, uint32_t g, W q, W two_q) {
  constexpr int h = 8 >> ST;
  const uint32_t base = (1u << (s0 + ST)) + (g << ST);  // even for ST >= 1
  constexpr int nb = 1 << ST;
#pragma unroll
  for (int blk = 0; blk < nb; blk += (nb > 1 ? 2 : 1)) {
    typename WordT<W>::Tw t[2];
    if constexpr (nb > 1)
      ld_tw2(tw + base + blk, t[0], t[1]);
    else
      t[0] = ld_tw(tw + base);
#pragma unroll
    for (int e = 0; e < (nb > 1 ? 2 : 1); e++)
#pragma unroll
      for (int u0 = 0; u0 < h; u0++) {
        const int i0 = (blk + e) * 2 * h + u0;
        ct_bfly(va[i0], va[i0 + h], t[e].w, t[e].wp, q, two_q);
        ct_bfly(vb[i0], vb[i0 + h], t[e].w, t[e].wp, q, two_q);
      }
  }
}

// skip_last omits the fourth stage: in the last pass of a forward transform
// that is the transform's final stage, which Algorithm 8 leaves out.
template <typename W>
__device__ __forceinline__ void ct16_2(W (&va)[16], W (&vb)[16],
                                       const typename WordT<W>::Tw* __restrict__ tw, uint32_t s0,
                                       uint32_t g, W q, W two_q, bool skip_last = false) {
  ct16_stage2<0>(va, vb, tw, s0, g, q, two_q);
  ct16_stage2<1>(va, vb, tw, s0, g, q, two_q);
  ct16_stage2<2>(va, vb, tw, s0, g, q, two_q);
  if (!skip_last) ct16_stage2<3>(va, vb, tw, s0, g, q, two_q);
}

template <typename W>
__device__ __forceinline__ void ct16(W (&v)[16], const typename WordT<W>::Tw* __restrict__ tw,
                                     uint32_t s0, uint32_t g, W q, W two_q,
                                     bool skip_last = false) {
  ct16_stage1<0>(v, tw, s0, g, q, two_q);
  ct16_stage1<1>(v, tw, s0, g, q, two_q);
  ct16_stage1<2>(v, tw, s0, g, q, two_q);
  if (!skip_last) ct16_stage1<3>(v, tw, s0, g, q, two_q);
}

// Four consecutive merged-GS stages (Algorithm 7, 1/2-scaled) on a group of
// 16 words.  GS stages sig0..sig0+3 (k = 2^sig); the group is block g of
// 2^(sig0+4) words.  Stage sig0+st pairs (u, u + 2^st) with twiddle
// Psi^-1_br[(N >> (sig0+st+1)) + g 2^(3-st) + (u >> (st+1))] (times 1/2).
template <int ST, bool HALVE, typename W>
__device__ __forceinline__ void gs16_stage(W (&v)[16], const typename WordT<W>::Tw* __restrict__ tw,
                                           uint32_t logn, uint32_t sig0, uint32_t g, W q,
                                           W two_q, W hq) {
  constexpr int h = 1 << ST;
  // base is even whenever the stage needs more than one twiddle (ST <= 2):
  // logn - sig0 - ST - 1 >= 1 there, and g << (3 - ST) is even
  const uint32_t base = (1u << (logn - sig0 - ST - 1)) + (g << (3 - ST));
  constexpr int nb = 8 >> ST;
#pragma unroll
  for (int blk = 0; blk < nb; blk += (nb > 1 ? 2 : 1)) {
    typename WordT<W>::Tw t[2];
    if constexpr (nb > 1)
      ld_tw2(tw + base + blk, t[0], t[1]);
    else
      t[0] = ld_tw(tw + base);
#pragma unroll
    for (int e = 0; e < (nb > 1 ? 2 : 1); e++)
#pragma unroll
      for (int u0 = 0; u0 < h; u0++)
        gs_bfly_mode<HALVE>(v[(blk + e) * 2 * h + u0], v[(blk + e) * 2 * h + u0 + h], t[e].w,
                            t[e].wp, q, two_q, hq);
  }
}

// skip_first omits the first stage (the transform's first when sig0 = 0,
// which Algorithm 8 leaves out).
template <bool HALVE, typename W>
__device__ __forceinline__ void gs16(W (&v)[16], const typename WordT<W>::Tw* __restrict__ tw,
                                     uint32_t logn, uint32_t sig0, uint32_t g, W q, W two_q,
                                     W hq, bool skip_first = false) {
  if (!skip_first) gs16_stage<0, HALVE>(v, tw, logn, sig0, g, q, two_q, hq);
  gs16_stage<1, HALVE>(v, tw, logn, sig0, g, q, two_q, hq);
  gs16_stage<2, HALVE>(v, tw, logn, sig0, g, q, two_q, hq);
  gs16_stage<3, HALVE>(v, tw, logn, sig0, g, q, two_q, hq);
}

// Merged CT on a column of R words (the first log2 R stages of the N-point
// transform): stage s pairs (t, t + R >> (s+1)) with twiddle Psi_br[2^s + blk].
// RED = false (wide lazy ranges, canonical input, R <= 128) reduces nothing:
// the outputs stay below (1 + 2 log2 R) q <= 15q.
template <int R, int S, bool RED, typename W>
__device__ __forceinline__ void ct_col_stage(W (&x)[R], const typename WordT<W>::Tw* __restrict__ tw,
                                             W q, W two_q) {
  if constexpr ((1 << S) < R) {
    constexpr int h = R >> (S + 1);
    constexpr int nb = 1 << S;
#pragma unroll
    for (int blk = 0; blk < nb; blk += (nb > 1 ? 2 : 1)) {
      typename WordT<W>::Tw t[2];
      if constexpr (nb > 1)
        ld_tw2(tw + nb + blk, t[0], t[1]);  // index nb + blk is even
      else
        t[0] = ld_tw(tw + 1);
#pragma unroll
      for (int e = 0; e < (nb > 1 ? 2 : 1); e++)
#pragma unroll
        for (int u0 = 0; u0 < h; u0++)
          ct_bfly_m<RED>(x[(blk + e) * 2 * h + u0], x[(blk + e) * 2 * h + u0 + h], t[e].w,
                         t[e].wp, q, two_q, two_q);
    }
    ct_col_stage<R, S + 1, RED>(x, tw, q, two_q);
  }
}

template <int R, typename W, bool RED = true>
__device__ __forceinline__ void ct_col(W (&x)[R], const typename WordT<W>::Tw* __restrict__ tw,
                                       W q, W two_q) {
  ct_col_stage<R, 0, RED>(x, tw, q, two_q);
}

// Merged GS on a column of R words (the last log2 R stages): the GS stage
// with k = 4096 * 2^E pairs (t, t + 2^E) with twiddle
// Psi^-1_br[(R >> (E+1)) + (t >> (E+1))].  Without per-stage halving the
// final stage (2^E = R/2, the transform's last) folds in 1/N.  LZ (wide
// lazy ranges, never with halving): inputs below 8q, every sum reduced by
// 8q, differences formed with + 8q.
template <int R, int E, bool HALVE, bool LZ, typename W>
__device__ __forceinline__ void gs_col_stage(W (&x)[R], const typename WordT<W>::Tw* __restrict__ tw,
                                             const typename WordT<W>::LC& K) {
  static_assert(!(LZ && HALVE), "wide lazy ranges fold 1/N at the end");
  if constexpr ((1 << E) < R) {
    constexpr int h = 1 << E;
    const W m = LZ ? W(K.two_q << 2) : K.two_q;
    if constexpr (!HALVE && 2 * h == R) {
#pragma unroll
      for (int u0 = 0; u0 < h; u0++) gs_bfly_last_m(x[u0], x[u0 + h], K, m);
    } else {
      constexpr int nb = R / (2 * h);  // table index nb + blk, even when nb > 1
#pragma unroll
      for (int blk = 0; blk < nb; blk += (nb > 1 ? 2 : 1)) {
        typename WordT<W>::Tw t[2];
        if constexpr (nb > 1)
          ld_tw2(tw + nb + blk, t[0], t[1]);
        else
          t[0] = ld_tw(tw + 1);
#pragma unroll
        for (int e = 0; e < (nb > 1 ? 2 : 1); e++)
#pragma unroll
          for (int u0 = 0; u0 < h; u0++) {
            W& a = x[(blk + e) * 2 * h + u0];
            W& b = x[(blk + e) * 2 * h + u0 + h];
            if constexpr (LZ)
              gs_bfly_m<true>(a, b, t[e].w, t[e].wp, K.q, m);
            else
              gs_bfly_mode<HALVE>(a, b, t[e].w, t[e].wp, K.q, K.two_q, K.half_q1);
          }
      }
    }
    gs_col_stage<R, E + 1, HALVE, LZ>(x, tw, K);
  }
}

template <int R, bool HALVE, typename W, bool LZ = false>
__device__ __forceinline__ void gs_col(W (&x)[R], const typename WordT<W>::Tw* __restrict__ tw,
                                       const typename WordT<W>::LC& K) {
  gs_col_stage<R, 0, HALVE, LZ>(x, tw, K);
}

__device__ __forceinline__ LimbConst ld_limb(const LimbConst* __restrict__ p) {
  LimbConst k;
  const ulonglong2* s = reinterpret_cast<const ulonglong2*>(p);
  const ulonglong2 v0 = __ldg(s), v1 = __ldg(s + 1), v2 = __ldg(s + 2), v3 = __ldg(s + 3),
                   v4 = __ldg(s + 4);
  k.q = v0.x;
  k.two_q = v0.y;
  k.half_q1 = v1.x;
  k.mu = v1.y;
  k.m = (uint32_t)v2.x;
  k.sh1 = (uint32_t)(v2.x >> 32);
  k.sh2 = (uint32_t)v2.y;
  k.halving = (uint32_t)(v2.y >> 32);
  k.ninv = v3.x;
  k.ninv_p = v3.y;
  k.w1ninv = v4.x;
  k.w1ninv_p = v4.y;
  return k;
}

__device__ __forceinline__ LimbConst32 ld_limb(const LimbConst32* __restrict__ p) {
  LimbConst32 k;
  const uint4* s = reinterpret_cast<const uint4*>(p);
  const uint4 v0 = __ldg(s), v1 = __ldg(s + 1), v2 = __ldg(s + 2);
  k.q = v0.x;
  k.two_q = v0.y;
  k.half_q1 = v0.z;
  k.mu = v0.w;
  k.m = v1.x;
  k.sh1 = v1.y;
  k.sh2 = v1.z;
  k.halving = v1.w;
  k.ninv = v2.x;
  k.ninv_p = v2.y;
  k.w1ninv = v2.z;
  k.w1ninv_p = v2.w;
  return k;
}

// Kernels are templates over the word type W (uint64_t: q < 2^62;
// uint32_t: q < 2^30); KParams carries untyped device pointers and KView<W>
// gives the typed views.

template <typename W>
struct KView {
  const W* a;
  const W* b;
  W* c;
  W* s;
  const typename WordT<W>::Tw* twf;
  const typename WordT<W>::Tw* twi;
  const typename WordT<W>::LC* lc;
  __device__ __forceinline__ explicit KView(const KParams& P)
      : a(reinterpret_cast<const W*>(P.a)),
        b(reinterpret_cast<const W*>(P.b)),
        c(reinterpret_cast<W*>(P.c)),
        s(reinterpret_cast<W*>(P.s)),
        twf(reinterpret_cast<const typename WordT<W>::Tw*>(P.twf)),
        twi(reinterpret_cast<const typename WordT<W>::Tw*>(P.twi)),
        lc(reinterpret_cast<const typename WordT<W>::LC*>(P.lc)) {}
};

// ----------------------------------------------------------- row pipeline

// The 12 in-row stages of one 4096-word row (row t of a unit of 2^logn
// words) as three radix-16 passes; 256 threads per row.  Each pass reads 16
// words per thread, runs 4 stages in registers and writes them back.  The
// three thread->word layouts
//   layout 0: j = th + 256 u                      (CT stages n-12.., GS 8..11)
//   layout 1: j = 256 (th>>4) + (th&15) + 16 u    (CT stages n-8..,  GS 4..7)
//   layout 2: j = 16 th + u                       (CT stages n-4..,  GS 0..3)
// use the padding described at kPadW.  The pass loop of the one-operand
// transforms is not unrolled: one copy of the radix-16 body serves all
// passes, which keeps the kernel small enough for the instruction cache.
struct PassGeo {
  int layout;    // 0, 1 or 2
  int pbase;     // padded smem index of u = 0
  uint32_t g;    // block index of the group within the whole transform
};

// With the padding p(j) = j + P floor(j/16), the padded index of word u of a
// group is pbase + off(u) with a compile-time offset per layout:
//   layout 0: (256 + 16 P) u;  layout 1: (16 + P) u;  layout 2: u.
template <int L, typename W>
__device__ __forceinline__ constexpr int lay_off(int u) {
  constexpr int P = kPadW<W>;
  return L == 0 ? (256 + 16 * P) * u : (L == 1 ? (16 + P) * u : u);
}

template <typename W = uint64_t>
__device__ __forceinline__ PassGeo pass_geo(int layout, int th, uint32_t t) {
  constexpr int P = kPadW<W>;
  PassGeo G;
  G.layout = layout;
  if (layout == 0) {
    G.pbase = th + P * (th >> 4);
    G.g = t;
  } else if (layout == 1) {
    G.pbase = (256 + 16 * P) * (th >> 4) + (th & 15);
    G.g = t * 16 + (th >> 4);
  } else {
    G.pbase = (16 + P) * th;
    G.g = t * 256 + th;
  }
  return G;
}

// With 64-bit words, layout 2 moves its 16 consecutive words as 8 16-byte
// pairs; 32-bit words move one by one.
template <int L, typename W>
__device__ __forceinline__ void ld16(W (&v)[16], const W* s) {
  if constexpr (L == 2 && sizeof(W) == 8) {
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(s);
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const ulonglong2 w = s2[k];
      v[2 * k] = w.x;
      v[2 * k + 1] = w.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 16; u++) v[u] = s[lay_off<L, W>(u)];
  }
}

template <int L, typename W>
__device__ __forceinline__ void st16(W* s, const W (&v)[16]) {
  if constexpr (L == 2 && sizeof(W) == 8) {
    ulonglong2* s2 = reinterpret_cast<ulonglong2*>(s);
#pragma unroll
    for (int k = 0; k < 8; k++) s2[k] = make_ulonglong2(v[2 * k], v[2 * k + 1]);
  } else {
#pragma unroll
    for (int u = 0; u < 16; u++) s[lay_off<L, W>(u)] = v[u];
  }
}

template <typename W>
__device__ __forceinline__ void ld_smem16(W (&v)[16], const W* s, const PassGeo& G) {
  const W* p = s + G.pbase;
  if (G.layout == 0) ld16<0>(v, p);
  else if (G.layout == 1) ld16<1>(v, p);
  else ld16<2>(v, p);
}

template <typename W>
__device__ __forceinline__ void st_smem16(W* s, const PassGeo& G, const W (&v)[16]) {
  W* p = s + G.pbase;
  if (G.layout == 0) st16<0>(p, v);
  else if (G.layout == 1) st16<1>(p, v);
  else st16<2>(p, v);
}

// Global loads of data written earlier in the same launch (persistent
// kernel) must bypass L1: CG selects ld.global.cg, otherwise the streaming
// ld.global.cs hint is used.
template <bool CG, typename W>
__device__ __forceinline__ W ld_g(const W* p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return __ldcs(p);
}

// Forward in-row stages of one operand.  Source: global row `g_src` (layout
// 0, coalesced) or, if null, the smem row `s` (already holding the row).
// Leaves the last pass's 16 words (layout 2, lazy [0,4q)) in v.
// With `trunc` the transform's final stage is omitted (Algorithm 8's
// truncated CT transform).
template <bool CG = false, typename W>
__device__ __forceinline__ void rows_fwd(W (&v)[16], const typename NoDeduce<W>::type* g_src, W* s,
                                         const typename WordT<W>::Tw* __restrict__ twf,
                                         uint32_t logn, uint32_t t, int th, W q, W two_q,
                                         bool trunc = false) {
#pragma unroll 1
  for (int p = 0; p < 3; p++) {
    const PassGeo G = pass_geo<W>(p, th, t);
    if (p == 0 && g_src) {
#pragma unroll
      for (int u = 0; u < 16; u++) v[u] = ld_g<CG>(g_src + th + 256 * u);
    } else {
      ld_smem16(v, s, G);
    }
    ct16(v, twf, logn - 12 + 4 * p, G.g, q, two_q, trunc && p == 2);
    if (p < 2) {
      st_smem16(s, G, v);
      // pass 1 -> 2 stays inside a half-warp: the layout-1 block g of 256
      // words is owned by threads 16g..16g+15, which are exactly the layout-2
      // threads that read it; pass 0 -> 1 crosses warps.
      if (p == 0)
        __syncthreads();
      else
        __syncwarp();
    }
  }
}

// Inverse in-row stages (1/2-scaled).  v holds layout-2 words on entry.
// The last pass writes layout 0 either to the global row `g_dst`
// (canonical if `final`) or, if null, back to smem.
// With `final` (the row is the whole transform, N = 4096) and no per-stage
// halving, the outputs are multiplied by N^-1 (K.ninv) before the store.
// With `trunc` the transform's first stage is omitted (Algorithm 8's
// truncated GS transform).
template <bool HALVE, typename W>
__device__ __forceinline__ void rows_inv(W (&v)[16], typename NoDeduce<W>::type* g_dst, bool final,
                                         W* s,
                                         const typename WordT<W>::Tw* __restrict__ twi,
                                         uint32_t logn, uint32_t t, int th,
                                         const typename WordT<W>::LC& K, bool trunc = false) {
  const W q = K.q, two_q = K.two_q, hq = K.half_q1;
#pragma unroll 1
  for (int p = 0; p < 3; p++) {
    const PassGeo G = pass_geo<W>(2 - p, th, t);
    if (p > 0) ld_smem16(v, s, G);
    gs16<HALVE>(v, twi, logn, 4 * p, G.g, q, two_q, hq, trunc && p == 0);
    if (p < 2) {
      st_smem16(s, G, v);
      // layout 2 -> 1 stays inside a half-warp, layout 1 -> 0 crosses warps
      if (p == 0)
        __syncwarp();
      else
        __syncthreads();
    }
  }
  if (g_dst) {
    if (!HALVE && final) {
#pragma unroll
      for (int u = 0; u < 16; u++) v[u] = mul_shoup_lazy(v[u], K.ninv, K.ninv_p, q);
    }
#pragma unroll
    for (int u = 0; u < 16; u++) __stcs(g_dst + th + 256 * u, final ? csub(v[u], q) : v[u]);
  } else {
    st_smem16(s, pass_geo<W>(0, th, t), v);
  }
}


// Forward in-row stages of a and b together (shared twiddles); leaves the
// layout-2 words of both in va, vb.
template <bool CG = false, typename W>
__device__ __forceinline__ void rows_fwd2(W (&va)[16], W (&vb)[16], const W* ga, const W* gb,
                                          W* sa, W* sb,
                                          const typename WordT<W>::Tw* __restrict__ twf,
                                          uint32_t logn, uint32_t t, int th, W q, W two_q,
                                          bool trunc = false) {
  // unrolled: with the layout of every pass known at compile time the
  // scheduler interleaves the two operands' loads and butterflies across
  // the pass (measured faster than the rolled loop here, unlike rows_fwd)
#pragma unroll
  for (int p = 0; p < 3; p++) {
    const PassGeo G = pass_geo<W>(p, th, t);
    if (p == 0) {
#pragma unroll
      for (int u = 0; u < 16; u++) {
        va[u] = ld_g<CG>(ga + th + 256 * u);
        vb[u] = ld_g<CG>(gb + th + 256 * u);
      }
    } else {
      ld_smem16(va, sa, G);
      ld_smem16(vb, sb, G);
    }
    ct16_2(va, vb, twf, logn - 12 + 4 * p, G.g, q, two_q, trunc && p == 2);
    if (p < 2) {
      st_smem16(sa, G, va);
      st_smem16(sb, G, vb);
      if (p == 0)
        __syncthreads();
      else
        __syncwarp();
    }
  }
}

// Algorithm 8's fused step for one pair of bit-reversed positions (2i, 2i+1):
// (x0, x1) from the truncated CT transform of a, (y0, y1) from that of b,
// lazy in [0, 4q).  With gamma = (-1)^i Psi_br[N/4 + floor(i/2)] (the square
// of the omitted last stage's twiddle Psi_br[N/2 + i]):
//   x0 <- x0 y0 + gamma x1 y1,   x1 <- x0 y1 + x1 y0 = (x0+x1)(y0+y1) - x0 y0 - x1 y1
// with three Algorithm 4 products and one Shoup product by Psi_br[..]; the
// sign (-1)^i is a compile-time choice between u + z and u - z.  This is the
// first GS stage's output with its 1/2, in [0, 2q).
// With LZ (the wide lazy ranges of the 1024-word rows) the inputs may be
// anything below 16q.
template <bool ODD, bool LZ = false, typename W>
__device__ __forceinline__ void fused_pair(W& x0, W& x1, W y0, W y1,
                                           const typename WordT<W>::Tw& w,
                                           const typename WordT<W>::LC& K) {
  const W q = K.q, two_q = K.two_q;
  auto red = [&](W x) { return LZ ? reduce16(x, q, two_q, W(two_q << 2)) : reduce4(x, q, two_q); };
  const W a0 = red(x0), a1 = red(x1);
  const W b0 = red(y0), b1 = red(y1);
  const W u = mul_barrett_alg4(a0, b0, K);                                      // [0, q)
  const W v = mul_barrett_alg4(a1, b1, K);                                      // [0, q)
  const W w3 = mul_barrett_alg4(csub(W(a0 + a1), q), csub(W(b0 + b1), q), K);  // [0, q)
  const W z = mul_shoup_lazy(v, w.w, w.wp, q);                                  // [0, 2q)
  x1 = csub(W(w3 + two_q - u - v), two_q);                                      // (0,3q) -> [0,2q)
  x0 = csub(W(ODD ? u + two_q - z : u + z), two_q);                             // [0,3q) -> [0,2q)
}

// The fused step on the 8 pairs (u, u+1) of a layout-2 register group (group
// g = 256 t + th holds bit-reversed positions 16 g + u): pair i = 8 g + u/2,
// so floor(i/2) = 4 g + u/4 and i is odd when u/2 is.  Result in va.  The
// step is symmetric in the two operands; the other operand comes from
// registers (vb) or from its layout-2 words in shared memory (sb, 16-byte
// pairs).
template <typename W>
__device__ __forceinline__ void fused_pairs16(W (&va)[16], const W (&vb)[16],
                                              const typename WordT<W>::Tw* __restrict__ twf,
                                              uint32_t logn, uint32_t g,
                                              const typename WordT<W>::LC& K) {
  const uint32_t base = (1u << (logn - 2)) + 4 * g;  // even
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    typename WordT<W>::Tw w[2];
    ld_tw2(twf + base + k, w[0], w[1]);
#pragma unroll
    for (int e = 0; e < 2; e++) {
      const int u = 4 * (k + e);
      fused_pair<false>(va[u], va[u + 1], vb[u], vb[u + 1], w[e], K);
      fused_pair<true>(va[u + 2], va[u + 3], vb[u + 2], vb[u + 3], w[e], K);
    }
  }
}

template <typename W>
__device__ __forceinline__ void fused_pairs16_smem(W (&va)[16], const W* sb,
                                                   const typename WordT<W>::Tw* __restrict__ twf,
                                                   uint32_t logn, uint32_t g,
                                                   const typename WordT<W>::LC& K) {
  const uint32_t base = (1u << (logn - 2)) + 4 * g;  // even
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    typename WordT<W>::Tw w[2];
    ld_tw2(twf + base + k, w[0], w[1]);
#pragma unroll
    for (int e = 0; e < 2; e++) {
      const int u = 4 * (k + e);
      W y[4];
      if constexpr (sizeof(W) == 8) {
        const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sb);
        const ulonglong2 p0 = s2[u / 2], p1 = s2[u / 2 + 1];
        y[0] = p0.x;
        y[1] = p0.y;
        y[2] = p1.x;
        y[3] = p1.y;
      } else {
#pragma unroll
        for (int i = 0; i < 4; i++) y[i] = sb[u + i];
      }
      fused_pair<false>(va[u], va[u + 1], y[0], y[1], w[e], K);
      fused_pair<true>(va[u + 2], va[u + 3], y[2], y[3], w[e], K);
    }
  }
}

// Algorithm 4 products of a register group with the other operand's
// layout-2 words in shared memory (16-byte pairs).
template <typename W>
__device__ __forceinline__ void pointwise16(W (&v)[16], const W* sb,
                                            const typename WordT<W>::LC& K) {
#pragma unroll
  for (int k = 0; k < 8; k++) {
    W y0, y1;
    if constexpr (sizeof(W) == 8) {
      const ulonglong2 y = reinterpret_cast<const ulonglong2*>(sb)[k];
      y0 = y.x;
      y1 = y.y;
    } else {
      y0 = sb[2 * k];
      y1 = sb[2 * k + 1];
    }
    v[2 * k] = mul_barrett_alg4(reduce4(y0, K.q, K.two_q), reduce4(v[2 * k], K.q, K.two_q), K);
    v[2 * k + 1] =
        mul_barrett_alg4(reduce4(y1, K.q, K.two_q), reduce4(v[2 * k + 1], K.q, K.two_q), K);
  }
}

// The product step between the forward and inverse in-row stages: Algorithm
// 4 pointwise products (Eq. 2) or, with `fused`, Algorithm 8's pair step.
template <typename W>
__device__ __forceinline__ void row_product(W (&va)[16], const W (&vb)[16], bool fused,
                                            const typename WordT<W>::Tw* __restrict__ twf,
                                            uint32_t logn, uint32_t g,
                                            const typename WordT<W>::LC& K) {
  if (fused) {
    fused_pairs16(va, vb, twf, logn, g, K);
  } else {
#pragma unroll
    for (int u = 0; u < 16; u++)
      va[u] = mul_barrett_alg4(reduce4(va[u], K.q, K.two_q), reduce4(vb[u], K.q, K.two_q), K);
  }
}

// Polymul row task with both operands in registers at once (2 CTAs per SM).
template <bool HALVE, bool CG, typename W>
__device__ __forceinline__ void row_task_polymul2(const W* ga, const W* gb, W* gc, bool single,
                                                  W* smem,
                                                  const typename WordT<W>::Tw* __restrict__ twf,
                                                  const typename WordT<W>::Tw* __restrict__ twi,
                                                  const typename WordT<W>::LC& K, uint32_t logn,
                                                  uint32_t t, bool fused = false) {
  const int th = threadIdx.x;
  W* sa = smem;
  W* sb = smem + kRowPadW<W>;
  W va[16], vb[16];
  rows_fwd2<CG>(va, vb, ga, gb, sa, sb, twf, logn, t, th, K.q, K.two_q, fused);
  row_product(va, vb, fused, twf, logn, pass_geo<W>(2, th, t).g, K);
  rows_inv<HALVE>(va, gc, single, sa, twi, logn, t, th, K, fused);
}

// Polymul row task: forward in-row stages of a and b, Algorithm 4 pointwise
// product, inverse in-row stages, for row t of `unit`.  `ga`, `gb` are the
// global rows of the operands (the column-transformed images for N > 4096),
// `gc` the output row.  `smem` holds 2 padded rows.
// With `fused` the task follows Algorithm 8 (truncated transforms around
// the pair step); K must then hold the fused constants (2/N).
template <bool HALVE, bool CG, typename W>
__device__ __forceinline__ void row_task_polymul(const W* ga, const W* gb, W* gc, bool single,
                                                 W* smem,
                                                 const typename WordT<W>::Tw* __restrict__ twf,
                                                 const typename WordT<W>::Tw* __restrict__ twi,
                                                 const typename WordT<W>::LC& K, uint32_t logn,
                                                 uint32_t t, bool fused = false) {
  const int th = threadIdx.x;
  W* sa = smem;
  W* sb = smem + kRowPadW<W>;
  W v[16];
  // operand a: keep its transform in smem (layout 2) while b is done
  rows_fwd<CG>(v, ga, sa, twf, logn, t, th, K.q, K.two_q, fused);
  const PassGeo G2 = pass_geo<W>(2, th, t);
  st_smem16(sa, G2, v);
  rows_fwd<CG>(v, gb, sb, twf, logn, t, th, K.q, K.two_q, fused);
  // product step in bit-reversed order (Algorithm 4 products, or Algorithm
  // 8's pair step); each thread re-reads only the words it stored itself
  const W* a2 = sa + G2.pbase;
  if (fused)
    fused_pairs16_smem(v, a2, twf, logn, G2.g, K);
  else
    pointwise16(v, a2, K);
  rows_inv<HALVE>(v, gc, single, sa, twi, logn, t, th, K, fused);
}

// ------------------------------------------------- latency row pipeline
// The 12 in-row stages of a 4096-word row as six radix-4 passes over 1024
// threads (4 words per thread and operand): a row task spread over 32 warps
// of one SM, for batches too small to fill the GPU with the radix-16 rows.
// Pass p (forward order) covers in-row stages 2p, 2p+1; its groups are 4
// words spaced 2^e apart, e = 10 - 2p, inside blocks of 2^(e+2) words:
//   j = blk 2^(e+2) + off + u 2^e,  off < 2^e.
// Threads are mapped offset-fastest for e >= 4 (a half-warp or warp reads
// consecutive words) and block-fastest for e < 4.  Shared memory is padded
// one word per 16 (64-bit words) or per 32 (32-bit words): all six layouts
// are then free of bank conflicts for 64-bit words, and have one 2-way
// conflict (pass e = 4) for 32-bit words.  The inverse runs the layouts in
// reverse order (GS stages 2p', 2p'+1 on the layout of pass 5 - p').
constexpr int kLatThreads = 1024;

template <typename W>
constexpr int kLatShift = sizeof(W) == 8 ? 4 : 5;
template <typename W>
constexpr int kLatRowPad = kRow + (kRow >> kLatShift<W>);

struct LatGeo {
  int pbase;    // padded smem index of u = 0
  uint32_t g;   // block index of the group within the whole transform
};

template <typename W>
__device__ __forceinline__ LatGeo lat_geo(int p, int th, uint32_t t) {
  const int e = 10 - 2 * p;
  int blk, off;
  if (e >= 4) {
    off = th & ((1 << e) - 1);
    blk = th >> e;
  } else {
    blk = th & ((1 << (10 - e)) - 1);
    off = th >> (10 - e);
  }
  const int j0 = (blk << (e + 2)) + off;
  LatGeo G;
  G.pbase = j0 + (j0 >> kLatShift<W>);
  G.g = (t << (2 * p)) + (uint32_t)blk;
  return G;
}

// Padded offset of word u of a group relative to u = 0 (compile-time per
// pass): u 2^e plus the pad words crossed (none inside the group's 16- or
// 32-word block when the stride is small; for 32-bit words and e = 4 the
// group starts at offset off < 16 of its 32-word block).
template <typename W, int E>
__device__ __forceinline__ constexpr int lat_off(int u) {
  constexpr int S = kLatShift<W>;
  if constexpr (E >= S)
    return u * ((1 << E) + (1 << (E - S)));
  else if constexpr (E == 4)
    return 16 * u + (u >> 1);
  else
    return u << E;
}

template <typename W, int E>
__device__ __forceinline__ void lat_ld(W (&v)[4], const W* s, int pbase) {
#pragma unroll
  for (int u = 0; u < 4; u++) v[u] = s[pbase + lat_off<W, E>(u)];
}

template <typename W, int E>
__device__ __forceinline__ void lat_st(W* s, int pbase, const W (&v)[4]) {
#pragma unroll
  for (int u = 0; u < 4; u++) s[pbase + lat_off<W, E>(u)] = v[u];
}

// Two consecutive merged-CT stages on a group of 4 words (global stages s0,
// s0+1; the group is block g at stage s0): stage s0 pairs (u, u+2) with
// twiddle Psi_br[2^s0 + g]; stage s0+1 pairs (u, u+1) with
// Psi_br[2^(s0+1) + 2g + u/2].  skip_last omits the second stage.
template <typename W>
__device__ __forceinline__ void ct4(W (&v)[4], const typename WordT<W>::Tw* __restrict__ tw,
                                    uint32_t s0, uint32_t g, W q, W two_q, bool skip_last) {
  const auto t0 = ld_tw(tw + (1u << s0) + g);
  ct_bfly(v[0], v[2], t0.w, t0.wp, q, two_q);
  ct_bfly(v[1], v[3], t0.w, t0.wp, q, two_q);
  if (!skip_last) {
    typename WordT<W>::Tw t1[2];
    ld_tw2(tw + (1u << (s0 + 1)) + 2 * g, t1[0], t1[1]);
    ct_bfly(v[0], v[1], t1[0].w, t1[0].wp, q, two_q);
    ct_bfly(v[2], v[3], t1[1].w, t1[1].wp, q, two_q);
  }
}

// The same on two operands sharing the twiddles.
template <typename W>
__device__ __forceinline__ void ct4_2(W (&va)[4], W (&vb)[4],
                                      const typename WordT<W>::Tw* __restrict__ tw, uint32_t s0,
                                      uint32_t g, W q, W two_q, bool skip_last) {
  const auto t0 = ld_tw(tw + (1u << s0) + g);
  ct_bfly(va[0], va[2], t0.w, t0.wp, q, two_q);
  ct_bfly(va[1], va[3], t0.w, t0.wp, q, two_q);
  ct_bfly(vb[0], vb[2], t0.w, t0.wp, q, two_q);
  ct_bfly(vb[1], vb[3], t0.w, t0.wp, q, two_q);
  if (!skip_last) {
    typename WordT<W>::Tw t1[2];
    ld_tw2(tw + (1u << (s0 + 1)) + 2 * g, t1[0], t1[1]);
    ct_bfly(va[0], va[1], t1[0].w, t1[0].wp, q, two_q);
    ct_bfly(va[2], va[3], t1[1].w, t1[1].wp, q, two_q);
    ct_bfly(vb[0], vb[1], t1[0].w, t1[0].wp, q, two_q);
    ct_bfly(vb[2], vb[3], t1[1].w, t1[1].wp, q, two_q);
  }
}

// Two consecutive merged-GS stages on a group of 4 words (GS stages sig0,
// sig0+1; the group is block g of 2^(sig0+2) words): stage sig0 pairs
// (u, u+1) with twiddle Psi^-1_br[(N >> (sig0+1)) + 2g + u/2]; stage sig0+1
// pairs (u, u+2) with Psi^-1_br[(N >> (sig0+2)) + g].  skip_first omits the
// first stage.
template <bool HALVE, typename W>
__device__ __forceinline__ void gs4(W (&v)[4], const typename WordT<W>::Tw* __restrict__ tw,
                                    uint32_t logn, uint32_t sig0, uint32_t g, W q, W two_q, W hq,
                                    bool skip_first) {
  if (!skip_first) {
    typename WordT<W>::Tw t0[2];
    ld_tw2(tw + (1u << (logn - sig0 - 1)) + 2 * g, t0[0], t0[1]);  // even index
    gs_bfly_mode<HALVE>(v[0], v[1], t0[0].w, t0[0].wp, q, two_q, hq);
    gs_bfly_mode<HALVE>(v[2], v[3], t0[1].w, t0[1].wp, q, two_q, hq);
  }
  const auto t1 = ld_tw(tw + (1u << (logn - sig0 - 2)) + g);
  gs_bfly_mode<HALVE>(v[0], v[2], t1.w, t1.wp, q, two_q, hq);
  gs_bfly_mode<HALVE>(v[1], v[3], t1.w, t1.wp, q, two_q, hq);
}

// One forward pass of the latency pipeline (compile-time pass index P).
// Pass 0 reads the global row when g_src (layout e = 10 is th + 1024 u);
// other passes read their layout from smem.  With two operands (vb != null)
// both are transformed with shared twiddles.
template <int P, bool TWO, typename W>
__device__ __forceinline__ void lat_fwd_pass(W (&va)[4], W (&vb)[4], const W* ga, const W* gb,
                                             W* sa, W* sb,
                                             const typename WordT<W>::Tw* __restrict__ twf,
                                             uint32_t logn, uint32_t t, int th, W q, W two_q,
                                             bool trunc) {
  constexpr int E = 10 - 2 * P;
  const LatGeo G = lat_geo<W>(P, th, t);
  if (P == 0 && ga) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      va[u] = ld_g<false>(ga + th + 1024 * u);
      if constexpr (TWO) vb[u] = ld_g<false>(gb + th + 1024 * u);
    }
  } else {
    lat_ld<W, E>(va, sa, G.pbase);
    if constexpr (TWO) lat_ld<W, E>(vb, sb, G.pbase);
  }
  const uint32_t s0 = logn - 12 + 2 * P;
  if constexpr (TWO)
    ct4_2(va, vb, twf, s0, G.g, q, two_q, trunc && P == 5);
  else
    ct4(va, twf, s0, G.g, q, two_q, trunc && P == 5);
  if constexpr (P < 5) {
    lat_st<W, E>(sa, G.pbase, va);
    if constexpr (TWO) lat_st<W, E>(sb, G.pbase, vb);
    __syncthreads();
  }
}

// Forward in-row stages (six passes); leaves the words of the last layout
// (e = 0: thread th holds words 4 th .. 4 th + 3) in va (and vb).
template <bool TWO, typename W>
__device__ __forceinline__ void lat_fwd(W (&va)[4], W (&vb)[4], const W* ga, const W* gb, W* sa,
                                        W* sb, const typename WordT<W>::Tw* __restrict__ twf,
                                        uint32_t logn, uint32_t t, int th, W q, W two_q,
                                        bool trunc) {
  lat_fwd_pass<0, TWO>(va, vb, ga, gb, sa, sb, twf, logn, t, th, q, two_q, trunc);
  lat_fwd_pass<1, TWO>(va, vb, ga, gb, sa, sb, twf, logn, t, th, q, two_q, trunc);
  lat_fwd_pass<2, TWO>(va, vb, ga, gb, sa, sb, twf, logn, t, th, q, two_q, trunc);
  lat_fwd_pass<3, TWO>(va, vb, ga, gb, sa, sb, twf, logn, t, th, q, two_q, trunc);
  lat_fwd_pass<4, TWO>(va, vb, ga, gb, sa, sb, twf, logn, t, th, q, two_q, trunc);
  lat_fwd_pass<5, TWO>(va, vb, ga, gb, sa, sb, twf, logn, t, th, q, two_q, trunc);
}

// One inverse pass (GS stages 2P', 2P'+1 on the layout of forward pass
// 5 - P').  The first pass works on the registers it is given.
template <int PI, bool HALVE, typename W>
__device__ __forceinline__ void lat_inv_pass(W (&v)[4], W* s,
                                             const typename WordT<W>::Tw* __restrict__ twi,
                                             uint32_t logn, uint32_t t, int th, W q, W two_q,
                                             W hq, bool trunc) {
  constexpr int PF = 5 - PI;
  constexpr int E = 10 - 2 * PF;
  const LatGeo G = lat_geo<W>(PF, th, t);
  if constexpr (PI > 0) lat_ld<W, E>(v, s, G.pbase);
  gs4<HALVE>(v, twi, logn, 2 * PI, G.g, q, two_q, hq, trunc && PI == 0);
  if constexpr (PI < 5) {
    lat_st<W, E>(s, G.pbase, v);
    __syncthreads();
  }
}

// Inverse in-row stages; the result (layout e = 10: words th + 1024 u) goes
// to the global row g_dst, canonical and times N^-1 when `final` (the row is
// the whole transform and 1/N is not applied per stage), else lazy.
template <bool HALVE, typename W>
__device__ __forceinline__ void lat_inv(W (&v)[4], W* g_dst, bool final, W* s,
                                        const typename WordT<W>::Tw* __restrict__ twi,
                                        uint32_t logn, uint32_t t, int th,
                                        const typename WordT<W>::LC& K, bool trunc) {
  const W q = K.q, two_q = K.two_q, hq = K.half_q1;
  lat_inv_pass<0, HALVE>(v, s, twi, logn, t, th, q, two_q, hq, trunc);
  lat_inv_pass<1, HALVE>(v, s, twi, logn, t, th, q, two_q, hq, trunc);
  lat_inv_pass<2, HALVE>(v, s, twi, logn, t, th, q, two_q, hq, trunc);
  lat_inv_pass<3, HALVE>(v, s, twi, logn, t, th, q, two_q, hq, trunc);
  lat_inv_pass<4, HALVE>(v, s, twi, logn, t, th, q, two_q, hq, trunc);
  lat_inv_pass<5, HALVE>(v, s, twi, logn, t, th, q, two_q, hq, trunc);
  if (!HALVE && final) {
#pragma unroll
    for (int u = 0; u < 4; u++) v[u] = mul_shoup_lazy(v[u], K.ninv, K.ninv_p, q);
  }
#pragma unroll
  for (int u = 0; u < 4; u++) __stcs(g_dst + th + 1024 * u, final ? csub(v[u], q) : v[u]);
}

}  // namespace pm
