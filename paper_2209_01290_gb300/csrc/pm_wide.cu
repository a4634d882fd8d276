// pm_wide.cu -- the default split for 64-bit words: one N = 2^n point
// transform viewed as R = N/1024 rows of 1024 words (arxiv 2209.01290,
// Algorithms 6 and 7; the same decomposition as pm_kernels.cu with a shorter
// row).  Measured faster than the 4096-word rows for single products and for
// large batches alike (fewer in-row stages per unit, more warps per SM,
// twiddles from shared memory).
//
// Why a second split.  With 4096-word rows one N = 2^16 product has 16 row
// tasks and keeps 16 SMs busy; each row task (two forward and one inverse
// 4096-point transform) is then compute-bound on its SM for ~20 us.  With
// 1024-word rows the same product has 64 row tasks on 64 SMs, each a quarter
// of the work.  The first n-10 stages of Algorithm 6 mix the R words of a
// column {c + 1024 t} (twiddles Psi_br[1 .. R-1] for every column); the last
// 10 stages act inside row t with twiddle Psi_br[2^s + t 2^(s-n+10) + i'].
// Algorithm 7 mirrors it.  As in the 4096-word split no twiddle
// multiplication appears between the two parts.
//
// Kernels (templates over the word type W)
//   k_wcol_fwd<CL> : the CL = n-10 forward column stages.  For CL <= 4 one
//                    thread holds a whole column.  For CL > 4, J = 2^(CL-4)
//                    threads share a column, 16 words each: the first 4
//                    stages run on words t = j + J k (k < 16; the pairs of
//                    those stages lie 8J, 4J, 2J, J apart), a shared-memory
//                    transpose regroups the column as words t = 16 j + i,
//                    and the last CL-4 stages (pairs J/2 .. 1 apart) run on
//                    its groups of J consecutive words.
//   k_wrows        : the 10 in-row stages as five radix-4 passes over 256
//                    threads (4 words per thread and operand), the product
//                    step (Algorithm 4, or Algorithm 8's pair step), the 10
//                    inverse in-row stages.  The row's twiddles -- in-row
//                    stage r uses 2^r consecutive table entries, 1023 per
//                    table -- are copied to shared memory with cp.async when
//                    the CTA starts, so the passes read them at shared-memory
//                    latency instead of waiting on global memory one pass
//                    after another.
//   k_wcol_inv<CL> : the CL inverse column stages (k_wcol_fwd mirrored), the
//                    1/N fold in the last stage and the reduction to [0, q).
//   k_wclu<CL>     : n = 11..13 (CL = 1..3; and n = 14 in batches of up to
//                    16 units, with clusters of 16 where the device allows
//                    that non-portable size) in one launch, one thread-block
//                    cluster of 2^CL CTAs per unit (CTA rank t = row t).
//                    Each CTA runs the column stages of 1024/2^CL columns
//                    and writes row t' of every column into CTA t''s shared
//                    memory (distributed shared memory); after a cluster
//                    barrier the rows run as in k_wrows and leave their
//                    result in shared memory; after a second barrier each
//                    CTA reads its columns back from all CTAs of the cluster
//                    for the inverse column stages.  No scratch and no second
//                    or third launch: the latency of small products.
// For n = 10 the row is the whole transform: k_wrows alone, canonical output.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <climits>
#include <cstdint>

#include "pm_arith.cuh"
#include "pm_internal.h"
#include "pm_passes.cuh"

namespace pm {
namespace {

constexpr int kWLog = 10;
constexpr int kW = 1 << kWLog;       // words per row
constexpr int kWThreads = kW / 4;    // 256: 4 words per thread and operand
constexpr int kWPasses = kWLog / 2;  // radix-4 passes per transform
constexpr int kWTw = kW;             // staged entries per table (1023 used)
constexpr int kWColThreads = 128;

// Rows in shared memory are padded one word per 16 (64-bit words) or per 32
// (32-bit words), as the 4096-word latency rows (kLatShift).  Threads map
// offset-fastest in passes whose group stride 2^e is at least 2^kWEf, else
// block-fastest: all five layouts are then free of bank conflicts for both
// word sizes (checked exhaustively on the host).
template <typename W>
constexpr int kWRowPad = kW + (kW >> kLatShift<W>);
template <typename W>
constexpr int kWEf = sizeof(W) == 8 ? 4 : 5;

template <typename W>
constexpr int kWRowsSmem = 2 * kWTw * (int)sizeof(typename WordT<W>::Tw) +
                           2 * kWRowPad<W> * (int)sizeof(W);

// ------------------------------------------------------------- cp.async
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Row t's twiddles of one table into shared memory.  Forward in-row stage r
// (global stage n-10+r) uses the 2^r entries Psi_br[2^(n-10+r) + t 2^r + i],
// i < 2^r; inverse GS stage 9-r uses Psi^-1_br at the same indices (GS stage
// sig has N/2^(sig+1) blocks, row t's are t 2^(9-sig) ...).  Slice r starts
// at dst[2^r - 1].  Even slices hold entry i at position i; odd slices, which
// the passes read in pairs (2 blk, 2 blk + 1), hold the even entries first
// and the odd ones after them (entry i at (i & 1) 2^(r-1) + i/2), so that
// threads with consecutive blk read consecutive positions in both halves
// (no bank conflicts in the block-fastest passes).
template <typename W>
__device__ __forceinline__ void w_stage_tw(typename WordT<W>::Tw* dst,
                                           const typename WordT<W>::Tw* __restrict__ tw,
                                           uint32_t logn, uint32_t t, int th) {
  using Tw = typename WordT<W>::Tw;
#pragma unroll
  for (int k = 0; k < kWTw / kWThreads; k++) {
    const int i = th + k * kWThreads;
    if (i < kWTw - 1) {
      const int r = 31 - __clz(i + 1);
      const int e = i + 1 - (1 << r);  // entry within the slice
      const uint32_t idx = (1u << (logn - kWLog + r)) + (t << r) + (uint32_t)e;
      const int pos = (r & 1) ? ((e & 1) << (r - 1)) + (e >> 1) : e;
      cp_async<(int)sizeof(Tw)>(dst + (1 << r) - 1 + pos, tw + idx);
    }
  }
}

// ------------------------------------------------------- row geometry
// Pass p (forward order) covers in-row stages 2p, 2p+1; its groups are the
// 4 words j0 + u 2^e (e = 8 - 2p) of block blk = j0 >> (e+2).
template <typename W, int E>
__device__ __forceinline__ void w_geo(int th, int& pbase, int& blk) {
  constexpr int TB = kWLog - 2;  // log2 threads
  int off;
  if constexpr (E >= kWEf<W>) {
    off = th & ((1 << E) - 1);
    blk = th >> E;
  } else {
    blk = th & ((1 << (TB - E)) - 1);
    off = th >> (TB - E);
  }
  const int j0 = (blk << (E + 2)) + off;
  pbase = j0 + (j0 >> kLatShift<W>);
}

// One forward pass: CT stage 2P pairs (u, u+2) with slice 2P's entry blk,
// stage 2P+1 pairs (u, u+1) with slice 2P+1's entries 2 blk + u/2 (staged at
// positions blk and 2^(2P) + blk).  Pass 0 takes its words from the caller
// (registers); later passes read their layout from shared memory.  With two operands (TWO) both share the
// twiddles.  `trunc` omits the transform's last stage (Algorithm 8).
// Ranges: classic (LZ false) reduces x by 2q at every stage, words in
// [0, 4q); with the wide lazy ranges (LZ) the input may be anything below
// 16q and only in-row stages 0, 4 and 8 (the first stage of passes 0, 2, 4)
// reduce x by m = 8q, so words stay below 16q.
template <int P, bool TWO, bool LZ, typename W>
__device__ __forceinline__ void w_fwd_pass(W (&va)[4], W (&vb)[4], W* sa, W* sb,
                                           const typename WordT<W>::Tw* tws, int th, W q,
                                           W two_q, W m, bool trunc) {
  using Tw = typename WordT<W>::Tw;
  constexpr int E = kWLog - 2 - 2 * P;
  constexpr bool R0 = !LZ || (P % 2 == 0);  // in-row stage 2P
  constexpr bool R1 = !LZ;                  // in-row stage 2P + 1
  int pb, blk;
  w_geo<W, E>(th, pb, blk);
  if constexpr (P > 0) {
    lat_ld<W, E>(va, sa, pb);
    if constexpr (TWO) lat_ld<W, E>(vb, sb, pb);
  }
  const Tw t0 = tws[(1 << (2 * P)) - 1 + blk];
  ct_bfly_m<R0>(va[0], va[2], t0.w, t0.wp, q, two_q, m);
  ct_bfly_m<R0>(va[1], va[3], t0.w, t0.wp, q, two_q, m);
  if constexpr (TWO) {
    ct_bfly_m<R0>(vb[0], vb[2], t0.w, t0.wp, q, two_q, m);
    ct_bfly_m<R0>(vb[1], vb[3], t0.w, t0.wp, q, two_q, m);
  }
  if (!(P == kWPasses - 1 && trunc)) {
    const Tw* t1 = tws + (1 << (2 * P + 1)) - 1 + blk;  // odd slice: evens, then odds
    const Tw t1a = t1[0], t1b = t1[1 << (2 * P)];
    ct_bfly_m<R1>(va[0], va[1], t1a.w, t1a.wp, q, two_q, m);
    ct_bfly_m<R1>(va[2], va[3], t1b.w, t1b.wp, q, two_q, m);
    if constexpr (TWO) {
      ct_bfly_m<R1>(vb[0], vb[1], t1a.w, t1a.wp, q, two_q, m);
      ct_bfly_m<R1>(vb[2], vb[3], t1b.w, t1b.wp, q, two_q, m);
    }
  }
  if constexpr (P < kWPasses - 1) {
    lat_st<W, E>(sa, pb, va);
    if constexpr (TWO) lat_st<W, E>(sb, pb, vb);
    __syncthreads();
  }
}

// Forward in-row stages; leaves the last layout (thread th holds words
// 4 th .. 4 th + 3, bit-reversed order, lazy: below 4q, or 16q with LZ) in
// va (and vb).
template <bool TWO, bool LZ = false, typename W>
__device__ __forceinline__ void w_fwd(W (&va)[4], W (&vb)[4], W* sa, W* sb,
                                      const typename WordT<W>::Tw* tws, int th, W q, W two_q,
                                      bool trunc) {
  const W m = LZ ? W(two_q << 2) : two_q;
  w_fwd_pass<0, TWO, LZ>(va, vb, sa, sb, tws, th, q, two_q, m, trunc);
  w_fwd_pass<1, TWO, LZ>(va, vb, sa, sb, tws, th, q, two_q, m, trunc);
  w_fwd_pass<2, TWO, LZ>(va, vb, sa, sb, tws, th, q, two_q, m, trunc);
  w_fwd_pass<3, TWO, LZ>(va, vb, sa, sb, tws, th, q, two_q, m, trunc);
  w_fwd_pass<4, TWO, LZ>(va, vb, sa, sb, tws, th, q, two_q, m, trunc);
}

// The forward rows' output (below 4q, or 16q with LZ) to [0, q).
template <bool LZ, typename W>
__device__ __forceinline__ W w_reduce_out(W x, W q, W two_q) {
  if constexpr (LZ)
    return reduce16(x, q, two_q, W(two_q << 2));
  else
    return reduce4(x, q, two_q);
}

// One inverse pass PI on the layout of forward pass PF = 4 - PI: GS stage
// 2 PI pairs (u, u+1) with slice 2 PF + 1's entries 2 blk + u/2, GS stage
// 2 PI + 1 pairs (u, u+2) with slice 2 PF's entry blk.  The first pass works
// on the registers it is given; `trunc` omits its first stage (Algorithm 8).
// Ranges: classic words in [0, 2q); with LZ (input below 2q) words stay
// below 8q: in-row GS stages 0..2 leave their sums unreduced, later ones
// reduce them by 8q.
template <int PI, bool HALVE, bool LZ, typename W>
__device__ __forceinline__ void w_inv_pass(W (&v)[4], W* s, const typename WordT<W>::Tw* tws,
                                           int th, W q, W two_q, W hq, W m, bool trunc) {
  using Tw = typename WordT<W>::Tw;
  static_assert(!(LZ && HALVE), "wide lazy ranges fold 1/N at the end");
  constexpr int PF = kWPasses - 1 - PI;
  constexpr int E = kWLog - 2 - 2 * PF;
  constexpr bool R0 = 2 * PI >= 3, R1 = 2 * PI + 1 >= 3;
  int pb, blk;
  w_geo<W, E>(th, pb, blk);
  if constexpr (PI > 0) lat_ld<W, E>(v, s, pb);
  if (!(PI == 0 && trunc)) {
    const Tw* t0 = tws + (1 << (2 * PF + 1)) - 1 + blk;  // odd slice: evens, then odds
    const Tw t0a = t0[0], t0b = t0[1 << (2 * PF)];
    if constexpr (LZ) {
      gs_bfly_m<R0>(v[0], v[1], t0a.w, t0a.wp, q, m);
      gs_bfly_m<R0>(v[2], v[3], t0b.w, t0b.wp, q, m);
    } else {
      gs_bfly_mode<HALVE>(v[0], v[1], t0a.w, t0a.wp, q, two_q, hq);
      gs_bfly_mode<HALVE>(v[2], v[3], t0b.w, t0b.wp, q, two_q, hq);
    }
  }
  const Tw t1 = tws[(1 << (2 * PF)) - 1 + blk];
  if constexpr (LZ) {
    gs_bfly_m<R1>(v[0], v[2], t1.w, t1.wp, q, m);
    gs_bfly_m<R1>(v[1], v[3], t1.w, t1.wp, q, m);
  } else {
    gs_bfly_mode<HALVE>(v[0], v[2], t1.w, t1.wp, q, two_q, hq);
    gs_bfly_mode<HALVE>(v[1], v[3], t1.w, t1.wp, q, two_q, hq);
  }
  if constexpr (PI < kWPasses - 1) {
    lat_st<W, E>(s, pb, v);
    __syncthreads();
  }
}

// Inverse in-row stages; leaves words th + 256 u of the row (lazy: below 2q,
// or 8q with LZ) in v.
template <bool HALVE, bool LZ = false, typename W>
__device__ __forceinline__ void w_inv_passes(W (&v)[4], W* s, const typename WordT<W>::Tw* tws,
                                             int th, const typename WordT<W>::LC& K, bool trunc) {
  const W q = K.q, two_q = K.two_q, hq = K.half_q1;
  const W m = LZ ? W(two_q << 2) : two_q;
  w_inv_pass<0, HALVE, LZ>(v, s, tws, th, q, two_q, hq, m, trunc);
  w_inv_pass<1, HALVE, LZ>(v, s, tws, th, q, two_q, hq, m, trunc);
  w_inv_pass<2, HALVE, LZ>(v, s, tws, th, q, two_q, hq, m, trunc);
  w_inv_pass<3, HALVE, LZ>(v, s, tws, th, q, two_q, hq, m, trunc);
  w_inv_pass<4, HALVE, LZ>(v, s, tws, th, q, two_q, hq, m, trunc);
}

// Inverse in-row stages; the result (words th + 256 u of the row) goes to
// g_dst: canonical, times N^-1 unless every stage halves, when `final` (the
// row is the whole transform), else lazy (below 2q, or 8q with LZ) for
// k_wcol_inv.
template <bool HALVE, bool LZ, typename W>
__device__ __forceinline__ void w_inv(W (&v)[4], W* g_dst, bool final, W* s,
                                      const typename WordT<W>::Tw* tws, int th,
                                      const typename WordT<W>::LC& K, bool trunc) {
  const W q = K.q;
  w_inv_passes<HALVE, LZ>(v, s, tws, th, K, trunc);
  if (!HALVE && final) {
#pragma unroll
    for (int u = 0; u < 4; u++) v[u] = mul_shoup_lazy(v[u], K.ninv, K.ninv_p, q);
  }
#pragma unroll
  for (int u = 0; u < 4; u++) __stcs(g_dst + th + kWThreads * u, final ? csub(v[u], q) : v[u]);
}

// ------------------------------------------------------------- kernels

// One unit's rows, tables and constants: from the batch layout [unit][N]
// and the unit's limb, or, in grouped uneven launches (DESC, 64-bit words),
// from the unit's descriptor.
template <typename W, bool DESC>
struct WUnit {
  const W* a;
  const W* b;
  W* c;
  W* s;
  const typename WordT<W>::Tw* twf;
  const typename WordT<W>::Tw* twi;
  typename WordT<W>::LC K;
  __device__ __forceinline__ WUnit(const KParams& P, uint32_t unit) {
    if constexpr (DESC) {
      static_assert(sizeof(W) == 8, "grouped launches take 64-bit words");
      const UnitDesc& D = P.desc[unit];
      a = D.a;
      b = D.b;
      c = D.c;
      s = D.s;
      twf = D.twf;
      twi = D.twi;
      K = ld_limb(D.lc);
    } else {
      const KView<W> V(P);
      const uint32_t limb = unit % P.nlimbs;
      const size_t base = (size_t)unit << P.logn;
      a = V.a ? V.a + base : nullptr;
      b = V.b ? V.b + base : nullptr;
      c = V.c + base;
      s = V.s ? V.s + base : nullptr;
      twf = V.twf + ((size_t)limb << P.logn);
      twi = V.twi + ((size_t)limb << P.logn);
      K = ld_limb(V.lc + limb);
    }
  }
};

// In-row stages for n >= 10, one CTA per 1024-word row.  Polymul reads the
// column images of a and b from c and s (n > 10) or a and b themselves
// (n = 10); forward NTT rows read c in natural order and write it
// bit-reversed and canonical; inverse NTT rows read c bit-reversed.
// LZ: the wide lazy ranges (64-bit words, q < 2^60, no per-stage halving):
// the column images arrive below 16q, the inverse output leaves below 8q.
template <int MODE, bool HALVE, typename W, bool DESC = false, bool LZ = false>
__global__ void __launch_bounds__(kWThreads, 4) k_wrows(KParams P) {
  using Tw = typename WordT<W>::Tw;
  extern __shared__ __align__(16) uint64_t smem_raw[];
  Tw* tw_f = reinterpret_cast<Tw*>(smem_raw);
  Tw* tw_i = tw_f + kWTw;
  W* sa = reinterpret_cast<W*>(tw_i + kWTw);
  W* sb = sa + kWRowPad<W>;
  const uint32_t logn = P.logn;
  const uint32_t cl = logn - kWLog;
  const uint32_t unit = blockIdx.x >> cl;
  const uint32_t t = blockIdx.x & ((1u << cl) - 1);
  if (unit >= P.nunits) return;  // whole CTA exits together
  const WUnit<W, DESC> U(P, unit);
  const auto& K = U.K;
  const Tw* twf = U.twf;
  const Tw* twi = U.twi;
  const size_t off = (size_t)t * kW;
  const bool single = (cl == 0);
  const int th = threadIdx.x;
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  if constexpr (MODE != MODE_INV) w_stage_tw<W>(tw_f, twf, logn, t, th);
  if constexpr (MODE != MODE_FWD) w_stage_tw<W>(tw_i, twi, logn, t, th);
  cp_async_commit();
  W va[4], vb[4];
  Tw wf{};
  if constexpr (MODE == MODE_INV) {
    // bit-reversed input in the last forward layout: words 4 th .. 4 th + 3
#pragma unroll
    for (int u = 0; u < 4; u++) va[u] = __ldcs(U.c + off + 4 * th + u);
  } else if constexpr (MODE == MODE_FWD) {
#pragma unroll
    for (int u = 0; u < 4; u++) va[u] = __ldcs(U.c + off + th + kWThreads * u);
  } else {
    const W* ga = (single ? U.a : U.c) + off;
    const W* gb = (single ? U.b : U.s) + off;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      va[u] = __ldcs(ga + th + kWThreads * u);
      vb[u] = __ldcs(gb + th + kWThreads * u);
    }
    // Algorithm 8: positions 4 th + u of row t are the pairs i = 2 (256 t +
    // th) (even) and i + 1 (odd); floor(i/2) = 256 t + th
    if constexpr (kFused) wf = ld_tw(twf + (1u << (logn - 2)) + (t << (kWLog - 2)) + th);
  }
  cp_async_wait_all();
  __syncthreads();
  if constexpr (MODE == MODE_INV) {
    w_inv<HALVE, LZ>(va, U.c + off, single, sa, tw_i, th, K, false);
  } else if constexpr (MODE == MODE_FWD) {
    w_fwd<false, LZ>(va, vb, sa, sb, tw_f, th, K.q, K.two_q, false);
#pragma unroll
    for (int u = 0; u < 4; u++)
      __stcs(U.c + off + 4 * th + u, w_reduce_out<LZ>(va[u], K.q, K.two_q));
  } else {
    w_fwd<true, LZ>(va, vb, sa, sb, tw_f, th, K.q, K.two_q, kFused);
    if constexpr (kFused) {
      fused_pair<false, LZ>(va[0], va[1], vb[0], vb[1], wf, K);
      fused_pair<true, LZ>(va[2], va[3], vb[2], vb[3], wf, K);
    } else {
#pragma unroll
      for (int u = 0; u < 4; u++)
        va[u] = mul_barrett_alg4(w_reduce_out<LZ>(va[u], K.q, K.two_q),
                                 w_reduce_out<LZ>(vb[u], K.q, K.two_q), K);
    }
    w_inv<HALVE, LZ>(va, U.c + off, single, sa, tw_i, th, K, kFused);
  }
}

// Column shape for CL column stages (R = 2^CL words per column).
template <int CL>
struct WCol {
  static constexpr int R = 1 << CL;
  static constexpr int J = CL > 4 ? 1 << (CL - 4) : 1;  // threads per column
  static constexpr int M = R / J;                        // words per thread
  static constexpr int CT = kWColThreads / J;            // columns per CTA
  static constexpr int kTiles = kW / CT;                 // CTAs per unit and operand
};

// Forward column stages 4 .. 4 + log2 G - 1 on the 16/G groups of G
// consecutive column words held in x (group m is block g0 + m at stage 4):
// stage 4 + D pairs words G/2^(D+1) apart with twiddle
// Psi_br[2^(4+D) + (g0 + m) 2^D + b] for block b of the group.
template <int G, int D, bool RED, typename W>
__device__ __forceinline__ void ct_tail(W (&x)[16], const typename WordT<W>::Tw* __restrict__ tw,
                                        uint32_t g0, W q, W two_q) {
  if constexpr ((1 << D) < G) {
    constexpr int h = G >> (D + 1);
    constexpr int nb = 1 << D;
#pragma unroll
    for (int m = 0; m < 16 / G; m++)
#pragma unroll
      for (int b = 0; b < nb; b++) {
        const auto w = ld_tw(tw + (1u << (4 + D)) + ((g0 + m) << D) + b);
#pragma unroll
        for (int u0 = 0; u0 < h; u0++)
          ct_bfly_m<RED>(x[G * m + 2 * h * b + u0], x[G * m + 2 * h * b + u0 + h], w.w, w.wp, q,
                         two_q, two_q);
      }
    ct_tail<G, D + 1, RED>(x, tw, g0, q, two_q);
  }
}

// Inverse column stages with word distance 2^D < G (the first log2 G column
// stages of Algorithm 7 after the 10 in-row ones) on the groups of G
// consecutive words held in x (group m = column words G (g0 + m) ...): the
// pair (t, t + 2^D) takes Psi^-1_br[(R >> (D+1)) + (t >> (D+1))] with
// R = 16 G.
template <int G, int D, bool HALVE, bool LZ, typename W>
__device__ __forceinline__ void gs_tail(W (&x)[16], const typename WordT<W>::Tw* __restrict__ tw,
                                        uint32_t g0, const typename WordT<W>::LC& K) {
  if constexpr ((1 << D) < G) {
    constexpr int h = 1 << D;
    constexpr int nb = G / (2 * h);
#pragma unroll
    for (int m = 0; m < 16 / G; m++)
#pragma unroll
      for (int b = 0; b < nb; b++) {
        const uint32_t idx = ((16u * G) >> (D + 1)) + (g0 + m) * (uint32_t)nb + b;
        const auto w = ld_tw(tw + idx);
#pragma unroll
        for (int u0 = 0; u0 < h; u0++) {
          W& lo = x[G * m + 2 * h * b + u0];
          W& hi = x[G * m + 2 * h * b + u0 + h];
          if constexpr (LZ)
            gs_bfly_m<true>(lo, hi, w.w, w.wp, K.q, W(K.two_q << 2));
          else
            gs_bfly_mode<HALVE>(lo, hi, w.w, w.wp, K.q, K.two_q, K.half_q1);
        }
      }
    gs_tail<G, D + 1, HALVE, LZ>(x, tw, g0, K);
  }
}

// Forward column stages: CTA = (unit, operand, tile of CT columns); operand 0
// (a) goes to c, operand 1 (b) to the scratch s.  Every word of a column is
// read (before the barrier) and written (after it) by the CTA that owns the
// column, so c may alias a.
// LZ: wide lazy ranges, no reduction at all (canonical input, CL <= 7
// stages: images below (1 + 2 CL) q <= 15q).
template <int CL, typename W, bool DESC = false, bool LZ = false>
__global__ void __launch_bounds__(kWColThreads) k_wcol_fwd(KParams P, int nops) {
  using S = WCol<CL>;
  const uint32_t tile = blockIdx.x % S::kTiles;
  const uint32_t rest = blockIdx.x / S::kTiles;
  const uint32_t op = rest % (uint32_t)nops, unit = rest / (uint32_t)nops;
  if (unit >= P.nunits) return;
  const WUnit<W, DESC> U(P, unit);
  if (DESC && op == 1 && U.a == U.b) return;  // a square: one image, read twice
  const int th = threadIdx.x;
  const int c = th % S::CT, j = th / S::CT;
  const auto& K = U.K;
  const auto* twf = U.twf;
  const size_t base = tile * S::CT + c;
  const W* src = (op == 0 ? U.a : U.b) + base;
  W* dst = (op == 0 ? U.c : U.s) + base;
  W x[S::M];
#pragma unroll
  for (int k = 0; k < S::M; k++) x[k] = __ldcs(src + (size_t)(j + S::J * k) * kW);
  ct_col<S::M, W, !LZ>(x, twf, K.q, K.two_q);
  if constexpr (S::J > 1) {
    __shared__ W tile_s[S::R * S::CT];
#pragma unroll
    for (int k = 0; k < S::M; k++) tile_s[(j + S::J * k) * S::CT + c] = x[k];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::M; i++) x[i] = tile_s[(S::M * j + i) * S::CT + c];
    ct_tail<S::J, 0, !LZ>(x, twf, (uint32_t)(S::M / S::J * j), K.q, K.two_q);
#pragma unroll
    for (int i = 0; i < S::M; i++) dst[(size_t)(S::M * j + i) * kW] = x[i];
  } else {
#pragma unroll
    for (int k = 0; k < S::M; k++) dst[(size_t)k * kW] = x[k];
  }
}

// Inverse column stages and the reduction, in place on c: the rows' lazy
// output [0, 2q) in, canonical words out.
// LZ: wide lazy ranges (rows' output below 8q; every sum reduced by 8q).
template <int CL, bool HALVE, typename W, bool DESC = false, bool LZ = false>
__global__ void __launch_bounds__(kWColThreads) k_wcol_inv(KParams P) {
  using S = WCol<CL>;
  const uint32_t tile = blockIdx.x % S::kTiles;
  const uint32_t unit = blockIdx.x / S::kTiles;
  if (unit >= P.nunits) return;
  const WUnit<W, DESC> U(P, unit);
  const int th = threadIdx.x;
  const int c = th % S::CT, j = th / S::CT;
  const auto& K = U.K;
  const auto* twi = U.twi;
  W* p = U.c + tile * S::CT + c;
  W x[S::M];
  if constexpr (S::J > 1) {
#pragma unroll
    for (int i = 0; i < S::M; i++) x[i] = p[(size_t)(S::M * j + i) * kW];
    gs_tail<S::J, 0, HALVE, LZ>(x, twi, (uint32_t)(S::M / S::J * j), K);
    __shared__ W tile_s[S::R * S::CT];
#pragma unroll
    for (int i = 0; i < S::M; i++) tile_s[(S::M * j + i) * S::CT + c] = x[i];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::M; k++) x[k] = tile_s[(j + S::J * k) * S::CT + c];
  } else {
#pragma unroll
    for (int k = 0; k < S::M; k++) x[k] = p[(size_t)k * kW];
  }
  // the last four (or all CL) stages: words t = j + J k, the pair distance
  // J 2^E' in t is 2^E' in k and the twiddle index reduces to gs_col's
  gs_col<S::M, HALVE, W, LZ>(x, twi, K);
#pragma unroll
  for (int k = 0; k < S::M; k++) __stcs(p + (size_t)(j + S::J * k) * kW, csub(x[k], K.q));
}

// N = 2^(10+CL), CL = 1..3: one cluster of R = 2^CL CTAs per unit, CTA rank
// t holding row t in shared memory.  Column steps: CTA t owns columns
// [t C, (t+1) C), C = 1024 / R.
template <int MODE, bool HALVE, typename W, int CL>
__global__ void __launch_bounds__(kWThreads, 4) k_wclu(KParams P) {
  namespace cg = cooperative_groups;
  using Tw = typename WordT<W>::Tw;
  constexpr int RR = 1 << CL;
  constexpr int C = kW / RR;
  extern __shared__ __align__(16) uint64_t smem_raw[];
  Tw* tw_f = reinterpret_cast<Tw*>(smem_raw);
  Tw* tw_i = tw_f + kWTw;
  W* sa = reinterpret_cast<W*>(tw_i + kWTw);
  W* sb = sa + kWRowPad<W>;
  cg::cluster_group cluster = cg::this_cluster();
  const KView<W> V(P);
  constexpr uint32_t logn = kWLog + CL;
  const uint32_t t = cluster.block_rank();
  const uint32_t unit = blockIdx.x >> CL;  // the grid is exactly nunits clusters
  const uint32_t limb = unit % P.nlimbs;
  const auto K = ld_limb(V.lc + limb);
  const Tw* twf = V.twf + ((size_t)limb << logn);
  const Tw* twi = V.twi + ((size_t)limb << logn);
  const size_t base = (size_t)unit << logn;
  const int th = threadIdx.x;
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  if constexpr (MODE != MODE_INV) w_stage_tw<W>(tw_f, twf, logn, t, th);
  if constexpr (MODE != MODE_FWD) w_stage_tw<W>(tw_i, twi, logn, t, th);
  cp_async_commit();
  Tw wf{};
  if constexpr (kFused) wf = ld_tw(twf + (1u << (logn - 2)) + (t << (kWLog - 2)) + th);
  W va[4], vb[4];
  if constexpr (MODE != MODE_INV) {
    // forward column stages; word j of row r goes to CTA r's row buffer at
    // the padded index j + (j >> kLatShift), the layout of the first pass
    constexpr int nops = (MODE == MODE_FWD) ? 1 : 2;
    for (int it = th; it < nops * C; it += kWThreads) {
      const int op = it / C;
      const int c = (int)t * C + (it % C);
      const W* src = ((MODE == MODE_FWD) ? V.c : (op == 0 ? V.a : V.b)) + base + c;
      W x[RR];
#pragma unroll
      for (int r = 0; r < RR; r++) x[r] = __ldcs(src + (size_t)r * kW);
      ct_col<RR>(x, twf, K.q, K.two_q);
      W* row = op == 0 ? sa : sb;
      const int pj = c + (c >> kLatShift<W>);
#pragma unroll
      for (int r = 0; r < RR; r++) cluster.map_shared_rank(row, r)[pj] = x[r];
    }
    cp_async_wait_all();
    cluster.sync();  // every column image (and this CTA's twiddles) in place
    int pb, blk;
    w_geo<W, kWLog - 2>(th, pb, blk);
    lat_ld<W, kWLog - 2>(va, sa, pb);
    if constexpr (MODE != MODE_FWD) lat_ld<W, kWLog - 2>(vb, sb, pb);
  } else {
    // bit-reversed input in the last forward layout: words 4 th .. 4 th + 3
#pragma unroll
    for (int u = 0; u < 4; u++) va[u] = __ldcs(V.c + base + (size_t)t * kW + 4 * th + u);
    cp_async_wait_all();
    __syncthreads();
  }
  if constexpr (MODE == MODE_FWD) {
    w_fwd<false>(va, vb, sa, sb, tw_f, th, K.q, K.two_q, false);
#pragma unroll
    for (int u = 0; u < 4; u++)
      __stcs(V.c + base + (size_t)t * kW + 4 * th + u, reduce4(va[u], K.q, K.two_q));
    return;  // no shared memory of another CTA is touched after the barrier
  } else {
    if constexpr (MODE != MODE_INV) {
      w_fwd<true>(va, vb, sa, sb, tw_f, th, K.q, K.two_q, kFused);
      if constexpr (kFused) {
        fused_pair<false>(va[0], va[1], vb[0], vb[1], wf, K);
        fused_pair<true>(va[2], va[3], vb[2], vb[3], wf, K);
      } else {
#pragma unroll
        for (int u = 0; u < 4; u++)
          va[u] =
              mul_barrett_alg4(reduce4(va[u], K.q, K.two_q), reduce4(vb[u], K.q, K.two_q), K);
      }
    }
    w_inv_passes<HALVE>(va, sa, tw_i, th, K, kFused);
    // the row's lazy result back into its buffer (each thread rewrites the
    // words it read in the last pass), then the inverse column stages
    int pb, blk;
    w_geo<W, kWLog - 2>(th, pb, blk);
    lat_st<W, kWLog - 2>(sa, pb, va);
    cluster.sync();
    for (int it = th; it < C; it += kWThreads) {
      const int c = (int)t * C + it;
      const int pj = c + (c >> kLatShift<W>);
      W x[RR];
#pragma unroll
      for (int r = 0; r < RR; r++) x[r] = cluster.map_shared_rank(sa, r)[pj];
      gs_col<RR, HALVE>(x, twi, K);
#pragma unroll
      for (int r = 0; r < RR; r++) __stcs(V.c + base + (size_t)r * kW + c, csub(x[r], K.q));
    }
    cluster.sync();  // keep this CTA's rows alive until every CTA has read them
  }
}

// ------------------------------------------------------------ launchers

// The wide lazy ranges apply to 64-bit words with every q < 2^60 and the
// 1/N fold (the host sets P.lazy16 only then).
template <typename W>
inline bool use_lazy16(const KParams& P) {
  return sizeof(W) == 8 && P.lazy16 && !P.halving;
}

template <int MODE, typename W>
cudaError_t wrows(const KParams& P, cudaStream_t st) {
  const size_t blocks = (size_t)P.nunits << (P.logn - kWLog);
  if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
  if (use_lazy16<W>(P))
    k_wrows<MODE, false, W, false, true><<<(unsigned)blocks, kWThreads, kWRowsSmem<W>, st>>>(P);
  else if (P.halving)
    k_wrows<MODE, true, W><<<(unsigned)blocks, kWThreads, kWRowsSmem<W>, st>>>(P);
  else
    k_wrows<MODE, false, W><<<(unsigned)blocks, kWThreads, kWRowsSmem<W>, st>>>(P);
  return cudaGetLastError();
}

template <int CL, typename W>
cudaError_t wcol_fwd_cl(const KParams& P, int nops, cudaStream_t st) {
  const size_t blocks = (size_t)P.nunits * nops * WCol<CL>::kTiles;
  if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
  if (use_lazy16<W>(P))
    k_wcol_fwd<CL, W, false, true><<<(unsigned)blocks, kWColThreads, 0, st>>>(P, nops);
  else
    k_wcol_fwd<CL, W><<<(unsigned)blocks, kWColThreads, 0, st>>>(P, nops);
  return cudaGetLastError();
}

template <int CL, typename W>
cudaError_t wcol_inv_cl(const KParams& P, cudaStream_t st) {
  const size_t blocks = (size_t)P.nunits * WCol<CL>::kTiles;
  if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
  if (use_lazy16<W>(P))
    k_wcol_inv<CL, false, W, false, true><<<(unsigned)blocks, kWColThreads, 0, st>>>(P);
  else if (P.halving)
    k_wcol_inv<CL, true, W><<<(unsigned)blocks, kWColThreads, 0, st>>>(P);
  else
    k_wcol_inv<CL, false, W><<<(unsigned)blocks, kWColThreads, 0, st>>>(P);
  return cudaGetLastError();
}

template <typename W>
cudaError_t wcol_fwd(const KParams& P, int nops, cudaStream_t st) {
  switch (P.logn - kWLog) {
    case 1: return wcol_fwd_cl<1, W>(P, nops, st);
    case 2: return wcol_fwd_cl<2, W>(P, nops, st);
    case 3: return wcol_fwd_cl<3, W>(P, nops, st);
    case 4: return wcol_fwd_cl<4, W>(P, nops, st);
    case 5: return wcol_fwd_cl<5, W>(P, nops, st);
    case 6: return wcol_fwd_cl<6, W>(P, nops, st);
    case 7: return wcol_fwd_cl<7, W>(P, nops, st);
  }
  return cudaErrorInvalidValue;
}

template <typename W>
cudaError_t wcol_inv(const KParams& P, cudaStream_t st) {
  switch (P.logn - kWLog) {
    case 1: return wcol_inv_cl<1, W>(P, st);
    case 2: return wcol_inv_cl<2, W>(P, st);
    case 3: return wcol_inv_cl<3, W>(P, st);
    case 4: return wcol_inv_cl<4, W>(P, st);
    case 5: return wcol_inv_cl<5, W>(P, st);
    case 6: return wcol_inv_cl<6, W>(P, st);
    case 7: return wcol_inv_cl<7, W>(P, st);
  }
  return cudaErrorInvalidValue;
}

template <int MODE, bool H, typename W, int CL>
cudaError_t clu_cl(const KParams& P, cudaStream_t st) {
  const size_t blocks = (size_t)P.nunits << CL;
  if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(kWThreads, 1, 1);
  cfg.dynamicSmemBytes = kWRowsSmem<W>;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_wclu<MODE, H, W, CL>, P);
}

template <int MODE, typename W>
cudaError_t clu(const KParams& P, cudaStream_t st) {
  switch (P.logn - kWLog) {
    case 1: return P.halving ? clu_cl<MODE, true, W, 1>(P, st) : clu_cl<MODE, false, W, 1>(P, st);
    case 2: return P.halving ? clu_cl<MODE, true, W, 2>(P, st) : clu_cl<MODE, false, W, 2>(P, st);
    case 3: return P.halving ? clu_cl<MODE, true, W, 3>(P, st) : clu_cl<MODE, false, W, 3>(P, st);
    case 4: return P.halving ? clu_cl<MODE, true, W, 4>(P, st) : clu_cl<MODE, false, W, 4>(P, st);
  }
  return cudaErrorInvalidValue;
}

// N = 2^14 as one launch needs clusters of 16 CTAs (above the portable 8):
// used when the device schedules them (checked when the kernels are
// prepared) and for batches of at most kClu14MaxUnits units.
bool g_clu16 = false;
constexpr uint32_t kClu14MaxUnits = 16;  // measured: faster up to 16 units, slower from 64

// Units of N = 2^11 .. 2^13 (and small batches of 2^14) run as one cluster
// launch.
inline bool clustered(uint32_t logn, uint32_t nunits) {
  return (logn > kWLog && logn <= kWLog + 3) ||
         (logn == kWLog + 4 && g_clu16 && nunits <= kClu14MaxUnits);
}

inline cudaError_t mark(const PhaseEvents* pe, int k, cudaStream_t st) {
  return (pe && k < pe->n) ? cudaEventRecord(pe->ev[k], st) : cudaSuccess;
}

template <typename W>
cudaError_t polymul_wide_w(const KParams& P0, cudaStream_t st, const PhaseEvents* pe) {
  KParams P = P0;
  if (P.nunits == 0) return cudaSuccess;
  // Algorithm 8 plans: the fused constants (2/N) follow the plain ones
  if (P.fused)
    P.lc = reinterpret_cast<const LimbConst*>(
        reinterpret_cast<const typename WordT<W>::LC*>(P.lc) + P.nlimbs);
  auto prows = [&](const KParams& Q) {
    return Q.fused ? wrows<MODE_POLYMUL_FUSED, W>(Q, st) : wrows<MODE_POLYMUL, W>(Q, st);
  };
  cudaError_t e = mark(pe, 0, st);
  if (e != cudaSuccess) return e;
  if (P.logn == kWLog || clustered(P.logn, P.nunits)) {
    if (P.logn == kWLog)
      e = prows(P);
    else
      e = P.fused ? clu<MODE_POLYMUL_FUSED, W>(P, st) : clu<MODE_POLYMUL, W>(P, st);
    if (e != cudaSuccess) return e;
    return mark(pe, 1, st);
  }
  // operand images: a's to c, b's to the scratch s (as in the 4096-word
  // split: one transform for a square, b's image in place when c == b)
  int nops = 2;
  if (P.a == P.b) {
    P.b = nullptr;
    P.s = P.c;
    nops = 1;
  } else if (P.c == P.b) {
    const uint64_t* t = P.a;
    P.a = P.b;
    P.b = t;
  }
  e = wcol_fwd<W>(P, nops, st);
  if (e == cudaSuccess) e = mark(pe, 1, st);
  if (e == cudaSuccess) e = prows(P);
  if (e == cudaSuccess) e = mark(pe, 2, st);
  if (e == cudaSuccess) e = wcol_inv<W>(P, st);
  if (e == cudaSuccess) e = mark(pe, 3, st);
  return e;
}

template <typename W>
cudaError_t ntt_fwd_wide_w(const KParams& P0, cudaStream_t st) {
  if (P0.nunits == 0) return cudaSuccess;
  if (clustered(P0.logn, P0.nunits)) return clu<MODE_FWD, W>(P0, st);
  KParams P = P0;
  if (P.logn > kWLog) {
    P.a = P.c;  // in place: the column stages read and write x
    cudaError_t e = wcol_fwd<W>(P, 1, st);
    if (e != cudaSuccess) return e;
  }
  return wrows<MODE_FWD, W>(P, st);
}

template <typename W>
cudaError_t ntt_inv_wide_w(const KParams& P, cudaStream_t st) {
  if (P.nunits == 0) return cudaSuccess;
  if (clustered(P.logn, P.nunits)) return clu<MODE_INV, W>(P, st);
  cudaError_t e = wrows<MODE_INV, W>(P, st);
  if (e != cudaSuccess || P.logn == kWLog) return e;
  return wcol_inv<W>(P, st);
}

template <bool H, typename W, int CL>
cudaError_t prepare_clu() {
  const void* fns[] = {(const void*)k_wclu<MODE_POLYMUL, H, W, CL>,
                       (const void*)k_wclu<MODE_POLYMUL_FUSED, H, W, CL>,
                       (const void*)k_wclu<MODE_FWD, H, W, CL>,
                       (const void*)k_wclu<MODE_INV, H, W, CL>};
  for (const void* f : fns) {
    cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kWRowsSmem<W>);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Grouped uneven launch (64-bit words): the units of one N >= 2^13 through
// the three wide-split kernels, each unit's rows, scratch, tables and
// constants (the fused ones for an Algorithm 8 plan) from P.desc.
template <int CL, bool H, bool F, bool LZ>
cudaError_t wide_desc_cl(const KParams& P, cudaStream_t st) {
  using W = uint64_t;
  constexpr int MODE = F ? MODE_POLYMUL_FUSED : MODE_POLYMUL;
  const size_t cols = (size_t)P.nunits * 2 * WCol<CL>::kTiles;
  const size_t rows = (size_t)P.nunits << CL;
  const size_t inv = (size_t)P.nunits * WCol<CL>::kTiles;
  if (cols > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
  k_wcol_fwd<CL, W, true, LZ><<<(unsigned)cols, kWColThreads, 0, st>>>(P, 2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_wrows<MODE, H, W, true, LZ><<<(unsigned)rows, kWThreads, kWRowsSmem<W>, st>>>(P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_wcol_inv<CL, H, W, true, LZ><<<(unsigned)inv, kWColThreads, 0, st>>>(P);
  return cudaGetLastError();
}

template <int CL>
cudaError_t wide_desc(const KParams& P, cudaStream_t st) {
  if (P.halving)
    return P.fused ? wide_desc_cl<CL, true, true, false>(P, st)
                   : wide_desc_cl<CL, true, false, false>(P, st);
  if (P.lazy16)
    return P.fused ? wide_desc_cl<CL, false, true, true>(P, st)
                   : wide_desc_cl<CL, false, false, true>(P, st);
  return P.fused ? wide_desc_cl<CL, false, true, false>(P, st)
                 : wide_desc_cl<CL, false, false, false>(P, st);
}

// Clusters of 16 CTAs for N = 2^14: allowed (non-portable size) and
// schedulable on this device?  A refusal only leaves g_clu16 false.
template <bool H, typename W>
bool prepare_clu16() {
  const void* fns[] = {(const void*)k_wclu<MODE_POLYMUL, H, W, 4>,
                       (const void*)k_wclu<MODE_POLYMUL_FUSED, H, W, 4>,
                       (const void*)k_wclu<MODE_FWD, H, W, 4>,
                       (const void*)k_wclu<MODE_INV, H, W, 4>};
  for (const void* f : fns) {
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kWRowsSmem<W>) !=
            cudaSuccess ||
        cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(kWThreads, 1, 1);
    cfg.dynamicSmemBytes = kWRowsSmem<W>;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return false;
    }
  }
  return true;
}

template <bool H, typename W>
cudaError_t wide_prepare_w(bool& clu16) {
  cudaError_t e;
  if ((e = prepare_clu<H, W, 1>()) != cudaSuccess || (e = prepare_clu<H, W, 2>()) != cudaSuccess ||
      (e = prepare_clu<H, W, 3>()) != cudaSuccess)
    return e;
  clu16 = clu16 && prepare_clu16<H, W>();
  const void* fns[] = {(const void*)k_wrows<MODE_POLYMUL, H, W>,
                       (const void*)k_wrows<MODE_POLYMUL_FUSED, H, W>,
                       (const void*)k_wrows<MODE_FWD, H, W>, (const void*)k_wrows<MODE_INV, H, W>};
  for (const void* f : fns) {
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kWRowsSmem<W>)) != cudaSuccess)
      return e;
  }
  if constexpr (sizeof(W) == 8) {  // the grouped (descriptor) rows exist for 64-bit words only
    const void* desc_fns[] = {(const void*)k_wrows<MODE_POLYMUL, H, W, true>,
                              (const void*)k_wrows<MODE_POLYMUL_FUSED, H, W, true>};
    for (const void* f : desc_fns) {
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kWRowsSmem<W>)) != cudaSuccess)
        return e;
    }
    if constexpr (!H) {  // the wide lazy ranges: 64-bit words, 1/N folded
      const void* lz_fns[] = {(const void*)k_wrows<MODE_POLYMUL, H, W, false, true>,
                              (const void*)k_wrows<MODE_POLYMUL_FUSED, H, W, false, true>,
                              (const void*)k_wrows<MODE_FWD, H, W, false, true>,
                              (const void*)k_wrows<MODE_INV, H, W, false, true>,
                              (const void*)k_wrows<MODE_POLYMUL, H, W, true, true>,
                              (const void*)k_wrows<MODE_POLYMUL_FUSED, H, W, true, true>};
      for (const void* f : lz_fns) {
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kWRowsSmem<W>)) != cudaSuccess)
          return e;
      }
    }
  }
  return cudaSuccess;
}

}  // namespace

bool wide_polymul_ok(uint32_t logn) { return logn >= kWLog && logn <= 17; }

bool wide_single_launch(uint32_t logn, uint32_t nunits) {
  return logn == kWLog || clustered(logn, nunits);
}

bool wide_ntt_ok(uint32_t logn) { return logn >= kWLog && logn <= 17; }

cudaError_t wide_prepare() {
  cudaError_t e;
  bool clu16 = true;
  if ((e = wide_prepare_w<false, uint64_t>(clu16)) != cudaSuccess ||
      (e = wide_prepare_w<true, uint64_t>(clu16)) != cudaSuccess ||
      (e = wide_prepare_w<false, uint32_t>(clu16)) != cudaSuccess ||
      (e = wide_prepare_w<true, uint32_t>(clu16)) != cudaSuccess)
    return e;
  g_clu16 = clu16;
  return cudaSuccess;
}

cudaError_t launch_polymul_wide(const KParams& P, cudaStream_t st, const PhaseEvents* pe) {
  return P.word32 ? polymul_wide_w<uint32_t>(P, st, pe) : polymul_wide_w<uint64_t>(P, st, pe);
}

cudaError_t launch_ntt_fwd_wide(const KParams& P, cudaStream_t st) {
  return P.word32 ? ntt_fwd_wide_w<uint32_t>(P, st) : ntt_fwd_wide_w<uint64_t>(P, st);
}

cudaError_t launch_polymul_wide_grouped(const KParams& P, cudaStream_t st) {
  if (P.nunits == 0) return cudaSuccess;
  if (P.word32 || !P.desc) return cudaErrorInvalidValue;
  switch (P.logn) {
    case 13: return wide_desc<3>(P, st);
    case 14: return wide_desc<4>(P, st);
    case 15: return wide_desc<5>(P, st);
    case 16: return wide_desc<6>(P, st);
    case 17: return wide_desc<7>(P, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ntt_inv_wide(const KParams& P, cudaStream_t st) {
  return P.word32 ? ntt_inv_wide_w<uint32_t>(P, st) : ntt_inv_wide_w<uint64_t>(P, st);
}

}  // namespace pm
