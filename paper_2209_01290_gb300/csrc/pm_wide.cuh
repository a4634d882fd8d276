// pm_wide.cuh -- the task bodies of the 1024-word split (arxiv 2209.01290,
// Algorithms 6 and 7 on N = R x 1024 words; the decomposition is described
// in pm_wide.cu): the in-row passes, the row task (in-row forward stages of
// a and b, pointwise product, in-row inverse stages), the column-forward and
// column-inverse tasks.  pm_wide.cu runs them as one task per CTA (the
// split launches); pm_wpersist.cu runs them from one persistent launch.
#pragma once
#include <cuda_runtime.h>
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

// Row t's twiddles of one table into shared memory with cp.async (every
// thread copies a few entries).  Forward in-row stage r (global stage
// n-10+r) uses the 2^r entries Psi_br[2^(n-10+r) + t 2^r + i], i < 2^r;
// inverse GS stage 9-r uses Psi^-1_br at the same indices (GS stage sig has
// N/2^(sig+1) blocks, row t's are t 2^(9-sig) ...).  Slice r is a contiguous
// run of the table; it is stored at dst[2^r - 1 + i].
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
      cp_async<(int)sizeof(Tw)>(dst + i, tw + idx);
    }
  }
}

// ------------------------------------------- programmatic dependent launch
// The split's second and third kernels are launched with a programmatic
// dependency on the one before: they may start while it finishes, do what
// does not depend on it (the row kernel stages its twiddles), and wait here
// for its completion and memory before reading its output.  The first two
// kernels let their dependents start once all their CTAs are running.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------ bulk copies (TMA)
// 64-bit words: the same slices copied by the tensor-memory-accelerator's
// 1-D bulk copies, ten per table (slice r is 2^r x 16 bytes, 16-byte aligned
// at both ends), issued by one thread and completed on an mbarrier.  The
// waits are bounded (about a second by %globaltimer, plus a poll-count
// backstop); a CTA that gives up records it in *err and skips its task.
constexpr uint64_t kBulkWaitNs = 1000000000ull;
constexpr uint32_t kBulkWaitPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t w_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One test of the phase; a thread whose phase is not yet complete is
// suspended in the instruction for up to kBulkSuspendNs (it resumes as soon
// as the phase completes), so a waiting warp issues a few instructions
// instead of spinning.
constexpr uint32_t kBulkSuspendNs = 20000;

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "n"(kBulkSuspendNs)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` of the barrier, for at most about a second.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = w_global_ns();
  for (uint32_t it = 0; it < kBulkWaitPolls; ++it) {
    if (mbar_test(bar, parity)) return true;
    // the clock every 8th poll: fewer instructions while the copies land
    if ((it & 7) == 7 && w_global_ns() - t0 > kBulkWaitNs) break;
  }
  return false;
}

// One thread: the barrier (one arrival per phase), made visible to the
// bulk-copy unit.  The caller synchronises the CTA before anyone waits.
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile(
      "mbarrier.init.shared::cta.b64 [%0], 1;\n\t"
      "fence.mbarrier_init.release.cluster;" ::"r"(smem_u32(bar))
      : "memory");
}

// Thread 0 of the CTA: arrive on the barrier expecting the row's slices of
// the tables the MODE needs, and issue their copies.
// `extra` (a test hook, normally 0) is added to the expected byte count.
template <int MODE>
__device__ __forceinline__ void w_stage_tw_bulk(TwPair* tw_f, TwPair* tw_i,
                                                const TwPair* __restrict__ twf,
                                                const TwPair* __restrict__ twi, uint32_t logn,
                                                uint32_t t, uint64_t* bar, uint32_t extra) {
  constexpr uint32_t ntab = (MODE == MODE_FWD || MODE == MODE_INV) ? 1 : 2;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(ntab * (kWTw - 1) * (uint32_t)sizeof(TwPair) + extra)
               : "memory");
#pragma unroll
  for (int r = 0; r < kWLog; r++) {
    const uint32_t idx = (1u << (logn - kWLog + r)) + (t << r);
    const uint32_t bytes = (1u << r) * (uint32_t)sizeof(TwPair);
    if constexpr (MODE != MODE_INV) bulk_g2s(tw_f + (1 << r) - 1, twf + idx, bytes, bar);
    if constexpr (MODE != MODE_FWD) bulk_g2s(tw_i + (1 << r) - 1, twi + idx, bytes, bar);
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
// stage 2P+1 pairs (u, u+1) with slice 2P+1's entries 2 blk + u/2.  Pass 0 takes its words from the caller
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
    const Tw* t1 = tws + (1 << (2 * P + 1)) - 1 + 2 * blk;  // entries 2 blk, 2 blk + 1
    const Tw t1a = t1[0], t1b = t1[1];
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
    const Tw* t0 = tws + (1 << (2 * PF + 1)) - 1 + 2 * blk;  // entries 2 blk, 2 blk + 1
    const Tw t0a = t0[0], t0b = t0[1];
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
  uint32_t logn;
  __device__ __forceinline__ WUnit(const KParams& P, uint32_t unit) {
    if constexpr (DESC) {
      static_assert(sizeof(W) == 8, "grouped launches take 64-bit words");
      const UnitDesc& D = P.desc[unit];
      logn = D.logn;
      a = D.a;
      b = D.b;
      c = D.c;
      s = D.s;
      twf = D.twf;
      twi = D.twi;
      K = ld_limb(D.lc);
    } else {
      const KView<W> V(P);
      logn = P.logn;
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
// The row task of row t of `unit` (256 threads; smem_raw: kWRowsSmem<W>
// bytes).  k_wrows runs one per CTA; the persistent kernels run them as
// tasks.  64-bit words stage the twiddles with bulk copies completed on the
// mbarrier kept in the twiddle area's unused last entry (w_row_bar): the
// caller has initialised it (mbar_init1, then a CTA barrier) and passes the
// phase this task completes.  Returns false when the wait for the copies
// gave up (the task's output is then not written; P.err is set).
template <typename W>
__device__ __forceinline__ uint64_t* w_row_bar(uint64_t* smem_raw) {
  return reinterpret_cast<uint64_t*>(reinterpret_cast<typename WordT<W>::Tw*>(smem_raw) + kWTw -
                                     1);
}

template <int MODE, bool HALVE, typename W, bool DESC, bool LZ>
__device__ __forceinline__ bool w_row_task(const KParams& P, uint32_t unit, uint32_t t,
                                           uint64_t* smem_raw, uint32_t parity) {
  using Tw = typename WordT<W>::Tw;
  Tw* tw_f = reinterpret_cast<Tw*>(smem_raw);
  Tw* tw_i = tw_f + kWTw;
  W* sa = reinterpret_cast<W*>(tw_i + kWTw);
  W* sb = sa + kWRowPad<W>;
  const WUnit<W, DESC> U(P, unit);
  const uint32_t logn = DESC ? U.logn : P.logn;
  const uint32_t cl = logn - kWLog;
  const auto& K = U.K;
  const Tw* twf = U.twf;
  const Tw* twi = U.twi;
  const size_t off = (size_t)t * kW;
  const bool single = (cl == 0);
  const int th = threadIdx.x;
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  uint64_t* bar = w_row_bar<W>(smem_raw);
  if constexpr (sizeof(W) == 8) {
    if (th == 0) w_stage_tw_bulk<MODE>(tw_f, tw_i, twf, twi, logn, t, bar, P.inject_tx);
  } else {
    if constexpr (MODE != MODE_INV) w_stage_tw<W>(tw_f, twf, logn, t, th);
    if constexpr (MODE != MODE_FWD) w_stage_tw<W>(tw_i, twi, logn, t, th);
    cp_async_commit();
  }
  if (P.pdl) pdl_wait();  // the rows are the previous kernel's output
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
  if constexpr (sizeof(W) == 8) {
    const bool done = mbar_wait_bounded(bar, parity);
    if (__syncthreads_or(!done)) {
      // give up: record it, let thread 0 wait (bounded) once more for the
      // copies still in flight, and skip the task
      if (th == 0) {
        if (P.err) atomicOr(P.err, 1);
        mbar_wait_bounded(bar, parity);
      }
      __syncthreads();
      return false;
    }
  } else {
    cp_async_wait_all();
    __syncthreads();
  }
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
  return true;
}

// Column shape for CL column stages (R = 2^CL words per column).
// TH threads work on CT = TH / J columns (a column-task tile), at most MW
// words per thread: a column of R > MW words is shared by J = R / MW
// threads, which needs R <= MW^2 (the stages after the transpose pair words
// of one thread's group).
template <int CL, int TH = kWColThreads, int MW = 16>
struct WCol {
  static constexpr int R = 1 << CL;
  static constexpr int J = R > MW ? R / MW : 1;          // threads per column
  static constexpr int M = R / J;                        // words per thread
  static constexpr int CT = TH / J;                      // columns per tile
  static constexpr int kTiles = kW / CT;                 // tiles per unit and operand
  static constexpr int kSmemWords = J > 1 ? R * CT : 1;  // transpose buffer
  static_assert(J <= M, "column too long for MW words per thread");
};

// Forward column stages LM .. LM + log2 G - 1 (LM = log2 M) on the M/G
// groups of G consecutive column words held in x (group m is block g0 + m at
// stage LM): stage LM + D pairs words G/2^(D+1) apart with twiddle
// Psi_br[2^(LM+D) + (g0 + m) 2^D + b] for block b of the group.
template <int G, int D, bool RED, typename W, int M>
__device__ __forceinline__ void ct_tail(W (&x)[M], const typename WordT<W>::Tw* __restrict__ tw,
                                        uint32_t g0, W q, W two_q) {
  constexpr int LM = M == 16 ? 4 : M == 8 ? 3 : M == 4 ? 2 : M == 2 ? 1 : 0;
  static_assert((1 << LM) == M, "M is a power of two up to 16");
  if constexpr ((1 << D) < G) {
    constexpr int h = G >> (D + 1);
    constexpr int nb = 1 << D;
#pragma unroll
    for (int m = 0; m < M / G; m++)
#pragma unroll
      for (int b = 0; b < nb; b++) {
        const auto w = ld_tw(tw + (1u << (LM + D)) + ((g0 + m) << D) + b);
#pragma unroll
        for (int u0 = 0; u0 < h; u0++)
          ct_bfly_m<RED>(x[G * m + 2 * h * b + u0], x[G * m + 2 * h * b + u0 + h], w.w, w.wp, q,
                         two_q, two_q);
      }
    ct_tail<G, D + 1, RED>(x, tw, g0, q, two_q);
  }
}

// Inverse column stages with word distance 2^D < G (the first log2 G column
// stages of Algorithm 7 after the 10 in-row ones) on the M/G groups of G
// consecutive words held in x (group m = column words G (g0 + m) ...): the
// pair (t, t + 2^D) takes Psi^-1_br[(R >> (D+1)) + (t >> (D+1))] with
// R = M G.
template <int G, int D, bool HALVE, bool LZ, typename W, int M>
__device__ __forceinline__ void gs_tail(W (&x)[M], const typename WordT<W>::Tw* __restrict__ tw,
                                        uint32_t g0, const typename WordT<W>::LC& K) {
  if constexpr ((1 << D) < G) {
    constexpr int h = 1 << D;
    constexpr int nb = G / (2 * h);
#pragma unroll
    for (int m = 0; m < M / G; m++)
#pragma unroll
      for (int b = 0; b < nb; b++) {
        const uint32_t idx = (((uint32_t)M * G) >> (D + 1)) + (g0 + m) * (uint32_t)nb + b;
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
// Column-forward task: columns [tile CT, (tile+1) CT) of operand op of
// `unit`, TH threads; tile_s: R CT words of shared memory (J > 1 only).
template <int CL, typename W, bool DESC, bool LZ, int TH = kWColThreads, int MW = 16>
__device__ __forceinline__ void w_colf_task(const KParams& P, uint32_t unit, uint32_t op,
                                            uint32_t tile, W* tile_s) {
  using S = WCol<CL, TH, MW>;
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
// Column-inverse task: columns [tile CT, (tile+1) CT) of `unit`, TH threads.
template <int CL, bool HALVE, typename W, bool DESC, bool LZ, int TH = kWColThreads,
          int MW = 16>
__device__ __forceinline__ void w_coli_task(const KParams& P, uint32_t unit, uint32_t tile,
                                            W* tile_s) {
  using S = WCol<CL, TH, MW>;
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

}  // namespace
}  // namespace pm
