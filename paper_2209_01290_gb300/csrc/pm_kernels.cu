// pm_kernels.cu -- sm_103a kernels for exact negacyclic polynomial
// multiplication (arxiv 2209.01290, Eq. 2):
//   c = NTT^{GS,psi^-1}_{bo->no,1/2}( NTT^{CT,psi}_{no->bo}(a) . NTT^{CT,psi}_{no->bo}(b) ).
//
// Decomposition of one N = 2^n point merged transform (n >= 12)
// ----------------------------------------------------------------
// View the N words as R = N/4096 rows of 4096.  In Algorithm 6 (forward, k
// halving from N/2) the first n-12 stages have strides k >= 4096: they mix
// only the R words of one column {c + 4096 t}, and all columns use the same
// twiddles Psi_br[1 .. R-1].  The remaining 12 stages have k < 4096 and act
// inside one row t; their twiddle for row t, stage s and block i' is
// Psi_br[2^s + t 2^(s-n+12) + i'] (Algorithm 6's Psi_br[m + i] with the
// block index i split into row and in-row parts).  Algorithm 7 (inverse, k
// doubling from 1) is the mirror image: 12 in-row stages first, then n-12
// column stages.  No extra twiddle multiplication appears at the split
// (unlike a classical four-step FFT), because the merged transforms keep the
// psi-powers inside the butterflies.
//
// Kernels (each a template over the word type W, 64-bit or 32-bit)
//   k_col_fwd<R>    : the n-12 forward column stages, streaming (registers
//                     only, coalesced loads/stores), one thread per column.
//   k_rows2         : polymul rows: the 12 in-row stages of a and b together
//                     (each thread holds 16 words of each operand), the
//                     product step (Algorithm 4, or Algorithm 8's pair step)
//                     and the 12 inverse in-row stages; rows are exchanged
//                     through padded shared memory between the radix-16
//                     passes.  The 4096-word row kernel for
//                     N = 2^12 batches and large 32-bit batches (row_ops 2);
//                     the 1024-word rows of pm_wide.cu serve the rest.
//   k_rows<MODE>    : the same passes one operand at a time (forward or
//                     inverse NTT rows, and polymul with row_ops 1).
//   k_col_inv<R>    : the n-12 inverse column stages and the final reduction.
//   k_fused13       : N = 2^13 in one CTA (column stage through smem).
//   k_small         : N <= 2^11, one CTA per unit, radix-2 stages in smem.
//   k_pointwise     : stand-alone Hadamard product with Algorithm 4.
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "pm_arith.cuh"
#include "pm_internal.h"
#include "pm_passes.cuh"

namespace pm {

// ------------------------------------------------------------------ kernels

// 16 consecutive words of a row (16-byte aligned) in or out with 16-byte
// accesses; the store reduces [0, 4q) -> [0, q).
template <typename W>
__device__ __forceinline__ void ld_row16(W (&v)[16], const W* p) {
  if constexpr (sizeof(W) == 8) {
    const ulonglong2* s = reinterpret_cast<const ulonglong2*>(p);
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const ulonglong2 w = __ldcs(s + k);
      v[2 * k] = w.x;
      v[2 * k + 1] = w.y;
    }
  } else {
    const uint4* s = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint4 w = __ldcs(s + k);
      v[4 * k] = w.x;
      v[4 * k + 1] = w.y;
      v[4 * k + 2] = w.z;
      v[4 * k + 3] = w.w;
    }
  }
}

template <typename W>
__device__ __forceinline__ void st_row16_reduced(W* p, const W (&v)[16], W q, W two_q) {
  if constexpr (sizeof(W) == 8) {
    ulonglong2* d = reinterpret_cast<ulonglong2*>(p);
#pragma unroll
    for (int k = 0; k < 8; k++)
      __stcs(d + k, make_ulonglong2(reduce4(v[2 * k], q, two_q), reduce4(v[2 * k + 1], q, two_q)));
  } else {
    uint4* d = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int k = 0; k < 4; k++)
      __stcs(d + k, make_uint4(reduce4(v[4 * k], q, two_q), reduce4(v[4 * k + 1], q, two_q),
                               reduce4(v[4 * k + 2], q, two_q), reduce4(v[4 * k + 3], q, two_q)));
  }
}

// In-row stages for n >= 12.  One CTA = one row (256 threads).  For n == 12
// the row is the whole unit (polymul reads a, b; output canonical).  For
// n > 12, polymul reads the column-transformed operands from c and the
// scratch s and leaves lazy c' rows for k_col_inv.
template <int MODE, bool HALVE, typename W>
__global__ void __launch_bounds__(256, sizeof(W) == 8 ? 3 : 4) k_rows(KParams P) {
  extern __shared__ __align__(16) uint64_t smem_raw[];
  W* smem = reinterpret_cast<W*>(smem_raw);
  const KView<W> V(P);
  const uint32_t logn = P.logn;
  const uint32_t unit = blockIdx.x >> (logn - kRowLog);
  const uint32_t t = blockIdx.x & ((1u << (logn - kRowLog)) - 1);
  if (unit >= P.nunits) return;  // whole CTA exits together
  const uint32_t limb = unit % P.nlimbs;
  const auto K = ld_limb(V.lc + limb);
  const auto* twf = V.twf + ((size_t)limb << logn);
  const auto* twi = V.twi + ((size_t)limb << logn);
  const size_t off = ((size_t)unit << logn) + (size_t)t * kRow;
  const bool single = (logn == kRowLog);
  const int th = threadIdx.x;
  W* sa = smem;
  W* sb = smem + kRowPadW<W>;
  W v[16];
  if constexpr (MODE == MODE_INV) {
    ld_row16(v, V.c + off + 16 * th);
    rows_inv<HALVE>(v, V.c + off, single, sa, twi, logn, t, th, K);
  } else if constexpr (MODE == MODE_FWD) {
    rows_fwd(v, V.c + off, sa, twf, logn, t, th, K.q, K.two_q);
    st_row16_reduced(V.c + off + 16 * th, v, K.q, K.two_q);
  } else {
    (void)sb;
    row_task_polymul<HALVE, false>((single ? V.a : V.c) + off, (single ? V.b : V.s) + off,
                                   V.c + off, single, smem, twf, twi, K, logn, t,
                                   MODE == MODE_POLYMUL_FUSED);
  }
}

// Polymul rows with a and b transformed together in registers (shared
// twiddle loads, half the barriers per word; 2 CTAs per SM).
template <bool HALVE, bool FUSED, typename W, bool DESC = false>
__global__ void __launch_bounds__(256, sizeof(W) == 8 ? 2 : 3) k_rows2(KParams P) {
  extern __shared__ __align__(16) uint64_t smem_raw[];
  W* smem = reinterpret_cast<W*>(smem_raw);
  const KView<W> V(P);
  const uint32_t logn = P.logn;
  const uint32_t unit = blockIdx.x >> (logn - kRowLog);
  const uint32_t t = blockIdx.x & ((1u << (logn - kRowLog)) - 1);
  if (unit >= P.nunits) return;
  if constexpr (DESC) {  // grouped uneven launch: the unit's own pointers
    static_assert(sizeof(W) == 8, "grouped launches take 64-bit words");
    const UnitDesc& D = P.desc[unit];
    const auto K = ld_limb(D.lc);
    const size_t off = (size_t)t * kRow;
    const bool single = (logn == kRowLog);
    row_task_polymul2<HALVE, false>((single ? D.a : D.c) + off, (single ? D.b : D.s) + off,
                                    D.c + off, single, smem, D.twf, D.twi, K, logn, t, FUSED);
    return;
  }
  const uint32_t limb = unit % P.nlimbs;
  const auto K = ld_limb(V.lc + limb);
  const auto* twf = V.twf + ((size_t)limb << logn);
  const auto* twi = V.twi + ((size_t)limb << logn);
  const size_t off = ((size_t)unit << logn) + (size_t)t * kRow;
  const bool single = (logn == kRowLog);
  row_task_polymul2<HALVE, false>((single ? V.a : V.c) + off, (single ? V.b : V.s) + off,
                                  V.c + off, single, smem, twf, twi, K, logn, t, FUSED);
}

// Rows for small batches: the same row task as k_rows2 (or k_rows for the
// forward and inverse NTT) over 1024 threads per row in six radix-4 passes,
// one CTA per SM; see the latency pipeline in pm_passes.cuh.
template <int MODE, bool HALVE, typename W>
__global__ void __launch_bounds__(kLatThreads, 1) k_rows_lat(KParams P) {
  extern __shared__ __align__(16) uint64_t smem_raw[];
  W* sa = reinterpret_cast<W*>(smem_raw);
  W* sb = sa + kLatRowPad<W>;
  const KView<W> V(P);
  const uint32_t logn = P.logn;
  const uint32_t unit = blockIdx.x >> (logn - kRowLog);
  const uint32_t t = blockIdx.x & ((1u << (logn - kRowLog)) - 1);
  if (unit >= P.nunits) return;
  const uint32_t limb = unit % P.nlimbs;
  const auto K = ld_limb(V.lc + limb);
  const auto* twf = V.twf + ((size_t)limb << logn);
  const auto* twi = V.twi + ((size_t)limb << logn);
  const size_t off = ((size_t)unit << logn) + (size_t)t * kRow;
  const bool single = (logn == kRowLog);
  const int th = threadIdx.x;
  W va[4], vb[4];
  if constexpr (MODE == MODE_INV) {
    // bit-reversed input in the last forward layout: words 4 th .. 4 th + 3
#pragma unroll
    for (int u = 0; u < 4; u++) va[u] = __ldcs(V.c + off + 4 * th + u);
    lat_inv<HALVE>(va, V.c + off, single, sa, twi, logn, t, th, K, false);
  } else if constexpr (MODE == MODE_FWD) {
    lat_fwd<false>(va, vb, V.c + off, (const W*)nullptr, sa, sb, twf, logn, t, th, K.q, K.two_q,
                   false);
#pragma unroll
    for (int u = 0; u < 4; u++) __stcs(V.c + off + 4 * th + u, reduce4(va[u], K.q, K.two_q));
  } else {
    constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
    lat_fwd<true>(va, vb, (single ? V.a : V.c) + off, (single ? V.b : V.s) + off, sa, sb, twf,
                  logn, t, th, K.q, K.two_q, kFused);
    if constexpr (kFused) {
      // Algorithm 8's pair step: positions 4 th + u of row t are pairs
      // i = 2 (1024 t + th) (even) and i + 1 (odd), floor(i/2) = 1024 t + th
      const auto w = ld_tw(twf + (1u << (logn - 2)) + (t << 10) + th);
      fused_pair<false>(va[0], va[1], vb[0], vb[1], w, K);
      fused_pair<true>(va[2], va[3], vb[2], vb[3], w, K);
    } else {
#pragma unroll
      for (int u = 0; u < 4; u++)
        va[u] = mul_barrett_alg4(reduce4(va[u], K.q, K.two_q), reduce4(vb[u], K.q, K.two_q), K);
    }
    lat_inv<HALVE>(va, V.c + off, single, sa, twi, logn, t, th, K, kFused);
  }
}

// Forward column stages for n = 12 + log2 R, R in {2..32}: thread = (unit,
// operand, column); loads the R words {c + 4096 t}, runs the first log2 R
// stages of Algorithm 6, stores them back in place (to `dst`).
// For polymul, operand 0 (a) goes to c and operand 1 (b) to the scratch s.
// Each thread walks S columns (stride = the grid's thread count) and loads
// column k+1 while it transforms column k, so that its loads are in flight
// during the arithmetic.
// The column kernels are __device__ bodies with two __global__ wrappers:
// k_col_* with the compiler's own register choice, and k_col_*_cap compiled
// for 2 CTAs per SM.  The capped form serves 64-bit words with R = 32, whose
// 64 data registers per column otherwise leave 1 CTA per SM (the cap costs a
// few bytes of spill and gains ~8% at N = 2^17).  An explicit minimum of 1
// is not the same as none: the compiler then takes more registers.
// With DESC (grouped uneven launches, 64-bit words, S = 1) the unit's
// pointers come from its descriptor; a square unit (a == b) transforms its
// operand once (the op-1 thread has nothing to do).
template <int R, int S, typename W, bool DESC = false>
__device__ __forceinline__ void col_fwd_body(const KParams& P, int nops) {
  const KView<W> V(P);
  if constexpr (DESC) {
    static_assert(S == 1 && sizeof(W) == 8, "grouped launches: 64-bit words, one column per thread");
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (size_t)P.nunits * nops * kRow) return;
    const uint32_t col = (uint32_t)(id & (kRow - 1));
    const size_t rest = id >> kRowLog;
    const uint32_t op = (uint32_t)(rest % nops);
    const UnitDesc& D = P.desc[rest / nops];
    if (op == 1 && D.a == D.b) return;
    const W* src = (op == 0 ? D.a : D.b) + col;
    W* dst = (op == 0 ? D.c : D.s) + col;
    W x[R];
#pragma unroll
    for (int t = 0; t < R; t++) x[t] = __ldcs(src + (size_t)t * kRow);
    const auto K = ld_limb(D.lc);
    ct_col<R>(x, D.twf, K.q, K.two_q);
#pragma unroll
    for (int t = 0; t < R; t++) dst[(size_t)t * kRow] = x[t];
    return;
  }
  const uint32_t logn = P.logn;
  const size_t total = (size_t)P.nunits * nops * kRow;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  W nx[R];
  auto locate = [&](size_t id, const W*& src, W*& dst, uint32_t& limb) {
    const uint32_t col = (uint32_t)(id & (kRow - 1));
    const size_t rest = id >> kRowLog;
    const uint32_t op = (uint32_t)(rest % nops);
    const uint32_t unit = (uint32_t)(rest / nops);
    limb = unit % P.nlimbs;
    const size_t off = ((size_t)unit << logn) + col;
    src = (op == 0 ? V.a : V.b) + off;
    dst = (op == 0 ? V.c : V.s) + off;
  };
  const W* src;
  W* dst;
  uint32_t limb;
  locate(gid, src, dst, limb);
#pragma unroll
  for (int t = 0; t < R; t++) nx[t] = __ldcs(src + (size_t)t * kRow);
#pragma unroll 1
  for (int k = 0; k < S; k++) {
    W x[R];
#pragma unroll
    for (int t = 0; t < R; t++) x[t] = nx[t];
    W* cur_dst = dst;
    const uint32_t cur_limb = limb;
    const size_t nid = gid + stride;
    const bool more = (k + 1 < S) && nid < total;
    if (more) {
      locate(nid, src, dst, limb);
#pragma unroll
      for (int t = 0; t < R; t++) nx[t] = __ldcs(src + (size_t)t * kRow);
    }
    const auto K = ld_limb(V.lc + cur_limb);
    ct_col<R>(x, V.twf + ((size_t)cur_limb << logn), K.q, K.two_q);
#pragma unroll
    for (int t = 0; t < R; t++) cur_dst[(size_t)t * kRow] = x[t];
    if (!more) break;
    gid = nid;
  }
}

template <int R, int S, typename W, bool DESC = false>
__global__ void __launch_bounds__(256) k_col_fwd(KParams P, int nops) {
  col_fwd_body<R, S, W, DESC>(P, nops);
}

template <int R, int S, typename W, bool DESC = false>
__global__ void __launch_bounds__(256, 2) k_col_fwd_cap(KParams P, int nops) {
  col_fwd_body<R, S, W, DESC>(P, nops);
}

// Inverse column stages (the last log2 R stages of Algorithm 7) plus the
// reduction to [0, q); in place on c.  S columns per thread, software
// pipelined as in k_col_fwd.
template <int R, int S, bool HALVE, typename W, bool DESC = false>
__device__ __forceinline__ void col_inv_body(const KParams& P) {
  const KView<W> V(P);
  if constexpr (DESC) {
    static_assert(S == 1 && sizeof(W) == 8, "grouped launches: 64-bit words, one column per thread");
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (size_t)P.nunits * kRow) return;
    const UnitDesc& D = P.desc[id >> kRowLog];
    W* p = D.c + (id & (kRow - 1));
    W x[R];
#pragma unroll
    for (int t = 0; t < R; t++) x[t] = p[(size_t)t * kRow];
    const auto K = ld_limb(D.lc);
    gs_col<R, HALVE>(x, D.twi, K);
#pragma unroll
    for (int t = 0; t < R; t++) __stcs(p + (size_t)t * kRow, csub(x[t], K.q));
    return;
  }
  const uint32_t logn = P.logn;
  const size_t total = (size_t)P.nunits * kRow;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  auto locate = [&](size_t id, W*& p, uint32_t& limb) {
    const uint32_t col = (uint32_t)(id & (kRow - 1));
    const uint32_t unit = (uint32_t)(id >> kRowLog);
    limb = unit % P.nlimbs;
    p = V.c + ((size_t)unit << logn) + col;
  };
  W* p;
  uint32_t limb;
  locate(gid, p, limb);
  W nx[R];
#pragma unroll
  for (int t = 0; t < R; t++) nx[t] = p[(size_t)t * kRow];
#pragma unroll 1
  for (int k = 0; k < S; k++) {
    W x[R];
#pragma unroll
    for (int t = 0; t < R; t++) x[t] = nx[t];
    W* cur = p;
    const uint32_t cur_limb = limb;
    const size_t nid = gid + stride;
    const bool more = (k + 1 < S) && nid < total;
    if (more) {
      locate(nid, p, limb);
#pragma unroll
      for (int t = 0; t < R; t++) nx[t] = p[(size_t)t * kRow];
    }
    const auto K = ld_limb(V.lc + cur_limb);
    gs_col<R, HALVE>(x, V.twi + ((size_t)cur_limb << logn), K);
#pragma unroll
    for (int t = 0; t < R; t++) __stcs(cur + (size_t)t * kRow, csub(x[t], K.q));
    if (!more) break;
    gid = nid;
  }
}

template <int R, int S, bool HALVE, typename W, bool DESC = false>
__global__ void __launch_bounds__(256) k_col_inv(KParams P) {
  col_inv_body<R, S, HALVE, W, DESC>(P);
}

template <int R, int S, bool HALVE, typename W, bool DESC = false>
__global__ void __launch_bounds__(256, 2) k_col_inv_cap(KParams P) {
  col_inv_body<R, S, HALVE, W, DESC>(P);
}

// N = 2^13 in one CTA of 512 threads: 2 rows.  The single column stage
// (k = 4096) runs between global memory and smem; rows as in k_rows.
template <int MODE, bool HALVE, typename W>
__global__ void __launch_bounds__(512, 1) k_fused13(KParams P) {
  extern __shared__ __align__(16) uint64_t smem_raw[];
  W* smem = reinterpret_cast<W*>(smem_raw);
  const KView<W> V(P);
  constexpr uint32_t logn = 13;
  const uint32_t unit = blockIdx.x;
  if (unit >= P.nunits) return;
  const uint32_t limb = unit % P.nlimbs;
  const auto K = ld_limb(V.lc + limb);
  const auto* twf = V.twf + ((size_t)limb << logn);
  const auto* twi = V.twi + ((size_t)limb << logn);
  const int tid = threadIdx.x;
  const int rho = tid >> 8, th = tid & 255;
  // smem: [a row0][a row1][b row0][b row1]
  W* sA = smem;
  W* sB = smem + 2 * kRowPadW<W>;
  W* sa = sA + rho * kRowPadW<W>;
  W* sb = sB + rho * kRowPadW<W>;
  const size_t base = (size_t)unit << logn;
  W v[16];
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  if constexpr (MODE != MODE_INV) {
    const int nops = (MODE == MODE_FWD) ? 1 : 2;
    const auto w = ld_tw(twf + 1);
    for (int op = 0; op < nops; op++) {
      const W* src = (MODE == MODE_FWD) ? V.c + base : (op == 0 ? V.a : V.b) + base;
      W* dsm = op == 0 ? sA : sB;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int c = tid + 512 * k;
        W x0 = __ldcs(src + c), x1 = __ldcs(src + kRow + c);
        ct_bfly(x0, x1, w.w, w.wp, K.q, K.two_q);
        dsm[padj<W>(c)] = x0;
        dsm[kRowPadW<W> + padj<W>(c)] = x1;
      }
    }
    __syncthreads();
    rows_fwd(v, nullptr, sa, twf, logn, rho, th, K.q, K.two_q, kFused);
    if constexpr (MODE == MODE_FWD) {
      st_row16_reduced(V.c + base + (size_t)rho * kRow + 16 * th, v, K.q, K.two_q);
      return;
    } else {
      const PassGeo G2 = pass_geo<W>(2, th, rho);
      st_smem16(sa, G2, v);
      rows_fwd(v, nullptr, sb, twf, logn, rho, th, K.q, K.two_q, kFused);
      const W* a2 = sa + G2.pbase;
      if constexpr (kFused)
        fused_pairs16_smem(v, a2, twf, logn, G2.g, K);
      else
        pointwise16(v, a2, K);
    }
  } else {
    ld_row16(v, V.c + base + (size_t)rho * kRow + 16 * th);
  }
  rows_inv<HALVE>(v, nullptr, false, sa, twi, logn, rho, th, K, kFused);
  __syncthreads();
  // last GS stage (k = 4096, twiddle Psi^-1_br[1]; 1/N folded in unless the
  // plan halves at every stage), then reduce
  const auto w = ld_tw(twi + 1);
  W* dst = V.c + base;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const int c = tid + 512 * k;
    W x0 = sA[padj<W>(c)], x1 = sA[kRowPadW<W> + padj<W>(c)];
    if constexpr (HALVE)
      gs_bfly_half(x0, x1, w.w, w.wp, K.q, K.two_q, K.half_q1);
    else
      gs_bfly_last(x0, x1, K);
    __stcs(dst + c, csub(x0, K.q));
    __stcs(dst + kRow + c, csub(x1, K.q));
  }
}

// N <= 2^11: one CTA per unit, Algorithms 6 and 7 stage by stage in smem.
template <int MODE, bool HALVE, typename W>
__global__ void __launch_bounds__(256) k_small(KParams P) {
  extern __shared__ __align__(16) uint64_t smem_raw[];
  W* smem = reinterpret_cast<W*>(smem_raw);
  const KView<W> V(P);
  const uint32_t logn = P.logn, n = 1u << logn;
  const uint32_t unit = blockIdx.x;
  if (unit >= P.nunits) return;
  const uint32_t limb = unit % P.nlimbs;
  const auto K = ld_limb(V.lc + limb);
  const auto* twf = V.twf + ((size_t)limb << logn);
  const auto* twi = V.twi + ((size_t)limb << logn);
  const size_t base = (size_t)unit << logn;
  W* xa = smem;
  W* xb = smem + n;
  const W q = K.q, two_q = K.two_q;
  // Algorithm 8 (n >= 4): CT stops before its last stage (m = n/2), the pair
  // step replaces that stage, the products and the first GS stage, and GS
  // starts at m = n/4.
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  if constexpr (MODE != MODE_INV) {
    const int nops = (MODE == MODE_FWD) ? 1 : 2;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      xa[i] = (MODE == MODE_FWD) ? V.c[base + i] : V.a[base + i];
      if (nops == 2) xb[i] = V.b[base + i];
    }
    __syncthreads();
    for (uint32_t m = 1, k = n >> 1; m < (kFused ? n >> 1 : n); m <<= 1, k >>= 1) {
      for (uint32_t b = threadIdx.x; b < n / 2; b += blockDim.x) {
        const uint32_t i = b / k, j = 2 * i * k + (b % k);
        const auto w = ld_tw(twf + m + i);
        ct_bfly(xa[j], xa[j + k], w.w, w.wp, q, two_q);
        if (nops == 2) ct_bfly(xb[j], xb[j + k], w.w, w.wp, q, two_q);
      }
      __syncthreads();
    }
    if constexpr (MODE == MODE_FWD) {
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) V.c[base + i] = reduce4(xa[i], q, two_q);
      return;
    }
    if constexpr (kFused) {
      for (uint32_t i = threadIdx.x; i < n / 2; i += blockDim.x) {
        const auto w = ld_tw(twf + n / 4 + i / 2);
        if (i & 1)
          fused_pair<true>(xa[2 * i], xa[2 * i + 1], xb[2 * i], xb[2 * i + 1], w, K);
        else
          fused_pair<false>(xa[2 * i], xa[2 * i + 1], xb[2 * i], xb[2 * i + 1], w, K);
      }
    } else {
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
        xa[i] = mul_barrett_alg4(reduce4(xa[i], q, two_q), reduce4(xb[i], q, two_q), K);
    }
  } else {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) xa[i] = V.c[base + i];
  }
  __syncthreads();
  for (uint32_t m = n >> (kFused ? 2 : 1), k = kFused ? 2 : 1; m >= 1; m >>= 1, k <<= 1) {
    for (uint32_t b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const uint32_t i = b / k, j = 2 * i * k + (b % k);
      if (!HALVE && m == 1) {
        gs_bfly_last(xa[j], xa[j + k], K);  // last stage: 1/N folded in
      } else {
        const auto w = ld_tw(twi + m + i);
        gs_bfly_mode<HALVE>(xa[j], xa[j + k], w.w, w.wp, q, two_q, K.half_q1);
      }
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) V.c[base + i] = csub(xa[i], q);
}

// Stand-alone pointwise product, Algorithm 4, two words per thread.
template <typename W>
__global__ void __launch_bounds__(256) k_pointwise(KParams P) {
  const KView<W> V(P);
  using V2 = typename std::conditional<sizeof(W) == 8, ulonglong2, uint2>::type;
  const size_t total = (size_t)P.nunits << P.logn;
  const size_t stride = (size_t)gridDim.x * blockDim.x * 2;
  for (size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 2; i < total; i += stride) {
    const uint32_t limb = (uint32_t)((i >> P.logn) % P.nlimbs);
    const auto K = ld_limb(V.lc + limb);
    if (i + 1 < total && ((i + 1) >> P.logn) == (i >> P.logn)) {
      const V2 a = *reinterpret_cast<const V2*>(V.a + i);
      const V2 b = *reinterpret_cast<const V2*>(V.b + i);
      V2 c;
      c.x = mul_barrett_alg4(W(a.x), W(b.x), K);
      c.y = mul_barrett_alg4(W(a.y), W(b.y), K);
      *reinterpret_cast<V2*>(V.c + i) = c;
    } else {
      for (size_t k = i; k < i + 2 && k < total; k++) {
        const auto K2 = ld_limb(V.lc + (uint32_t)((k >> P.logn) % P.nlimbs));
        V.c[k] = mul_barrett_alg4(V.a[k], V.b[k], K2);
      }
    }
  }
}

// Range check 0 <= x < q_l; sets *flag = 1 on any violation.
template <typename W>
__global__ void __launch_bounds__(256) k_check_reduced(KParams P, int* flag) {
  const KView<W> V(P);
  const size_t total = (size_t)P.nunits << P.logn;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t limb = (uint32_t)((i >> P.logn) % P.nlimbs);
    if (V.a[i] >= __ldg(&V.lc[limb].q)) atomicOr(flag, 1);
  }
}

// ------------------------------------------------------------ launchers
// Templates over the word type W; the entry points at the end dispatch on
// KParams::word32.

static cudaError_t set_smem(const void* fn, int bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Columns per thread in the column kernels (software-pipelined loads).  Only
// batches of at least kPipeMinCols columns use it; small batches keep one
// column per thread so that they spread over as many SMs as possible.
constexpr int kColsPerThread = 4;
constexpr size_t kPipeMinCols = (size_t)1 << 20;

template <int R, typename W>
static cudaError_t launch_col_fwd(const KParams& P, int nops, cudaStream_t st) {
  const size_t cols = (size_t)P.nunits * nops * kRow;
  if constexpr (R < 32) {  // R = 32 holds too many registers to pipeline columns
    if (cols >= kPipeMinCols) {
      constexpr int S = kColsPerThread;
      const unsigned blocks = (unsigned)(((cols + S - 1) / S + 255) / 256);
      k_col_fwd<R, S, W><<<blocks, 256, 0, st>>>(P, nops);
      return cudaGetLastError();
    }
  }
  const unsigned blocks = (unsigned)((cols + 255) / 256);
  if constexpr (R == 32 && sizeof(W) == 8)
    k_col_fwd_cap<R, 1, W><<<blocks, 256, 0, st>>>(P, nops);
  else
    k_col_fwd<R, 1, W><<<blocks, 256, 0, st>>>(P, nops);
  return cudaGetLastError();
}

template <int R, typename W>
static cudaError_t launch_col_inv(const KParams& P, cudaStream_t st) {
  const size_t cols = (size_t)P.nunits * kRow;
  if constexpr (R < 32) {  // as in launch_col_fwd
    if (cols >= kPipeMinCols) {
      constexpr int S = kColsPerThread;
      const unsigned blocks = (unsigned)(((cols + S - 1) / S + 255) / 256);
      if (P.halving)
        k_col_inv<R, S, true, W><<<blocks, 256, 0, st>>>(P);
      else
        k_col_inv<R, S, false, W><<<blocks, 256, 0, st>>>(P);
      return cudaGetLastError();
    }
  }
  const unsigned blocks = (unsigned)((cols + 255) / 256);
  if constexpr (R == 32 && sizeof(W) == 8) {
    if (P.halving)
      k_col_inv_cap<R, 1, true, W><<<blocks, 256, 0, st>>>(P);
    else
      k_col_inv_cap<R, 1, false, W><<<blocks, 256, 0, st>>>(P);
  } else {
    if (P.halving)
      k_col_inv<R, 1, true, W><<<blocks, 256, 0, st>>>(P);
    else
      k_col_inv<R, 1, false, W><<<blocks, 256, 0, st>>>(P);
  }
  return cudaGetLastError();
}

template <typename W>
static cudaError_t col_fwd(const KParams& P, int nops, cudaStream_t st) {
  switch (P.logn) {
    case 13: return launch_col_fwd<2, W>(P, nops, st);
    case 14: return launch_col_fwd<4, W>(P, nops, st);
    case 15: return launch_col_fwd<8, W>(P, nops, st);
    case 16: return launch_col_fwd<16, W>(P, nops, st);
    case 17: return launch_col_fwd<32, W>(P, nops, st);
  }
  return cudaErrorInvalidValue;
}

template <typename W>
static cudaError_t col_inv(const KParams& P, cudaStream_t st) {
  switch (P.logn) {
    case 13: return launch_col_inv<2, W>(P, st);
    case 14: return launch_col_inv<4, W>(P, st);
    case 15: return launch_col_inv<8, W>(P, st);
    case 16: return launch_col_inv<16, W>(P, st);
    case 17: return launch_col_inv<32, W>(P, st);
  }
  return cudaErrorInvalidValue;
}

template <typename W>
constexpr int kRowsSmem = 2 * kRowPadW<W> * (int)sizeof(W);
template <typename W>
constexpr int kFused13Smem = 4 * kRowPadW<W> * (int)sizeof(W);

template <typename W>
constexpr int kLatSmem = 2 * kLatRowPad<W> * (int)sizeof(W);

template <int MODE, typename W>
static cudaError_t rows(const KParams& P, cudaStream_t st) {
  const unsigned blocks = P.nunits << (P.logn - kRowLog);
  constexpr int smem = kRowsSmem<W>;
  if (P.row_ops == 3) {
    if (P.halving)
      k_rows_lat<MODE, true, W><<<blocks, kLatThreads, kLatSmem<W>, st>>>(P);
    else
      k_rows_lat<MODE, false, W><<<blocks, kLatThreads, kLatSmem<W>, st>>>(P);
    return cudaGetLastError();
  }
  if ((MODE == MODE_POLYMUL || MODE == MODE_POLYMUL_FUSED) && P.row_ops == 2) {
    constexpr bool F = (MODE == MODE_POLYMUL_FUSED);
    if (P.halving)
      k_rows2<true, F, W><<<blocks, 256, smem, st>>>(P);
    else
      k_rows2<false, F, W><<<blocks, 256, smem, st>>>(P);
    return cudaGetLastError();
  }
  if (P.halving)
    k_rows<MODE, true, W><<<blocks, 256, smem, st>>>(P);
  else
    k_rows<MODE, false, W><<<blocks, 256, smem, st>>>(P);
  return cudaGetLastError();
}

template <int MODE, typename W>
static cudaError_t fused13(const KParams& P, cudaStream_t st) {
  if (P.halving)
    k_fused13<MODE, true, W><<<P.nunits, 512, kFused13Smem<W>, st>>>(P);
  else
    k_fused13<MODE, false, W><<<P.nunits, 512, kFused13Smem<W>, st>>>(P);
  return cudaGetLastError();
}

template <int MODE, typename W>
static cudaError_t small(const KParams& P, cudaStream_t st) {
  const int smem = 2 * (1 << P.logn) * (int)sizeof(W);
  if (P.halving)
    k_small<MODE, true, W><<<P.nunits, 256, smem, st>>>(P);
  else
    k_small<MODE, false, W><<<P.nunits, 256, smem, st>>>(P);
  return cudaGetLastError();
}

template <bool H, typename W>
static cudaError_t prepare_mode() {
  constexpr int rs = kRowsSmem<W>, fs = kFused13Smem<W>;
  const void* rows_fns[] = {(const void*)k_rows<MODE_POLYMUL, H, W>,
                            (const void*)k_rows<MODE_POLYMUL_FUSED, H, W>,
                            (const void*)k_rows2<H, false, W>,
                            (const void*)k_rows2<H, true, W>,
                            (const void*)k_rows2<H, false, W, sizeof(W) == 8>,
                            (const void*)k_rows2<H, true, W, sizeof(W) == 8>,
                            (const void*)k_rows<MODE_FWD, H, W>,
                            (const void*)k_rows<MODE_INV, H, W>};
  const void* lat_fns[] = {(const void*)k_rows_lat<MODE_POLYMUL, H, W>,
                           (const void*)k_rows_lat<MODE_POLYMUL_FUSED, H, W>,
                           (const void*)k_rows_lat<MODE_FWD, H, W>,
                           (const void*)k_rows_lat<MODE_INV, H, W>};
  const void* f13_fns[] = {(const void*)k_fused13<MODE_POLYMUL, H, W>,
                           (const void*)k_fused13<MODE_POLYMUL_FUSED, H, W>,
                           (const void*)k_fused13<MODE_FWD, H, W>,
                           (const void*)k_fused13<MODE_INV, H, W>};
  cudaError_t e;
  for (const void* f : rows_fns)
    if ((e = set_smem(f, rs)) != cudaSuccess) return e;
  for (const void* f : f13_fns)
    if ((e = set_smem(f, fs)) != cudaSuccess) return e;
  for (const void* f : lat_fns)
    if ((e = set_smem(f, kLatSmem<W>)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Opt the large-smem kernels in to their dynamic shared memory on the current
// device (once per device, before the first launch).
cudaError_t kernels_prepare() {
  cudaError_t e;
  if ((e = wide_prepare()) != cudaSuccess) return e;
  if ((e = prepare_mode<false, uint64_t>()) != cudaSuccess) return e;
  if ((e = prepare_mode<true, uint64_t>()) != cudaSuccess) return e;
  if ((e = prepare_mode<false, uint32_t>()) != cudaSuccess) return e;
  return prepare_mode<true, uint32_t>();
}

static inline cudaError_t mark(const PhaseEvents* pe, int k, cudaStream_t st) {
  return (pe && k < pe->n) ? cudaEventRecord(pe->ev[k], st) : cudaSuccess;
}

template <int MODE, typename W>
static cudaError_t polymul_rows(const KParams& P, cudaStream_t st) {
  if (P.logn <= 11) return small<MODE, W>(P, st);
  if (P.logn == 12) return rows<MODE, W>(P, st);
  if (P.logn == 13) return fused13<MODE, W>(P, st);
  return rows<MODE, W>(P, st);
}

template <typename W>
static cudaError_t launch_polymul_w(const KParams& P0, cudaStream_t st, const PhaseEvents* pe) {
  KParams P = P0;
  if (P.nunits == 0) return cudaSuccess;
  // Algorithm 8 plans: the fused constants (2/N) follow the plain ones
  if (P.fused)
    P.lc = reinterpret_cast<const LimbConst*>(
        reinterpret_cast<const typename WordT<W>::LC*>(P.lc) + P.nlimbs);
  auto prows = [&](const KParams& Q) {
    return Q.fused ? polymul_rows<MODE_POLYMUL_FUSED, W>(Q, st)
                   : polymul_rows<MODE_POLYMUL, W>(Q, st);
  };
  cudaError_t e0 = mark(pe, 0, st);
  if (e0 != cudaSuccess) return e0;
  if (P.logn <= 13) {
    e0 = prows(P);
    if (e0 != cudaSuccess) return e0;
    return mark(pe, 1, st);
  }
  // Column stages of a and b: one operand goes to c, the other to the
  // scratch s; the row kernel reads (c, s) in either order since the
  // pointwise product commutes.  Each column thread reads its own words
  // before writing them, so c may alias the operand whose image it receives.
  int nops = 2;
  if (P.a == P.b) {
    P.b = nullptr;
    P.s = P.c;  // square: one transform, read twice
    nops = 1;
  } else if (P.c == P.b) {
    const uint64_t* t = P.a;  // b's image stays in place, a's goes to s
    P.a = P.b;
    P.b = t;
  }
  cudaError_t e = col_fwd<W>(P, nops, st);
  if (e == cudaSuccess) e = mark(pe, 1, st);
  if (e == cudaSuccess) e = prows(P);
  if (e == cudaSuccess) e = mark(pe, 2, st);
  if (e == cudaSuccess) e = col_inv<W>(P, st);
  if (e == cudaSuccess) e = mark(pe, 3, st);
  return e;
}

template <typename W>
static cudaError_t launch_ntt_fwd_w(const KParams& P0, cudaStream_t st) {
  if (P0.nunits == 0) return cudaSuccess;
  KParams P = P0;
  if (P.logn <= 11) return small<MODE_FWD, W>(P, st);
  if (P.logn == 13) return fused13<MODE_FWD, W>(P, st);
  if (P.logn > 13) {
    P.a = P.c;  // in place: column stages read and write x
    cudaError_t e = col_fwd<W>(P, 1, st);
    if (e != cudaSuccess) return e;
  }
  return rows<MODE_FWD, W>(P, st);
}

template <typename W>
static cudaError_t launch_ntt_inv_w(const KParams& P, cudaStream_t st) {
  if (P.nunits == 0) return cudaSuccess;
  if (P.logn <= 11) return small<MODE_INV, W>(P, st);
  if (P.logn == 13) return fused13<MODE_INV, W>(P, st);
  cudaError_t e = rows<MODE_INV, W>(P, st);
  if (e != cudaSuccess || P.logn == 12) return e;
  return col_inv<W>(P, st);
}

// Grouped uneven launch (64-bit words): all units of one N, pointers from
// P.desc; the column stages one column per thread, the two-operand rows.
template <int R>
static cudaError_t polymul_desc_r(const KParams& P, cudaStream_t st) {
  using W = uint64_t;
  const unsigned rows = P.nunits << (P.logn - kRowLog);
  if constexpr (R > 1) {
    const unsigned fb = (unsigned)(((size_t)P.nunits * 2 * kRow + 255) / 256);
    if constexpr (R == 32)
      k_col_fwd_cap<R, 1, W, true><<<fb, 256, 0, st>>>(P, 2);
    else
      k_col_fwd<R, 1, W, true><<<fb, 256, 0, st>>>(P, 2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (P.halving) {
    if (P.fused)
      k_rows2<true, true, W, true><<<rows, 256, kRowsSmem<W>, st>>>(P);
    else
      k_rows2<true, false, W, true><<<rows, 256, kRowsSmem<W>, st>>>(P);
  } else {
    if (P.fused)
      k_rows2<false, true, W, true><<<rows, 256, kRowsSmem<W>, st>>>(P);
    else
      k_rows2<false, false, W, true><<<rows, 256, kRowsSmem<W>, st>>>(P);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || R == 1) return e;
  const unsigned ib = (unsigned)(((size_t)P.nunits * kRow + 255) / 256);
  if constexpr (R == 32) {
    if (P.halving)
      k_col_inv_cap<R, 1, true, W, true><<<ib, 256, 0, st>>>(P);
    else
      k_col_inv_cap<R, 1, false, W, true><<<ib, 256, 0, st>>>(P);
  } else if constexpr (R > 1) {
    if (P.halving)
      k_col_inv<R, 1, true, W, true><<<ib, 256, 0, st>>>(P);
    else
      k_col_inv<R, 1, false, W, true><<<ib, 256, 0, st>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t launch_polymul_grouped(const KParams& P, cudaStream_t st) {
  if (P.nunits == 0) return cudaSuccess;
  if (P.word32 || !P.desc) return cudaErrorInvalidValue;
  if (P.row_ops == 4 && P.logn >= 13) return launch_polymul_wide_grouped(P, st);
  switch (P.logn) {
    case 12: return polymul_desc_r<1>(P, st);
    case 13: return polymul_desc_r<2>(P, st);
    case 14: return polymul_desc_r<4>(P, st);
    case 15: return polymul_desc_r<8>(P, st);
    case 16: return polymul_desc_r<16>(P, st);
    case 17: return polymul_desc_r<32>(P, st);
  }
  return cudaErrorInvalidValue;
}

static unsigned grid_cap(size_t blocks, int num_sms) {
  const size_t cap = (size_t)num_sms * 8;
  return (unsigned)(blocks > cap ? cap : blocks);
}

cudaError_t launch_polymul(const KParams& P, cudaStream_t st, const PhaseEvents* pe) {
  if (P.row_ops == 4 && wide_polymul_ok(P.logn)) return launch_polymul_wide(P, st, pe);
  return P.word32 ? launch_polymul_w<uint32_t>(P, st, pe) : launch_polymul_w<uint64_t>(P, st, pe);
}

bool polymul_writes_scratch(const KParams& P) {
  if (P.nunits == 0 || !polymul_needs_scratch(P.logn) || P.a == P.b) return false;
  if (P.row_ops == 4 && wide_polymul_ok(P.logn)) return !wide_single_launch(P.logn, P.nunits);
  return true;
}

cudaError_t launch_ntt_fwd(const KParams& P, cudaStream_t st) {
  if (P.row_ops == 4 && wide_ntt_ok(P.logn)) return launch_ntt_fwd_wide(P, st);
  return P.word32 ? launch_ntt_fwd_w<uint32_t>(P, st) : launch_ntt_fwd_w<uint64_t>(P, st);
}

cudaError_t launch_ntt_inv(const KParams& P, cudaStream_t st) {
  if (P.row_ops == 4 && wide_ntt_ok(P.logn)) return launch_ntt_inv_wide(P, st);
  return P.word32 ? launch_ntt_inv_w<uint32_t>(P, st) : launch_ntt_inv_w<uint64_t>(P, st);
}

cudaError_t launch_pointwise(const KParams& P, cudaStream_t st, int num_sms) {
  const size_t total = (size_t)P.nunits << P.logn;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = grid_cap((total / 2 + 255) / 256, num_sms);
  if (P.word32)
    k_pointwise<uint32_t><<<blocks, 256, 0, st>>>(P);
  else
    k_pointwise<uint64_t><<<blocks, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_check_reduced(const KParams& P, int* d_flag, cudaStream_t st, int num_sms) {
  const size_t total = (size_t)P.nunits << P.logn;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = grid_cap((total + 255) / 256, num_sms);
  if (P.word32)
    k_check_reduced<uint32_t><<<blocks, 256, 0, st>>>(P, d_flag);
  else
    k_check_reduced<uint64_t><<<blocks, 256, 0, st>>>(P, d_flag);
  return cudaGetLastError();
}

}  // namespace pm
