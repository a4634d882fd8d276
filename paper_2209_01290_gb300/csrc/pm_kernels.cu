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
// Kernels
//   k_col_fwd<R>    : the n-12 forward column stages, streaming (registers
//                     only, coalesced loads/stores), one thread per column.
//   k_rows<MODE>    : the 12 in-row stages as three radix-16 passes; each
//                     thread keeps 16 words per operand in registers and
//                     rows are exchanged through padded shared memory between
//                     passes.  For polymul the last forward pass, the
//                     Barrett product (Algorithm 4) and the first inverse pass
//                     run back to back in registers.
//   k_col_inv<R>    : the n-12 inverse column stages and the final reduction.
//   k_fused13       : N = 2^13 in one CTA (column stage through smem).
//   k_small         : N <= 2^11, one CTA per unit, radix-2 stages in smem.
//   k_pointwise     : stand-alone Hadamard product with Algorithm 4.
#include <cuda_runtime.h>
#include <cstdint>

#include "pm_arith.cuh"
#include "pm_internal.h"
#include "pm_passes.cuh"

namespace pm {

// ------------------------------------------------------------------ kernels

// In-row stages for n >= 12.  One CTA = one row (256 threads).  For n == 12
// the row is the whole unit (polymul reads a, b; output canonical).  For
// n > 12, polymul reads the column-transformed operands from c and the
// scratch s and leaves lazy c' rows for k_col_inv.
template <int MODE, bool HALVE>
__global__ void __launch_bounds__(256, 3) k_rows(KParams P) {
  extern __shared__ __align__(16) uint64_t smem[];
  const uint32_t logn = P.logn;
  const uint32_t unit = blockIdx.x >> (logn - kRowLog);
  const uint32_t t = blockIdx.x & ((1u << (logn - kRowLog)) - 1);
  if (unit >= P.nunits) return;  // whole CTA exits together
  const uint32_t limb = unit % P.nlimbs;
  const LimbConst K = ld_limb(P.lc + limb);
  const TwPair* twf = P.twf + ((size_t)limb << logn);
  const TwPair* twi = P.twi + ((size_t)limb << logn);
  const size_t off = ((size_t)unit << logn) + (size_t)t * kRow;
  const bool single = (logn == kRowLog);
  const int th = threadIdx.x;
  uint64_t* sa = smem;
  uint64_t* sb = smem + kRowPad;
  uint64_t v[16];
  if constexpr (MODE == MODE_INV) {
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(P.c + off + 16 * th);
#pragma unroll
    for (int u = 0; u < 16; u += 2) {
      const ulonglong2 w = __ldcs(src + u / 2);
      v[u] = w.x;
      v[u + 1] = w.y;
    }
    rows_inv<HALVE>(v, P.c + off, single, sa, twi, logn, t, th, K);
  } else if constexpr (MODE == MODE_FWD) {
    rows_fwd(v, P.c + off, sa, twf, logn, t, th, K.q, K.two_q);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(P.c + off + 16 * th);
#pragma unroll
    for (int u = 0; u < 16; u += 2)
      __stcs(dst + u / 2, make_ulonglong2(reduce4(v[u], K.q, K.two_q),
                                          reduce4(v[u + 1], K.q, K.two_q)));
  } else {
    (void)sb;
    row_task_polymul<HALVE, false>((single ? P.a : P.c) + off, (single ? P.b : P.s) + off,
                                   P.c + off, single, smem, twf, twi, K, logn, t,
                                   MODE == MODE_POLYMUL_FUSED);
  }
}

// Polymul rows with a and b transformed together in registers (shared
// twiddle loads, half the barriers per word; 2 CTAs per SM).
template <bool HALVE, bool FUSED>
__global__ void __launch_bounds__(256, 2) k_rows2(KParams P) {
  extern __shared__ __align__(16) uint64_t smem[];
  const uint32_t logn = P.logn;
  const uint32_t unit = blockIdx.x >> (logn - kRowLog);
  const uint32_t t = blockIdx.x & ((1u << (logn - kRowLog)) - 1);
  if (unit >= P.nunits) return;
  const uint32_t limb = unit % P.nlimbs;
  const LimbConst K = ld_limb(P.lc + limb);
  const TwPair* twf = P.twf + ((size_t)limb << logn);
  const TwPair* twi = P.twi + ((size_t)limb << logn);
  const size_t off = ((size_t)unit << logn) + (size_t)t * kRow;
  const bool single = (logn == kRowLog);
  row_task_polymul2<HALVE, false>((single ? P.a : P.c) + off, (single ? P.b : P.s) + off,
                                  P.c + off, single, smem, twf, twi, K, logn, t, FUSED);
}

// Forward column stages for n = 12 + log2 R, R in {2..32}: thread = (unit,
// operand, column); loads the R words {c + 4096 t}, runs the first log2 R
// stages of Algorithm 6, stores them back in place (to `dst`).
// For polymul, operand 0 (a) goes to c and operand 1 (b) to the scratch s.
// Each thread walks S columns (stride = the grid's thread count) and loads
// column k+1 while it transforms column k, so that its loads are in flight
// during the arithmetic.
template <int R, int S>
__global__ void __launch_bounds__(256) k_col_fwd(KParams P, int nops) {
  const uint32_t logn = P.logn;
  const size_t total = (size_t)P.nunits * nops * kRow;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  uint64_t nx[R];
  auto locate = [&](size_t id, const uint64_t*& src, uint64_t*& dst, uint32_t& limb) {
    const uint32_t col = (uint32_t)(id & (kRow - 1));
    const size_t rest = id >> kRowLog;
    const uint32_t op = (uint32_t)(rest % nops);
    const uint32_t unit = (uint32_t)(rest / nops);
    limb = unit % P.nlimbs;
    const size_t off = ((size_t)unit << logn) + col;
    src = (op == 0 ? P.a : P.b) + off;
    dst = (op == 0 ? P.c : P.s) + off;
  };
  const uint64_t* src;
  uint64_t* dst;
  uint32_t limb;
  locate(gid, src, dst, limb);
#pragma unroll
  for (int t = 0; t < R; t++) nx[t] = __ldcs(src + (size_t)t * kRow);
#pragma unroll 1
  for (int k = 0; k < S; k++) {
    uint64_t x[R];
#pragma unroll
    for (int t = 0; t < R; t++) x[t] = nx[t];
    uint64_t* cur_dst = dst;
    const uint32_t cur_limb = limb;
    const size_t nid = gid + stride;
    const bool more = (k + 1 < S) && nid < total;
    if (more) {
      locate(nid, src, dst, limb);
#pragma unroll
      for (int t = 0; t < R; t++) nx[t] = __ldcs(src + (size_t)t * kRow);
    }
    const LimbConst K = ld_limb(P.lc + cur_limb);
    ct_col<R>(x, P.twf + ((size_t)cur_limb << logn), K.q, K.two_q);
#pragma unroll
    for (int t = 0; t < R; t++) cur_dst[(size_t)t * kRow] = x[t];
    if (!more) break;
    gid = nid;
  }
}

// Inverse column stages (the last log2 R stages of Algorithm 7) plus the
// reduction to [0, q); in place on c.  S columns per thread, software
// pipelined as in k_col_fwd.
template <int R, int S, bool HALVE>
__global__ void __launch_bounds__(256) k_col_inv(KParams P) {
  const uint32_t logn = P.logn;
  const size_t total = (size_t)P.nunits * kRow;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  auto locate = [&](size_t id, uint64_t*& p, uint32_t& limb) {
    const uint32_t col = (uint32_t)(id & (kRow - 1));
    const uint32_t unit = (uint32_t)(id >> kRowLog);
    limb = unit % P.nlimbs;
    p = P.c + ((size_t)unit << logn) + col;
  };
  uint64_t* p;
  uint32_t limb;
  locate(gid, p, limb);
  uint64_t nx[R];
#pragma unroll
  for (int t = 0; t < R; t++) nx[t] = p[(size_t)t * kRow];
#pragma unroll 1
  for (int k = 0; k < S; k++) {
    uint64_t x[R];
#pragma unroll
    for (int t = 0; t < R; t++) x[t] = nx[t];
    uint64_t* cur = p;
    const uint32_t cur_limb = limb;
    const size_t nid = gid + stride;
    const bool more = (k + 1 < S) && nid < total;
    if (more) {
      locate(nid, p, limb);
#pragma unroll
      for (int t = 0; t < R; t++) nx[t] = p[(size_t)t * kRow];
    }
    const LimbConst K = ld_limb(P.lc + cur_limb);
    gs_col<R, HALVE>(x, P.twi + ((size_t)cur_limb << logn), K);
#pragma unroll
    for (int t = 0; t < R; t++) __stcs(cur + (size_t)t * kRow, csub(x[t], K.q));
    if (!more) break;
    gid = nid;
  }
}

// N = 2^13 in one CTA of 512 threads: 2 rows.  The single column stage
// (k = 4096) runs between global memory and smem; rows as in k_rows.
template <int MODE, bool HALVE>
__global__ void __launch_bounds__(512, 1) k_fused13(KParams P) {
  extern __shared__ __align__(16) uint64_t smem[];
  constexpr uint32_t logn = 13;
  const uint32_t unit = blockIdx.x;
  if (unit >= P.nunits) return;
  const uint32_t limb = unit % P.nlimbs;
  const LimbConst K = ld_limb(P.lc + limb);
  const TwPair* twf = P.twf + ((size_t)limb << logn);
  const TwPair* twi = P.twi + ((size_t)limb << logn);
  const int tid = threadIdx.x;
  const int rho = tid >> 8, th = tid & 255;
  // smem: [a row0][a row1][b row0][b row1]
  uint64_t* sA = smem;
  uint64_t* sB = smem + 2 * kRowPad;
  uint64_t* sa = sA + rho * kRowPad;
  uint64_t* sb = sB + rho * kRowPad;
  const size_t base = (size_t)unit << logn;
  uint64_t v[16];
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  if constexpr (MODE != MODE_INV) {
    const int nops = (MODE == MODE_FWD) ? 1 : 2;
    const TwPair w = ld_tw(twf + 1);
    for (int op = 0; op < nops; op++) {
      const uint64_t* src = (MODE == MODE_FWD) ? P.c + base : (op == 0 ? P.a : P.b) + base;
      uint64_t* dsm = op == 0 ? sA : sB;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int c = tid + 512 * k;
        uint64_t x0 = __ldcs(src + c), x1 = __ldcs(src + kRow + c);
        ct_bfly(x0, x1, w.w, w.wp, K.q, K.two_q);
        dsm[padj(c)] = x0;
        dsm[kRowPad + padj(c)] = x1;
      }
    }
    __syncthreads();
    rows_fwd(v, nullptr, sa, twf, logn, rho, th, K.q, K.two_q, kFused);
    if constexpr (MODE == MODE_FWD) {
      ulonglong2* dst = reinterpret_cast<ulonglong2*>(P.c + base + (size_t)rho * kRow + 16 * th);
#pragma unroll
      for (int u = 0; u < 16; u += 2)
        __stcs(dst + u / 2, make_ulonglong2(reduce4(v[u], K.q, K.two_q),
                                            reduce4(v[u + 1], K.q, K.two_q)));
      return;
    } else {
      const PassGeo G2 = pass_geo(2, th, rho);
      st_smem16(sa, G2, v);
      rows_fwd(v, nullptr, sb, twf, logn, rho, th, K.q, K.two_q, kFused);
      const uint64_t* a2 = sa + G2.pbase;
      if constexpr (kFused)
        fused_pairs16_smem(v, a2, twf, logn, G2.g, K);
      else
        pointwise16(v, a2, K);
    }
  } else {
    const ulonglong2* src =
        reinterpret_cast<const ulonglong2*>(P.c + base + (size_t)rho * kRow + 16 * th);
#pragma unroll
    for (int u = 0; u < 16; u += 2) {
      const ulonglong2 w = __ldcs(src + u / 2);
      v[u] = w.x;
      v[u + 1] = w.y;
    }
  }
  rows_inv<HALVE>(v, nullptr, false, sa, twi, logn, rho, th, K, kFused);
  __syncthreads();
  // last GS stage (k = 4096, twiddle Psi^-1_br[1]; 1/N folded in unless the
  // plan halves at every stage), then reduce
  const TwPair w = ld_tw(twi + 1);
  uint64_t* dst = P.c + base;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const int c = tid + 512 * k;
    uint64_t x0 = sA[padj(c)], x1 = sA[kRowPad + padj(c)];
    if constexpr (HALVE)
      gs_bfly_half(x0, x1, w.w, w.wp, K.q, K.two_q, K.half_q1);
    else
      gs_bfly_last(x0, x1, K);
    __stcs(dst + c, csub(x0, K.q));
    __stcs(dst + kRow + c, csub(x1, K.q));
  }
}

// N <= 2^11: one CTA per unit, Algorithms 6 and 7 stage by stage in smem.
template <int MODE, bool HALVE>
__global__ void __launch_bounds__(256) k_small(KParams P) {
  extern __shared__ __align__(16) uint64_t smem[];
  const uint32_t logn = P.logn, n = 1u << logn;
  const uint32_t unit = blockIdx.x;
  if (unit >= P.nunits) return;
  const uint32_t limb = unit % P.nlimbs;
  const LimbConst K = ld_limb(P.lc + limb);
  const TwPair* twf = P.twf + ((size_t)limb << logn);
  const TwPair* twi = P.twi + ((size_t)limb << logn);
  const size_t base = (size_t)unit << logn;
  uint64_t* xa = smem;
  uint64_t* xb = smem + n;
  const uint64_t q = K.q, two_q = K.two_q;
  // Algorithm 8 (n >= 4): CT stops before its last stage (m = n/2), the pair
  // step replaces that stage, the products and the first GS stage, and GS
  // starts at m = n/4.
  constexpr bool kFused = (MODE == MODE_POLYMUL_FUSED);
  if constexpr (MODE != MODE_INV) {
    const int nops = (MODE == MODE_FWD) ? 1 : 2;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      xa[i] = (MODE == MODE_FWD) ? P.c[base + i] : P.a[base + i];
      if (nops == 2) xb[i] = P.b[base + i];
    }
    __syncthreads();
    for (uint32_t m = 1, k = n >> 1; m < (kFused ? n >> 1 : n); m <<= 1, k >>= 1) {
      for (uint32_t b = threadIdx.x; b < n / 2; b += blockDim.x) {
        const uint32_t i = b / k, j = 2 * i * k + (b % k);
        const TwPair w = ld_tw(twf + m + i);
        ct_bfly(xa[j], xa[j + k], w.w, w.wp, q, two_q);
        if (nops == 2) ct_bfly(xb[j], xb[j + k], w.w, w.wp, q, two_q);
      }
      __syncthreads();
    }
    if constexpr (MODE == MODE_FWD) {
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) P.c[base + i] = reduce4(xa[i], q, two_q);
      return;
    }
    if constexpr (kFused) {
      for (uint32_t i = threadIdx.x; i < n / 2; i += blockDim.x) {
        const TwPair w = ld_tw(twf + n / 4 + i / 2);
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
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) xa[i] = P.c[base + i];
  }
  __syncthreads();
  for (uint32_t m = n >> (kFused ? 2 : 1), k = kFused ? 2 : 1; m >= 1; m >>= 1, k <<= 1) {
    for (uint32_t b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const uint32_t i = b / k, j = 2 * i * k + (b % k);
      if (!HALVE && m == 1) {
        gs_bfly_last(xa[j], xa[j + k], K);  // last stage: 1/N folded in
      } else {
        const TwPair w = ld_tw(twi + m + i);
        gs_bfly_mode<HALVE>(xa[j], xa[j + k], w.w, w.wp, q, two_q, K.half_q1);
      }
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) P.c[base + i] = csub(xa[i], q);
}

// Stand-alone pointwise product, Algorithm 4, two words per thread.
__global__ void __launch_bounds__(256) k_pointwise(KParams P) {
  const size_t total = (size_t)P.nunits << P.logn;
  const size_t stride = (size_t)gridDim.x * blockDim.x * 2;
  for (size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 2; i < total; i += stride) {
    const uint32_t limb = (uint32_t)((i >> P.logn) % P.nlimbs);
    const LimbConst K = ld_limb(P.lc + limb);
    if (i + 1 < total && ((i + 1) >> P.logn) == (i >> P.logn)) {
      const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(P.a + i);
      const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(P.b + i);
      *reinterpret_cast<ulonglong2*>(P.c + i) =
          make_ulonglong2(mul_barrett_alg4(a.x, b.x, K), mul_barrett_alg4(a.y, b.y, K));
    } else {
      for (size_t k = i; k < i + 2 && k < total; k++) {
        const LimbConst K2 = ld_limb(P.lc + (uint32_t)((k >> P.logn) % P.nlimbs));
        P.c[k] = mul_barrett_alg4(P.a[k], P.b[k], K2);
      }
    }
  }
}

// Range check 0 <= x < q_l; sets *flag = 1 on any violation.
__global__ void __launch_bounds__(256) k_check_reduced(KParams P, int* flag) {
  const size_t total = (size_t)P.nunits << P.logn;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t limb = (uint32_t)((i >> P.logn) % P.nlimbs);
    if (P.a[i] >= __ldg(&P.lc[limb].q)) atomicOr(flag, 1);
  }
}

// ------------------------------------------------------------ launchers

static cudaError_t set_smem(const void* fn, int bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Columns per thread in the column kernels (software-pipelined loads).  Only
// batches of at least kPipeMinCols columns use it; small batches keep one
// column per thread so that they spread over as many SMs as possible.
constexpr int kColsPerThread = 4;
constexpr size_t kPipeMinCols = (size_t)1 << 20;

template <int R>
static cudaError_t launch_col_fwd(const KParams& P, int nops, cudaStream_t st) {
  const size_t cols = (size_t)P.nunits * nops * kRow;
  if (R < 32 && cols >= kPipeMinCols) {
    constexpr int S = kColsPerThread;
    const unsigned blocks = (unsigned)(((cols + S - 1) / S + 255) / 256);
    k_col_fwd<R, S><<<blocks, 256, 0, st>>>(P, nops);
  } else {
    k_col_fwd<R, 1><<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(P, nops);
  }
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_col_inv(const KParams& P, cudaStream_t st) {
  const size_t cols = (size_t)P.nunits * kRow;
  const bool pipe = R < 32 && cols >= kPipeMinCols;
  constexpr int S = kColsPerThread;
  const unsigned blocks = (unsigned)((((pipe ? (cols + S - 1) / S : cols)) + 255) / 256);
  if (pipe) {
    if (P.halving)
      k_col_inv<R, S, true><<<blocks, 256, 0, st>>>(P);
    else
      k_col_inv<R, S, false><<<blocks, 256, 0, st>>>(P);
  } else {
    if (P.halving)
      k_col_inv<R, 1, true><<<blocks, 256, 0, st>>>(P);
    else
      k_col_inv<R, 1, false><<<blocks, 256, 0, st>>>(P);
  }
  return cudaGetLastError();
}

static cudaError_t col_fwd(const KParams& P, int nops, cudaStream_t st) {
  switch (P.logn) {
    case 13: return launch_col_fwd<2>(P, nops, st);
    case 14: return launch_col_fwd<4>(P, nops, st);
    case 15: return launch_col_fwd<8>(P, nops, st);
    case 16: return launch_col_fwd<16>(P, nops, st);
    case 17: return launch_col_fwd<32>(P, nops, st);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t col_inv(const KParams& P, cudaStream_t st) {
  switch (P.logn) {
    case 13: return launch_col_inv<2>(P, st);
    case 14: return launch_col_inv<4>(P, st);
    case 15: return launch_col_inv<8>(P, st);
    case 16: return launch_col_inv<16>(P, st);
    case 17: return launch_col_inv<32>(P, st);
  }
  return cudaErrorInvalidValue;
}

constexpr int kRowsSmem = 2 * kRowPad * 8;
constexpr int kFused13Smem = 4 * kRowPad * 8;

template <int MODE>
static cudaError_t rows(const KParams& P, cudaStream_t st) {
  const unsigned blocks = P.nunits << (P.logn - kRowLog);
  if ((MODE == MODE_POLYMUL || MODE == MODE_POLYMUL_FUSED) && P.row_ops == 2) {
    constexpr bool F = (MODE == MODE_POLYMUL_FUSED);
    if (P.halving)
      k_rows2<true, F><<<blocks, 256, kRowsSmem, st>>>(P);
    else
      k_rows2<false, F><<<blocks, 256, kRowsSmem, st>>>(P);
    return cudaGetLastError();
  }
  if (P.halving)
    k_rows<MODE, true><<<blocks, 256, kRowsSmem, st>>>(P);
  else
    k_rows<MODE, false><<<blocks, 256, kRowsSmem, st>>>(P);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t fused13(const KParams& P, cudaStream_t st) {
  if (P.halving)
    k_fused13<MODE, true><<<P.nunits, 512, kFused13Smem, st>>>(P);
  else
    k_fused13<MODE, false><<<P.nunits, 512, kFused13Smem, st>>>(P);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t small(const KParams& P, cudaStream_t st) {
  const int smem = 2 * (1 << P.logn) * 8;
  if (P.halving)
    k_small<MODE, true><<<P.nunits, 256, smem, st>>>(P);
  else
    k_small<MODE, false><<<P.nunits, 256, smem, st>>>(P);
  return cudaGetLastError();
}

template <bool H>
static cudaError_t prepare_mode() {
  cudaError_t e;
  if ((e = set_smem((const void*)k_rows<MODE_POLYMUL, H>, kRowsSmem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_rows<MODE_POLYMUL_FUSED, H>, kRowsSmem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_rows2<H, false>, kRowsSmem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_rows2<H, true>, kRowsSmem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_rows<MODE_FWD, H>, kRowsSmem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_rows<MODE_INV, H>, kRowsSmem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_fused13<MODE_POLYMUL, H>, kFused13Smem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_fused13<MODE_POLYMUL_FUSED, H>, kFused13Smem)) != cudaSuccess)
    return e;
  if ((e = set_smem((const void*)k_fused13<MODE_FWD, H>, kFused13Smem)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_fused13<MODE_INV, H>, kFused13Smem)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Opt the large-smem kernels in to their dynamic shared memory on the current
// device (once per device, before the first launch).
cudaError_t kernels_prepare() {
  cudaError_t e = prepare_mode<false>();
  return e != cudaSuccess ? e : prepare_mode<true>();
}

static inline cudaError_t mark(const PhaseEvents* pe, int k, cudaStream_t st) {
  return (pe && k < pe->n) ? cudaEventRecord(pe->ev[k], st) : cudaSuccess;
}

template <int MODE>
static cudaError_t polymul_rows(const KParams& P, cudaStream_t st) {
  if (P.logn <= 11) return small<MODE>(P, st);
  if (P.logn == 12) return rows<MODE>(P, st);
  if (P.logn == 13) return fused13<MODE>(P, st);
  return rows<MODE>(P, st);
}

cudaError_t launch_polymul(const KParams& P0, cudaStream_t st, const PhaseEvents* pe) {
  KParams P = P0;
  if (P.nunits == 0) return cudaSuccess;
  // Algorithm 8 plans: the fused constants (2/N) follow the plain ones
  if (P.fused) P.lc += P.nlimbs;
  auto prows = [&](const KParams& Q) {
    return Q.fused ? polymul_rows<MODE_POLYMUL_FUSED>(Q, st) : polymul_rows<MODE_POLYMUL>(Q, st);
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
  cudaError_t e = col_fwd(P, nops, st);
  if (e == cudaSuccess) e = mark(pe, 1, st);
  if (e == cudaSuccess) e = prows(P);
  if (e == cudaSuccess) e = mark(pe, 2, st);
  if (e == cudaSuccess) e = col_inv(P, st);
  if (e == cudaSuccess) e = mark(pe, 3, st);
  return e;
}

cudaError_t launch_ntt_fwd(const KParams& P0, cudaStream_t st) {
  if (P0.nunits == 0) return cudaSuccess;
  KParams P = P0;
  if (P.logn <= 11) return small<MODE_FWD>(P, st);
  if (P.logn == 13) return fused13<MODE_FWD>(P, st);
  if (P.logn > 13) {
    P.a = P.c;  // in place: column stages read and write x
    cudaError_t e = col_fwd(P, 1, st);
    if (e != cudaSuccess) return e;
  }
  return rows<MODE_FWD>(P, st);
}

cudaError_t launch_ntt_inv(const KParams& P, cudaStream_t st) {
  if (P.nunits == 0) return cudaSuccess;
  if (P.logn <= 11) return small<MODE_INV>(P, st);
  if (P.logn == 13) return fused13<MODE_INV>(P, st);
  cudaError_t e = rows<MODE_INV>(P, st);
  if (e != cudaSuccess || P.logn == 12) return e;
  return col_inv(P, st);
}

cudaError_t launch_pointwise(const KParams& P, cudaStream_t st, int num_sms) {
  const size_t total = (size_t)P.nunits << P.logn;
  if (total == 0) return cudaSuccess;
  size_t blocks = (total / 2 + 255) / 256;
  const size_t cap = (size_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  k_pointwise<<<(unsigned)blocks, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_check_reduced(const KParams& P, int* d_flag, cudaStream_t st, int num_sms) {
  const size_t total = (size_t)P.nunits << P.logn;
  if (total == 0) return cudaSuccess;
  size_t blocks = (total + 255) / 256;
  const size_t cap = (size_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  k_check_reduced<<<(unsigned)blocks, 256, 0, st>>>(P, d_flag);
  return cudaGetLastError();
}

}  // namespace pm
