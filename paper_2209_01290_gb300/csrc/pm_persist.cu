// pm_persist.cu -- one persistent launch for a whole batch of negacyclic
// products (arxiv 2209.01290, Eq. 2, batched over RNS limbs and polynomials
// like the paper's throughput-oriented TOM-NTT, Sec. V-C).
//
// The column-split path (N = R * 4096) has three kinds of work per unit:
//   F column-forward tasks (256 columns of one operand each, the first
//     log2 R stages of Algorithm 6),
//   W = R row tasks (the 12 in-row forward stages of a and b, the
//     Algorithm 4 pointwise product, the 12 in-row inverse stages),
//   I = 16 column-inverse tasks (the last log2 R stages of Algorithm 7 and
//     the reduction to [0, q)).
// Instead of three launches, a grid of CTAs that stays resident takes
// tickets from a global counter in a fixed software-pipelined order: ticket
// group g holds the column-forward tasks of unit g, the row tasks of unit
// g - lagF and the column-inverse tasks of unit g - lagI.  Memory-bound
// column work of one unit therefore runs on the SMs at the same time as the
// compute-bound row work of others, and each unit's intermediate image is
// read back a few groups after it was written, while it is still in L2.
//
// A row task waits until all column-forward tasks of its unit are done, a
// column-inverse task until all its unit's rows are done (per-unit counters,
// release/acquire at GPU scope).  Tickets are handed out in order and a
// task only ever waits for tasks with smaller tickets, which were taken by
// running CTAs, so every wait ends; each wait is still bounded (about a
// second), after which the CTA records PM_ERR_TIMEOUT in the control block
// and carries on.
#include <cuda_runtime.h>

#include <cstdint>

#include "pm_arith.cuh"
#include "pm_internal.h"
#include "pm_passes.cuh"
#include "pm_sync.cuh"

namespace pm {

namespace {

constexpr int kTaskCols = 256;        // columns per column task (one per thread)
// Column-forward task, R <= 16: thread = one column of one operand.
template <int R>
__device__ __forceinline__ void colf_regs(const uint64_t* src, uint64_t* dst,
                                          const TwPair* __restrict__ twf, const LimbConst& K) {
  uint64_t x[R];
#pragma unroll
  for (int t = 0; t < R; t++) x[t] = __ldcg(src + (size_t)t * kRow);
  ct_col<R>(x, twf, K.q, K.two_q);
#pragma unroll
  for (int t = 0; t < R; t++) dst[(size_t)t * kRow] = x[t];
}

// Column-forward task, R = 32: the column is parked in smem (stride 256,
// private to the thread) between the first stage (pairs t, t+16) and the
// radix-16 groups of the two halves (stages 1..4, block index = half).
__device__ __forceinline__ void colf_32(const uint64_t* src, uint64_t* dst, uint64_t* sm,
                                        const TwPair* __restrict__ twf, const LimbConst& K) {
  const int th = threadIdx.x;
  const TwPair w = ld_tw(twf + 1);
#pragma unroll 1
  for (int b = 0; b < 2; b++) {
    uint64_t lo[8], hi[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      lo[i] = __ldcg(src + (size_t)(8 * b + i) * kRow);
      hi[i] = __ldcg(src + (size_t)(8 * b + i + 16) * kRow);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
      ct_bfly(lo[i], hi[i], w.w, w.wp, K.q, K.two_q);
      sm[(8 * b + i) * kTaskCols + th] = lo[i];
      sm[(8 * b + i + 16) * kTaskCols + th] = hi[i];
    }
  }
#pragma unroll 1
  for (int h = 0; h < 2; h++) {
    uint64_t v[16];
#pragma unroll
    for (int u = 0; u < 16; u++) v[u] = sm[(16 * h + u) * kTaskCols + th];
    ct16(v, twf, 1, h, K.q, K.two_q);
#pragma unroll
    for (int u = 0; u < 16; u++) dst[(size_t)(16 * h + u) * kRow] = v[u];
  }
}

// Column-inverse task, R <= 16: thread = one column of c'.
template <int R, bool HALVE>
__device__ __forceinline__ void coli_regs(uint64_t* p, const TwPair* __restrict__ twi,
                                          const LimbConst& K) {
  uint64_t x[R];
#pragma unroll
  for (int t = 0; t < R; t++) x[t] = __ldcg(p + (size_t)t * kRow);
  gs_col<R, HALVE>(x, twi, K);
#pragma unroll
  for (int t = 0; t < R; t++) __stcs(p + (size_t)t * kRow, csub(x[t], K.q));
}

// Column-inverse task, R = 32: radix-16 GS groups on the two halves (GS
// stages with k = 4096 * 2^e, e = 0..3, viewed as a 32-point transform), then
// the last stage (pairs t, t+16, twiddle Psi^-1_br[1]) and the reduction.
template <bool HALVE>
__device__ __forceinline__ void coli_32(uint64_t* p, uint64_t* sm, const TwPair* __restrict__ twi,
                                        const LimbConst& K) {
  const int th = threadIdx.x;
#pragma unroll 1
  for (int h = 0; h < 2; h++) {
    uint64_t v[16];
#pragma unroll
    for (int u = 0; u < 16; u++) v[u] = __ldcg(p + (size_t)(16 * h + u) * kRow);
    gs16<HALVE>(v, twi, 5, 0, h, K.q, K.two_q, K.half_q1);
#pragma unroll
    for (int u = 0; u < 16; u++) sm[(16 * h + u) * kTaskCols + th] = v[u];
  }
  const TwPair w = ld_tw(twi + 1);
#pragma unroll 1
  for (int b = 0; b < 2; b++) {
#pragma unroll
    for (int i = 0; i < 8; i++) {
      uint64_t x0 = sm[(8 * b + i) * kTaskCols + th], x1 = sm[(8 * b + i + 16) * kTaskCols + th];
      if constexpr (HALVE)
        gs_bfly_half(x0, x1, w.w, w.wp, K.q, K.two_q, K.half_q1);
      else
        gs_bfly_last(x0, x1, K);
      __stcs(p + (size_t)(8 * b + i) * kRow, csub(x0, K.q));
      __stcs(p + (size_t)(8 * b + i + 16) * kRow, csub(x1, K.q));
    }
  }
}

template <int R, bool HALVE>
__device__ void run_task(const KParams& P, const PersistArgs& A, uint32_t ticket, uint64_t* smem) {
  const uint32_t logn = P.logn;
  const uint32_t GS = A.F + A.W + A.I;
  const uint32_t g = ticket / GS;
  uint32_t r = ticket - g * GS;
  uint32_t* done = A.ctl + 4;  // [unit][2]: column-forward tasks done, rows done
  int* err = reinterpret_cast<int*>(A.ctl + 1);
  if (r < A.F) {  // ---- column forward, unit g
    const uint32_t unit = g;
    if (unit >= P.nunits) return;
    const uint32_t op = r / (kRow / kTaskCols), cs = r % (kRow / kTaskCols);
    const uint32_t limb = unit % P.nlimbs;
    const LimbConst K = ld_limb(P.lc + limb);
    const TwPair* twf = P.twf + ((size_t)limb << logn);
    const size_t off = ((size_t)unit << logn) + cs * kTaskCols + threadIdx.x;
    const uint64_t* src = (op == 0 ? P.a : P.b) + off;
    uint64_t* dst = (op == 0 ? P.c : P.s) + off;
    if constexpr (R == 32)
      colf_32(src, dst, smem, twf, K);
    else
      colf_regs<R>(src, dst, twf, K);
    cta_signal(done + 2 * unit);
    return;
  }
  r -= A.F;
  if (r < A.W) {  // ---- row r of unit g - lagF
    if (g < A.lagF || g - A.lagF >= P.nunits) return;
    const uint32_t unit = g - A.lagF;
    if (A.F) cta_wait(done + 2 * unit, A.F + A.withheld, err);
    const uint32_t limb = unit % P.nlimbs;
    const LimbConst K = ld_limb(P.lc + limb);
    const TwPair* twf = P.twf + ((size_t)limb << logn);
    const TwPair* twi = P.twi + ((size_t)limb << logn);
    const size_t off = ((size_t)unit << logn) + (size_t)r * kRow;
    const bool single = (logn == kRowLog);
    row_task_polymul<HALVE, true>((single ? P.a : P.c) + off, (single ? P.b : P.s) + off,
                                  P.c + off, single, smem, twf, twi, K, logn, r, P.fused != 0);
    if (A.I) cta_signal(done + 2 * unit + 1);
    return;
  }
  r -= A.W;
  // ---- column inverse, unit g - lagI
  if (g < A.lagI || g - A.lagI >= P.nunits) return;
  const uint32_t unit = g - A.lagI;
  cta_wait(done + 2 * unit + 1, A.W, err);
  const uint32_t limb = unit % P.nlimbs;
  const LimbConst K = ld_limb(P.lc + limb);
  const TwPair* twi = P.twi + ((size_t)limb << logn);
  uint64_t* p = P.c + ((size_t)unit << logn) + r * kTaskCols + threadIdx.x;
  if constexpr (R == 32)
    coli_32<HALVE>(p, smem, twi, K);
  else
    coli_regs<R, HALVE>(p, twi, K);
}

}  // namespace

template <int R, bool HALVE>
__global__ void __launch_bounds__(256, 3) k_persist(KParams P, PersistArgs A) {
  extern __shared__ __align__(16) uint64_t smem[];
  __shared__ uint32_t s_ticket;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(A.ctl, 1u);
    __syncthreads();
    const uint32_t ticket = s_ticket;
    __syncthreads();  // everyone has read s_ticket before thread 0 rewrites it
    if (ticket >= A.ntasks) break;
    run_task<R, HALVE>(P, A, ticket, smem);
    __syncthreads();  // smem reuse by the next task
  }
}

namespace {

constexpr int kPersistSmem = 2 * kRowPad * 8;

template <int R>
cudaError_t launch_r(const KParams& P, const PersistArgs& A, int grid, cudaStream_t st) {
  if (P.halving)
    k_persist<R, true><<<grid, 256, kPersistSmem, st>>>(P, A);
  else
    k_persist<R, false><<<grid, 256, kPersistSmem, st>>>(P, A);
  return cudaGetLastError();
}

template <int R, bool H>
cudaError_t set_attr() {
  return cudaFuncSetAttribute((const void*)k_persist<R, H>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
}

}  // namespace

cudaError_t persist_prepare() {
  cudaError_t e = cudaSuccess;
  if ((e = set_attr<1, false>()) || (e = set_attr<1, true>()) || (e = set_attr<2, false>()) ||
      (e = set_attr<2, true>()) || (e = set_attr<4, false>()) || (e = set_attr<4, true>()) ||
      (e = set_attr<8, false>()) || (e = set_attr<8, true>()) || (e = set_attr<16, false>()) ||
      (e = set_attr<16, true>()) || (e = set_attr<32, false>()) || (e = set_attr<32, true>()))
    return e;
  return cudaSuccess;
}

size_t persist_ctl_words(uint32_t nunits) { return 4 + 2 * (size_t)nunits; }

// Launch the persistent polymul for N >= 4096.  `ctl` is a zeroed control
// block of persist_ctl_words(nunits) words.  P.a/P.b/P.c/P.s follow the same
// aliasing rules as the column-split path (see launch_polymul).
cudaError_t launch_polymul_persistent(const KParams& P0, uint32_t* ctl, int grid, uint32_t lagF,
                                      uint32_t lagI, cudaStream_t st, uint32_t withheld) {
  if (P0.nunits == 0) return cudaSuccess;
  if (P0.logn < 12 || P0.logn > 17) return cudaErrorInvalidValue;
  KParams P = P0;
  if (P.fused) P.lc += P.nlimbs;  // Algorithm 8: the fused constants (2/N)
  int nops = 2;
  if (P.logn > 12) {
    if (P.a == P.b) {
      P.b = nullptr;
      P.s = P.c;
      nops = 1;
    } else if (P.c == P.b) {
      const uint64_t* t = P.a;
      P.a = P.b;
      P.b = t;
    }
  }
  PersistArgs A{};
  A.ctl = ctl;
  const uint32_t R = 1u << (P.logn - kRowLog);
  A.F = (P.logn > 12) ? (uint32_t)nops * (kRow / kTaskCols) : 0;
  A.W = R;
  A.I = (P.logn > 12) ? (kRow / kTaskCols) : 0;
  A.lagF = A.F ? lagF : 0;
  A.lagI = A.I ? (lagI > A.lagF ? lagI : A.lagF + 1) : A.lagF;
  A.ntasks = (P.nunits + A.lagI) * (A.F + A.W + A.I);
  A.withheld = A.F ? withheld : 0;
  cudaError_t e = cudaMemsetAsync(ctl, 0, persist_ctl_words(P.nunits) * 4, st);
  if (e != cudaSuccess) return e;
  switch (R) {
    case 1: return launch_r<1>(P, A, grid, st);
    case 2: return launch_r<2>(P, A, grid, st);
    case 4: return launch_r<4>(P, A, grid, st);
    case 8: return launch_r<8>(P, A, grid, st);
    case 16: return launch_r<16>(P, A, grid, st);
    case 32: return launch_r<32>(P, A, grid, st);
  }
  return cudaErrorInvalidValue;
}


// --------------------------------------------------------------------------
// Uneven batch: products of different N and limb counts in one launch.
//
// Every (job, polynomial, limb) is a unit with its own descriptor (pointers,
// plan tables, log2 N).  The tickets are laid out in three sections -- all
// column-forward tasks, then all row tasks, then all column-inverse tasks,
// each ordered by unit -- and decoded with a binary search over per-unit
// prefix counts.  Dependencies and bounded waits are the same as above.
// N = 4096 units have only a row task; N <= 2048 is not handled here (the
// host routes such jobs to the per-plan path).

namespace {

__device__ __forceinline__ uint32_t find_unit(const uint32_t* __restrict__ pre, uint32_t n,
                                              uint32_t x) {
  // largest u with pre[u] <= x, pre[0] = 0, pre non-decreasing, n >= 1
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <bool HALVE, bool FUSED>
__device__ void run_uneven_task(const UnevenArgs& A, uint32_t ticket, uint64_t* smem) {
  uint32_t* done = A.ctl + 4;
  int* err = reinterpret_cast<int*>(A.ctl + 1);
  const uint32_t U = A.nunits;
  uint32_t section, base;
  const uint32_t* pre;
  if (ticket < A.tf) {
    section = 0; base = 0; pre = A.pre_f;
  } else if (ticket < A.tf + A.tw) {
    section = 1; base = A.tf; pre = A.pre_w;
  } else {
    section = 2; base = A.tf + A.tw; pre = A.pre_i;
  }
  __shared__ uint32_t s_unit;
  if (threadIdx.x == 0) s_unit = find_unit(pre, U, ticket - base);
  __syncthreads();
  const uint32_t unit = s_unit;
  __syncthreads();
  const UnitDesc D = A.units[unit];
  const uint32_t r = ticket - base - __ldg(pre + unit);
  const uint32_t logn = D.logn;
  const uint32_t R = 1u << (logn - kRowLog);
  const LimbConst K = ld_limb(D.lc);
  if (section == 0) {
    const uint32_t op = r / (kRow / kTaskCols), cs = r % (kRow / kTaskCols);
    const size_t off = cs * kTaskCols + threadIdx.x;
    const uint64_t* src = (op == 0 ? D.a : D.b) + off;
    uint64_t* dst = (op == 0 ? D.c : D.s) + off;
    switch (R) {
      case 2: colf_regs<2>(src, dst, D.twf, K); break;
      case 4: colf_regs<4>(src, dst, D.twf, K); break;
      case 8: colf_regs<8>(src, dst, D.twf, K); break;
      case 16: colf_regs<16>(src, dst, D.twf, K); break;
      default: colf_32(src, dst, smem, D.twf, K); break;
    }
    cta_signal(done + 2 * unit);
  } else if (section == 1) {
    const uint32_t nf = (logn > kRowLog) ? ((D.a == D.b ? 1u : 2u) * (kRow / kTaskCols)) : 0u;
    if (nf) cta_wait(done + 2 * unit, nf, err);
    const size_t off = (size_t)r * kRow;
    const bool single = (logn == kRowLog);
    row_task_polymul<HALVE, true>((single ? D.a : D.c) + off, (single ? D.b : D.s) + off,
                                  D.c + off, single, smem, D.twf, D.twi, K, logn, r, FUSED);
    if (!single) cta_signal(done + 2 * unit + 1);
  } else {
    cta_wait(done + 2 * unit + 1, R, err);
    uint64_t* p = D.c + r * kTaskCols + threadIdx.x;
    switch (R) {
      case 2: coli_regs<2, HALVE>(p, D.twi, K); break;
      case 4: coli_regs<4, HALVE>(p, D.twi, K); break;
      case 8: coli_regs<8, HALVE>(p, D.twi, K); break;
      case 16: coli_regs<16, HALVE>(p, D.twi, K); break;
      default: coli_32<HALVE>(p, smem, D.twi, K); break;
    }
  }
}

}  // namespace

// FUSED: every unit's plan has PM_PLAN_FUSED (Algorithm 8 row tasks).  A
// compile-time choice: with a run-time flag the row task's two product
// steps raise the kernel's register spills several-fold.
template <bool HALVE, bool FUSED>
__global__ void __launch_bounds__(256, 3) k_uneven(UnevenArgs A) {
  extern __shared__ __align__(16) uint64_t smem[];
  __shared__ uint32_t s_ticket;
  const uint32_t total = A.tf + A.tw + A.ti;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(A.ctl, 1u);
    __syncthreads();
    const uint32_t ticket = s_ticket;
    __syncthreads();
    if (ticket >= total) break;
    run_uneven_task<HALVE, FUSED>(A, ticket, smem);
    __syncthreads();
  }
}

cudaError_t uneven_prepare() {
  const void* fns[4] = {(const void*)k_uneven<false, false>, (const void*)k_uneven<true, false>,
                        (const void*)k_uneven<false, true>, (const void*)k_uneven<true, true>};
  for (const void* f : fns) {
    cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_uneven(const UnevenArgs& A, bool halving, bool fused, int grid,
                          cudaStream_t st) {
  if (A.nunits == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(A.ctl, 0, (4 + 2 * (size_t)A.nunits) * 4, st);
  if (e != cudaSuccess) return e;
  if (halving) {
    if (fused)
      k_uneven<true, true><<<grid, 256, kPersistSmem, st>>>(A);
    else
      k_uneven<true, false><<<grid, 256, kPersistSmem, st>>>(A);
  } else {
    if (fused)
      k_uneven<false, true><<<grid, 256, kPersistSmem, st>>>(A);
    else
      k_uneven<false, false><<<grid, 256, kPersistSmem, st>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace pm
