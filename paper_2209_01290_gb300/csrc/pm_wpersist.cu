// pm_wpersist.cu -- one persistent launch for a whole batch of negacyclic
// products built on the 1024-word split (arxiv 2209.01290, Eq. 2; batched
// like the paper's throughput-oriented TOM-NTT, Sec. V-C).
//
// The split has three kinds of task per unit (N = 2^(10+CL)):
//   F column-forward tasks: CT = 256 / J columns of one operand each, the
//     first CL stages of Algorithm 6 (w_colf_task);
//   W = 2^CL row tasks: the 10 in-row forward stages of a and b, the
//     pointwise product (Algorithm 4, or Algorithm 8's pair step), the 10
//     in-row inverse stages (w_row_task);
//   I column-inverse tasks: the last CL stages of Algorithm 7, the 1/N fold
//     and the reduction to [0, q) (w_coli_task).
// A grid of 4 CTAs per SM stays resident and takes tickets from a global
// counter.  k_wpersist (units of one N): ticket group g holds the
// column-forward tasks of unit g, the row tasks of unit g - lagF and the
// column-inverse tasks of unit g - lagI, so the memory-heavier column work
// of some units runs beside the row work of others and each unit's images
// are read back while they are still in L2.  k_wuneven (units of different
// N, from descriptors): three sections, all column-forward tasks, then all
// row tasks, then all column-inverse tasks, each in unit order.
//
// A row task waits until every column-forward task of its unit is done, a
// column-inverse task until every row of its unit is done (per-unit
// counters, pm_sync.cuh).  A task only waits for tasks with smaller tickets,
// which running CTAs took, so every wait ends; each wait is still bounded
// (about a second) and a CTA that gives up records PM_ERR_TIMEOUT in the
// control block.  The row tasks stage their twiddles with bulk copies on
// the CTA's mbarrier, one phase per row task.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pm_internal.h"
#include "pm_sync.cuh"
#include "pm_wide.cuh"

namespace pm {
namespace {

// Column tasks hold at most 8 words per thread for N <= 2^16, so that a
// task of any kind fits 64 registers and 4 CTAs (50 KB of shared memory
// each) stay resident per SM; N = 2^17 columns (128 words) take 16 words per
// thread and 3 CTAs per SM.
template <int CL>
constexpr int kWpMW = CL <= 6 ? 8 : 16;
template <int CL>
constexpr int kWpCtas = CL <= 6 ? 4 : 3;

// Column tasks keep their transpose buffer (at most 128 x 32 words) in the
// shared memory from the inverse twiddle slices on; the forward slices'
// unused last entry, the mbarrier, stays untouched.
__device__ __forceinline__ uint64_t* wp_tile(uint64_t* smem) {
  return reinterpret_cast<uint64_t*>(reinterpret_cast<TwPair*>(smem) + kWTw);
}

template <int CL>
constexpr bool kWpTileFits = WCol<CL, kWThreads, kWpMW<CL>>::kSmemWords * 8 <=
                             kWRowsSmem<uint64_t> - kWTw * (int)sizeof(TwPair);

template <int CL, int MODE, bool LZ>
__global__ void __launch_bounds__(kWThreads, kWpCtas<CL>) k_wpersist(KParams P, PersistArgs A) {
  using S = WCol<CL, kWThreads, kWpMW<CL>>;
  static_assert(kWpTileFits<CL>, "column transpose buffer exceeds the task's shared memory");
  extern __shared__ __align__(16) uint64_t smem[];
  __shared__ uint32_t s_ticket;
  uint32_t* done = A.ctl + 4;  // [unit][2]: column-forward tasks done, rows done
  int* err = reinterpret_cast<int*>(A.ctl + 1);
  if (threadIdx.x == 0) mbar_init1(w_row_bar<uint64_t>(smem));
  __syncthreads();
  uint32_t phase = 0;
  // Tickets are taken one at a time: fetching the next one during a task
  // (as k_wuneven does) was measured slower here -- an unstarted column task
  // held by a busy CTA delays the rows that wait for it (C3 at lags 8/32:
  // 104 vs 87 us).
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(A.ctl, 1u);
    __syncthreads();
    const uint32_t ticket = s_ticket;
    __syncthreads();  // everyone has read s_ticket before thread 0 rewrites it
    if (ticket >= A.ntasks) break;
    // the ticket's segment, group and task within the group (no empty tickets)
    uint32_t k = 0;
    while (k + 1 < A.nseg && ticket >= A.seg_t[k + 1]) ++k;
    const uint32_t mask = A.seg_mask[k];
    const uint32_t gs = ((mask & 1) ? A.F : 0u) + ((mask & 2) ? A.W : 0u) + ((mask & 4) ? A.I : 0u);
    const uint32_t off = ticket - A.seg_t[k];
    const uint32_t g = A.seg_g[k] + off / gs;
    uint32_t r = off % gs;
    uint32_t kind = 0;  // 0: column forward, 1: row, 2: column inverse
    if (!((mask & 1) && r < A.F)) {
      if (mask & 1) r -= A.F;
      if ((mask & 2) && r < A.W) {
        kind = 1;
      } else {
        if (mask & 2) r -= A.W;
        kind = 2;
      }
    }
    bool stop = false;
    if (kind == 0) {  // ---- column forward, unit g
      w_colf_task<CL, uint64_t, false, LZ, kWThreads, kWpMW<CL>>(P, g, r / S::kTiles,
                                                                  r % S::kTiles, wp_tile(smem));
      cta_signal(done + 2 * g);
    } else if (kind == 1) {  // ---- row r of unit g - lagF
      const uint32_t unit = g - A.lagF;
      cta_wait(done + 2 * unit, A.F + A.withheld, err);
      stop = !w_row_task<MODE, false, uint64_t, false, LZ>(P, unit, r, smem, phase);
      phase ^= 1u;
      cta_signal(done + 2 * unit + 1);
    } else {  // ---- column inverse r of unit g - lagI
      const uint32_t unit = g - A.lagI;
      cta_wait(done + 2 * unit + 1, A.W, err);
      w_coli_task<CL, false, uint64_t, false, LZ, kWThreads, kWpMW<CL>>(P, unit, r,
                                                                        wp_tile(smem));
    }
    // a row task whose copies never completed leaves the barrier's phase
    // unknown: this CTA stops taking tickets (the others finish the queue)
    if (stop) break;
    __syncthreads();  // shared memory is reused by the next task
  }
}

// ------------------------------------------------------------ uneven batch
// Tasks per unit of the 1024-word split with 256-thread column tasks.
__host__ __device__ constexpr uint32_t wp_tiles(uint32_t cl) {
  // kW / CT = 4 J with J = R / MW threads per column (MW = 8, or 16 at 2^17)
  return cl == 7 ? 32u : cl > 3 ? 4u << (cl - 3) : 4u;
}

template <bool LZ>
__device__ __forceinline__ void wu_colf(const KParams& P, uint32_t cl, uint32_t unit,
                                        uint32_t op, uint32_t tile, uint64_t* sm) {
  switch (cl) {
    case 2: w_colf_task<2, uint64_t, true, LZ, kWThreads, kWpMW<2>>(P, unit, op, tile, sm); break;
    case 3: w_colf_task<3, uint64_t, true, LZ, kWThreads, kWpMW<3>>(P, unit, op, tile, sm); break;
    case 4: w_colf_task<4, uint64_t, true, LZ, kWThreads, kWpMW<4>>(P, unit, op, tile, sm); break;
    case 5: w_colf_task<5, uint64_t, true, LZ, kWThreads, kWpMW<5>>(P, unit, op, tile, sm); break;
    case 6: w_colf_task<6, uint64_t, true, LZ, kWThreads, kWpMW<6>>(P, unit, op, tile, sm); break;
    default: w_colf_task<7, uint64_t, true, LZ, kWThreads, kWpMW<7>>(P, unit, op, tile, sm); break;
  }
}

template <bool LZ>
__device__ __forceinline__ void wu_coli(const KParams& P, uint32_t cl, uint32_t unit,
                                        uint32_t tile, uint64_t* sm) {
  switch (cl) {
    case 2: w_coli_task<2, false, uint64_t, true, LZ, kWThreads, kWpMW<2>>(P, unit, tile, sm); break;
    case 3: w_coli_task<3, false, uint64_t, true, LZ, kWThreads, kWpMW<3>>(P, unit, tile, sm); break;
    case 4: w_coli_task<4, false, uint64_t, true, LZ, kWThreads, kWpMW<4>>(P, unit, tile, sm); break;
    case 5: w_coli_task<5, false, uint64_t, true, LZ, kWThreads, kWpMW<5>>(P, unit, tile, sm); break;
    case 6: w_coli_task<6, false, uint64_t, true, LZ, kWThreads, kWpMW<6>>(P, unit, tile, sm); break;
    default: w_coli_task<7, false, uint64_t, true, LZ, kWThreads, kWpMW<7>>(P, unit, tile, sm); break;
  }
}

// Units of N = 2^12 .. 2^17 (descriptors in P.desc, A.units == P.desc).
template <int MODE, bool LZ>
__global__ void __launch_bounds__(kWThreads, kWpCtas<7>) k_wuneven(KParams P, UnevenArgs A) {
  static_assert(kWpTileFits<7>, "column transpose buffer exceeds the task's shared memory");
  extern __shared__ __align__(16) uint64_t smem[];
  __shared__ uint32_t s_ticket, s_unit;
  uint32_t* done = A.ctl + 4;
  int* err = reinterpret_cast<int*>(A.ctl + 1);
  const uint32_t total = A.tf + A.tw + A.ti;
  // thread 0: the unit of ticket t (the block table's unit, then a forward
  // scan of the section's prefix counts)
  auto unit_of = [&](uint32_t t) {
    const uint32_t sec = t < A.tf ? 0u : t < A.tf + A.tw ? 1u : 2u;
    const uint32_t* pre = sec == 0 ? A.pre_f : sec == 1 ? A.pre_w : A.pre_i;
    const uint32_t* blk = sec == 0 ? A.blk_f : sec == 1 ? A.blk_w : A.blk_i;
    const uint32_t x = t - (sec == 0 ? 0u : sec == 1 ? A.tf : A.tf + A.tw);
    uint32_t u = __ldg(blk + (x >> 5));
    while (u + 1 < A.nunits && __ldg(pre + u + 1) <= x) ++u;
    return u;
  };
  if (threadIdx.x == 0) {
    mbar_init1(w_row_bar<uint64_t>(smem));
    const uint32_t t = atomicAdd(A.ctl, 1u);
    s_ticket = t;
    s_unit = t < total ? unit_of(t) : 0u;
  }
  __syncthreads();
  uint32_t ticket = s_ticket, unit = s_unit;
  uint32_t phase = 0;
  for (;;) {
    __syncthreads();  // everyone has read s_ticket / s_unit
    if (ticket >= total) break;
    // the next ticket is taken now (its latency overlaps the task) and its
    // unit looked up after the task.  Holding one unstarted ticket is safe:
    // every task waits only for smaller tickets, and the smallest unfinished
    // ticket is always one a CTA is running.  (C4: 23.2 -> 22.8 ms.)
    uint32_t next = 0;
    if (threadIdx.x == 0) next = atomicAdd(A.ctl, 1u);
    const uint32_t cl = __ldg(&A.units[unit].logn) - kWLog;
    bool stop = false;
    if (ticket < A.tf) {
      const uint32_t r = ticket - __ldg(A.pre_f + unit);
      const uint32_t nt = wp_tiles(cl);
      wu_colf<LZ>(P, cl, unit, r / nt, r % nt, wp_tile(smem));
      cta_signal(done + 2 * unit);
    } else if (ticket < A.tf + A.tw) {
      const uint32_t r = ticket - A.tf - __ldg(A.pre_w + unit);
      const UnitDesc& D = A.units[unit];
      const uint32_t nf = (D.a == D.b ? 1u : 2u) * wp_tiles(cl);
      cta_wait(done + 2 * unit, nf, err);
      stop = !w_row_task<MODE, false, uint64_t, true, LZ>(P, unit, r, smem, phase);
      phase ^= 1u;
      cta_signal(done + 2 * unit + 1);
    } else {
      const uint32_t r = ticket - A.tf - A.tw - __ldg(A.pre_i + unit);
      cta_wait(done + 2 * unit + 1, 1u << cl, err);
      wu_coli<LZ>(P, cl, unit, r, wp_tile(smem));
    }
    if (stop) break;
    if (threadIdx.x == 0) {
      s_ticket = next;
      s_unit = next < total ? unit_of(next) : 0u;
    }
    __syncthreads();
    ticket = s_ticket;
    unit = s_unit;
  }
}

template <int CL, int MODE, bool LZ>
cudaError_t wp_launch(const KParams& P, const PersistArgs& A, int grid, cudaStream_t st) {
  k_wpersist<CL, MODE, LZ><<<grid, kWThreads, kWRowsSmem<uint64_t>, st>>>(P, A);
  return cudaGetLastError();
}

template <int CL>
cudaError_t wp_launch_cl(const KParams& P, const PersistArgs& A, int grid, cudaStream_t st) {
  if (P.fused)
    return P.lazy16 ? wp_launch<CL, MODE_POLYMUL_FUSED, true>(P, A, grid, st)
                    : wp_launch<CL, MODE_POLYMUL_FUSED, false>(P, A, grid, st);
  return P.lazy16 ? wp_launch<CL, MODE_POLYMUL, true>(P, A, grid, st)
                  : wp_launch<CL, MODE_POLYMUL, false>(P, A, grid, st);
}

template <int CL, int MODE, bool LZ>
cudaError_t wp_attr() {
  return cudaFuncSetAttribute((const void*)k_wpersist<CL, MODE, LZ>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kWRowsSmem<uint64_t>);
}

template <int CL>
cudaError_t wp_attr_cl() {
  cudaError_t e;
  if ((e = wp_attr<CL, MODE_POLYMUL, false>()) != cudaSuccess ||
      (e = wp_attr<CL, MODE_POLYMUL, true>()) != cudaSuccess ||
      (e = wp_attr<CL, MODE_POLYMUL_FUSED, false>()) != cudaSuccess ||
      (e = wp_attr<CL, MODE_POLYMUL_FUSED, true>()) != cudaSuccess)
    return e;
  return cudaSuccess;
}

}  // namespace

bool wpersist_ok(uint32_t logn) { return logn >= 13 && logn <= 17; }

int wpersist_ctas_per_sm(uint32_t logn) {
  return logn == 0 ? kWpCtas<7> : logn <= kWLog + 6 ? kWpCtas<6> : kWpCtas<7>;
}

uint32_t wuneven_tasks(uint32_t logn, bool square, uint32_t* f, uint32_t* w, uint32_t* i) {
  const uint32_t cl = logn - kWLog;
  *f = (square ? 1u : 2u) * wp_tiles(cl);
  *w = 1u << cl;
  *i = wp_tiles(cl);
  return *f + *w + *i;
}

cudaError_t wpersist_prepare() {
  cudaError_t e;
  if ((e = wp_attr_cl<3>()) != cudaSuccess || (e = wp_attr_cl<4>()) != cudaSuccess ||
      (e = wp_attr_cl<5>()) != cudaSuccess || (e = wp_attr_cl<6>()) != cudaSuccess ||
      (e = wp_attr_cl<7>()) != cudaSuccess)
    return e;
  const void* fns[] = {(const void*)k_wuneven<MODE_POLYMUL, false>,
                       (const void*)k_wuneven<MODE_POLYMUL, true>,
                       (const void*)k_wuneven<MODE_POLYMUL_FUSED, false>,
                       (const void*)k_wuneven<MODE_POLYMUL_FUSED, true>};
  for (const void* f : fns) {
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kWRowsSmem<uint64_t>)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// One persistent launch of a uniform batch through the 1024-word split,
// N = 2^13 .. 2^17, 64-bit words, 1/N folded.  `ctl` is a control block of
// persist_ctl_words(nunits) words (zeroed here).  Aliasing as in the split.
cudaError_t launch_polymul_wpersistent(const KParams& P0, uint32_t* ctl, int grid,
                                       uint32_t lagF, uint32_t lagI, cudaStream_t st,
                                       uint32_t withheld) {
  if (P0.nunits == 0) return cudaSuccess;
  if (!wpersist_ok(P0.logn) || P0.word32 || P0.halving) return cudaErrorInvalidValue;
  KParams P = P0;
  if (P.fused) P.lc += P.nlimbs;  // Algorithm 8: the fused constants (2/N)
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
  const uint32_t cl = P.logn - kWLog;
  PersistArgs A{};
  A.ctl = ctl;
  A.F = (uint32_t)nops * wp_tiles(cl);
  A.W = 1u << cl;
  A.I = wp_tiles(cl);
  A.lagF = lagF;
  A.lagI = lagI > lagF ? lagI : lagF + 1;
  A.withheld = withheld;
  // segments of groups with the same set of tasks: breakpoints at lagF,
  // lagI, U, U + lagF (U + lagI ends the last one)
  const uint32_t U = P.nunits, G = U + A.lagI;
  uint32_t bp[6] = {0, A.lagF, A.lagI, U, U + A.lagF, G};
  std::sort(bp, bp + 6);
  uint32_t t = 0;
  A.nseg = 0;
  for (int k = 0; k < 5; ++k) {
    const uint32_t g0 = bp[k], g1 = bp[k + 1];
    if (g1 <= g0 || g0 >= G) continue;
    const uint32_t mask = (g0 < U ? 1u : 0u) | (g0 >= A.lagF && g0 < U + A.lagF ? 2u : 0u) |
                          (g0 >= A.lagI && g0 < U + A.lagI ? 4u : 0u);
    const uint32_t gs = ((mask & 1) ? A.F : 0u) + ((mask & 2) ? A.W : 0u) + ((mask & 4) ? A.I : 0u);
    if (gs == 0) continue;
    A.seg_g[A.nseg] = g0;
    A.seg_t[A.nseg] = t;
    A.seg_mask[A.nseg] = mask;
    ++A.nseg;
    t += (g1 - g0) * gs;
  }
  A.ntasks = t;
  cudaError_t e = cudaMemsetAsync(ctl, 0, persist_ctl_words(P.nunits) * 4, st);
  if (e != cudaSuccess) return e;
  switch (cl) {
    case 3: return wp_launch_cl<3>(P, A, grid, st);
    case 4: return wp_launch_cl<4>(P, A, grid, st);
    case 5: return wp_launch_cl<5>(P, A, grid, st);
    case 6: return wp_launch_cl<6>(P, A, grid, st);
    case 7: return wp_launch_cl<7>(P, A, grid, st);
  }
  return cudaErrorInvalidValue;
}

// One launch of an uneven batch through the 1024-word split: units of
// N = 2^12 .. 2^17 from A.units (64-bit words, 1/N folded), prefix counts
// from wuneven_tasks.  `lazy16`: every unit's q < 2^60; `fused`: every
// unit's plan is an Algorithm 8 plan (its descriptor's constants are the
// fused ones).
cudaError_t launch_wuneven(const UnevenArgs& A, bool lazy16, bool fused, int grid,
                           cudaStream_t st) {
  if (A.nunits == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(A.ctl, 0, (4 + 2 * (size_t)A.nunits) * 4, st);
  if (e != cudaSuccess) return e;
  KParams P{};
  P.desc = A.units;
  P.nunits = A.nunits;
  P.err = reinterpret_cast<int*>(A.ctl + 1);
  const size_t smem = kWRowsSmem<uint64_t>;
  if (fused) {
    if (lazy16)
      k_wuneven<MODE_POLYMUL_FUSED, true><<<grid, kWThreads, smem, st>>>(P, A);
    else
      k_wuneven<MODE_POLYMUL_FUSED, false><<<grid, kWThreads, smem, st>>>(P, A);
  } else {
    if (lazy16)
      k_wuneven<MODE_POLYMUL, true><<<grid, kWThreads, smem, st>>>(P, A);
    else
      k_wuneven<MODE_POLYMUL, false><<<grid, kWThreads, smem, st>>>(P, A);
  }
  return cudaGetLastError();
}

}  // namespace pm
