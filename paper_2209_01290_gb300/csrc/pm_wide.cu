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

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime)

#include "pm_wide.cuh"

namespace pm {
namespace {

// One row task per CTA.
template <int MODE, bool HALVE, typename W, bool DESC = false, bool LZ = false>
__global__ void __launch_bounds__(kWThreads, 4) k_wrows(KParams P) {
  extern __shared__ __align__(16) uint64_t smem_raw[];
  pdl_trigger();
  const uint32_t cl = P.logn - kWLog;
  const uint32_t unit = blockIdx.x >> cl;
  if (unit >= P.nunits) return;  // whole CTA exits together
  if constexpr (sizeof(W) == 8) {
    if (threadIdx.x == 0) mbar_init1(w_row_bar<W>(smem_raw));
    __syncthreads();
  }
  w_row_task<MODE, HALVE, W, DESC, LZ>(P, unit, blockIdx.x & ((1u << cl) - 1), smem_raw, 0);
}

// Forward column stages: CTA = (unit, operand, tile of CT columns); operand 0
// (a) goes to c, operand 1 (b) to the scratch s.  Every word of a column is
// read (before the barrier) and written (after it) by the CTA that owns the
// column, so c may alias a.
template <int CL, typename W, bool DESC = false, bool LZ = false>
__global__ void __launch_bounds__(kWColThreads) k_wcol_fwd(KParams P, int nops) {
  using S = WCol<CL>;
  __shared__ W tile_s[S::kSmemWords];
  pdl_trigger();
  const uint32_t tile = blockIdx.x % S::kTiles;
  const uint32_t rest = blockIdx.x / S::kTiles;
  const uint32_t op = rest % (uint32_t)nops, unit = rest / (uint32_t)nops;
  if (unit >= P.nunits) return;
  w_colf_task<CL, W, DESC, LZ>(P, unit, op, tile, tile_s);
}

// Inverse column stages and the reduction, in place on c.
template <int CL, bool HALVE, typename W, bool DESC = false, bool LZ = false>
__global__ void __launch_bounds__(kWColThreads) k_wcol_inv(KParams P) {
  using S = WCol<CL>;
  __shared__ W tile_s[S::kSmemWords];
  if (P.pdl) pdl_wait();  // c is the row kernel's output
  const uint32_t tile = blockIdx.x % S::kTiles;
  const uint32_t unit = blockIdx.x / S::kTiles;
  if (unit >= P.nunits) return;
  w_coli_task<CL, HALVE, W, DESC, LZ>(P, unit, tile, tile_s);
}

// ------------------------------------------------- tensor-copy column tiles
// The same column stages with the CTA's tile -- R rows x CT columns of the
// unit's [R][1024] image -- loaded by one 2-D tensor copy (TMA) into shared
// memory instead of 16 strided loads per thread; the inverse kernel also
// writes its tile back with one 2-D tensor copy.  64-bit words, 1/N folded.
// The tensor maps view an operand array as a 2-D tensor of nunits R rows of
// 1024 words (row stride 8 KB) with a box of CT x R words; tile x of unit u
// is the box at (x CT, u R).  The mbarrier wait is bounded like the row
// kernel's (P.err on giving up).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n\t"
      "cp.async.bulk.commit_group;" ::"l"(map),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}

// One thread: load the CTA's tile; every thread: wait for it (bounded).
// Returns false (CTA-uniform) when the wait gave up.
template <int BYTES>
__device__ __forceinline__ bool tma_tile_in(uint64_t* tile, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar, const KParams& P) {
  if (threadIdx.x == 0) {
    mbar_init1(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(BYTES + P.inject_tx)
                 : "memory");
    tma_load_2d(tile, map, x, y, bar);
  }
  __syncthreads();
  const bool done = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(!done)) {
    if (threadIdx.x == 0) {
      if (P.err) atomicOr(P.err, 1);
      mbar_wait_bounded(bar, 0);
    }
    __syncthreads();
    return false;
  }
  return true;
}

template <int CL, bool LZ>
__global__ void __launch_bounds__(kWColThreads) k_wcol_fwd_tma(KParams P, int nops,
                                                               const __grid_constant__ CUtensorMap ma,
                                                               const __grid_constant__ CUtensorMap mb) {
  using W = uint64_t;
  using S = WCol<CL>;
  __shared__ __align__(128) W tile[S::R * S::CT];
  __shared__ uint64_t bar;
  const uint32_t t = blockIdx.x % S::kTiles;
  const uint32_t rest = blockIdx.x / S::kTiles;
  const uint32_t op = rest % (uint32_t)nops, unit = rest / (uint32_t)nops;
  if (unit >= P.nunits) return;
  if (!tma_tile_in<S::R * S::CT * 8>(tile, op == 0 ? &ma : &mb, (int)(t * S::CT),
                                      (int)(unit * S::R), &bar, P))
    return;
  const WUnit<W, false> U(P, unit);
  const int th = threadIdx.x;
  const int c = th % S::CT, j = th / S::CT;
  const auto& K = U.K;
  W* dst = (op == 0 ? U.c : U.s) + t * S::CT + c;
  W x[S::M];
#pragma unroll
  for (int k = 0; k < S::M; k++) x[k] = tile[(j + S::J * k) * S::CT + c];
  ct_col<S::M, W, !LZ>(x, U.twf, K.q, K.two_q);
  if constexpr (S::J > 1) {
#pragma unroll
    for (int k = 0; k < S::M; k++) tile[(j + S::J * k) * S::CT + c] = x[k];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < S::M; i++) x[i] = tile[(S::M * j + i) * S::CT + c];
    ct_tail<S::J, 0, !LZ>(x, U.twf, (uint32_t)(S::M / S::J * j), K.q, K.two_q);
#pragma unroll
    for (int i = 0; i < S::M; i++) dst[(size_t)(S::M * j + i) * kW] = x[i];
  } else {
#pragma unroll
    for (int k = 0; k < S::M; k++) dst[(size_t)k * kW] = x[k];
  }
}

template <int CL, bool LZ>
__global__ void __launch_bounds__(kWColThreads) k_wcol_inv_tma(KParams P,
                                                               const __grid_constant__ CUtensorMap mc) {
  using W = uint64_t;
  using S = WCol<CL>;
  __shared__ __align__(128) W tile[S::R * S::CT];
  __shared__ uint64_t bar;
  const uint32_t t = blockIdx.x % S::kTiles;
  const uint32_t unit = blockIdx.x / S::kTiles;
  if (unit >= P.nunits) return;
  if (!tma_tile_in<S::R * S::CT * 8>(tile, &mc, (int)(t * S::CT), (int)(unit * S::R), &bar, P))
    return;
  const WUnit<W, false> U(P, unit);
  const int th = threadIdx.x;
  const int c = th % S::CT, j = th / S::CT;
  const auto& K = U.K;
  W x[S::M];
  if constexpr (S::J > 1) {
#pragma unroll
    for (int i = 0; i < S::M; i++) x[i] = tile[(S::M * j + i) * S::CT + c];
    gs_tail<S::J, 0, false, LZ>(x, U.twi, (uint32_t)(S::M / S::J * j), K);
#pragma unroll
    for (int i = 0; i < S::M; i++) tile[(S::M * j + i) * S::CT + c] = x[i];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S::M; k++) x[k] = tile[(j + S::J * k) * S::CT + c];
  } else {
#pragma unroll
    for (int k = 0; k < S::M; k++) x[k] = tile[k * S::CT + c];
  }
  gs_col<S::M, false, W, LZ>(x, U.twi, K);
  // the canonical words back into the tile, then one tensor copy to c
  if constexpr (S::J > 1) __syncthreads();  // everyone has read the transposed words
#pragma unroll
  for (int k = 0; k < S::M; k++) tile[(j + S::J * k) * S::CT + c] = csub(x[k], K.q);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (th == 0) {
    tma_store_2d(&mc, (int)(t * S::CT), (int)(unit * S::R), tile);
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // tile read before exit
  }
}

// N = 2^(10+CL), CL = 1..3: one cluster of R = 2^CL CTAs per unit, CTA rank
// t holding row t in shared memory.  Column steps: CTA t owns columns
// [t C, (t+1) C), C = 1024 / R.
// LZ: the wide lazy ranges (64-bit words, q < 2^60, 1/N folded).
template <int MODE, bool HALVE, typename W, int CL, bool LZ = false>
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
      ct_col<RR, W, !LZ>(x, twf, K.q, K.two_q);
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
    w_fwd<false, LZ>(va, vb, sa, sb, tw_f, th, K.q, K.two_q, false);
#pragma unroll
    for (int u = 0; u < 4; u++)
      __stcs(V.c + base + (size_t)t * kW + 4 * th + u, w_reduce_out<LZ>(va[u], K.q, K.two_q));
    return;  // no shared memory of another CTA is touched after the barrier
  } else {
    if constexpr (MODE != MODE_INV) {
      w_fwd<true, LZ>(va, vb, sa, sb, tw_f, th, K.q, K.two_q, kFused);
      if constexpr (kFused) {
        fused_pair<false, LZ>(va[0], va[1], vb[0], vb[1], wf, K);
        fused_pair<true, LZ>(va[2], va[3], vb[2], vb[3], wf, K);
      } else {
#pragma unroll
        for (int u = 0; u < 4; u++)
          va[u] =
              mul_barrett_alg4(w_reduce_out<LZ>(va[u], K.q, K.two_q),
                               w_reduce_out<LZ>(vb[u], K.q, K.two_q), K);
      }
    }
    w_inv_passes<HALVE, LZ>(va, sa, tw_i, th, K, kFused);
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
      gs_col<RR, HALVE, W, LZ>(x, twi, K);
#pragma unroll
      for (int r = 0; r < RR; r++) __stcs(V.c + base + (size_t)r * kW + c, csub(x[r], K.q));
    }
    cluster.sync();  // keep this CTA's rows alive until every CTA has read them
  }
}

// ------------------------------------------------------------ launchers

// A launch of `k`, with a programmatic dependency on the stream's previous
// kernel when `pdl` (the kernel then waits in pdl_wait before reading that
// kernel's output), else an ordinary launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_dep(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t st, bool pdl, Args... args) {
  if (!pdl) {
    k<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(block, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

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
  const bool pdl = P.pdl != 0;
  if (use_lazy16<W>(P))
    return launch_dep(k_wrows<MODE, false, W, false, true>, (unsigned)blocks, kWThreads,
                      kWRowsSmem<W>, st, pdl, P);
  if (P.halving)
    return launch_dep(k_wrows<MODE, true, W>, (unsigned)blocks, kWThreads, kWRowsSmem<W>, st, pdl,
                      P);
  return launch_dep(k_wrows<MODE, false, W>, (unsigned)blocks, kWThreads, kWRowsSmem<W>, st, pdl,
                    P);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// An operand array of nunits R rows of 1024 words as a 2-D tensor, box CT x R.
cudaError_t col_map(CUtensorMap* m, const void* base, uint32_t nunits, int R, int CT) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)kW, (cuuint64_t)nunits * (cuuint64_t)R};
  const cuuint64_t strides[1] = {(cuuint64_t)kW * 8};
  const cuuint32_t box[2] = {(cuuint32_t)CT, (cuuint32_t)R};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CL, typename W>
cudaError_t wcol_fwd_cl(const KParams& P, int nops, cudaStream_t st) {
  if constexpr (sizeof(W) == 8) {
    if (P.tma_cols && !P.halving) {
      using S = WCol<CL>;
      CUtensorMap ma, mb;
      cudaError_t e = col_map(&ma, P.a, P.nunits, S::R, S::CT);
      if (e == cudaSuccess) e = col_map(&mb, nops > 1 ? P.b : P.a, P.nunits, S::R, S::CT);
      if (e != cudaSuccess) return e;
      const size_t blocks = (size_t)P.nunits * nops * S::kTiles;
      if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
      if (use_lazy16<W>(P))
        k_wcol_fwd_tma<CL, true><<<(unsigned)blocks, kWColThreads, 0, st>>>(P, nops, ma, mb);
      else
        k_wcol_fwd_tma<CL, false><<<(unsigned)blocks, kWColThreads, 0, st>>>(P, nops, ma, mb);
      return cudaGetLastError();
    }
  }
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
  if constexpr (sizeof(W) == 8) {
    if (P.tma_cols && !P.halving) {
      using S = WCol<CL>;
      CUtensorMap mc;
      cudaError_t e = col_map(&mc, P.c, P.nunits, S::R, S::CT);
      if (e != cudaSuccess) return e;
      const size_t blocks = (size_t)P.nunits * S::kTiles;
      if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
      if (use_lazy16<W>(P))
        k_wcol_inv_tma<CL, true><<<(unsigned)blocks, kWColThreads, 0, st>>>(P, mc);
      else
        k_wcol_inv_tma<CL, false><<<(unsigned)blocks, kWColThreads, 0, st>>>(P, mc);
      return cudaGetLastError();
    }
  }
  const size_t blocks = (size_t)P.nunits * WCol<CL>::kTiles;
  if (blocks > (size_t)INT_MAX) return cudaErrorInvalidConfiguration;
  const bool pdl = P.pdl != 0;
  if (use_lazy16<W>(P))
    return launch_dep(k_wcol_inv<CL, false, W, false, true>, (unsigned)blocks, kWColThreads, 0,
                      st, pdl, P);
  if (P.halving)
    return launch_dep(k_wcol_inv<CL, true, W>, (unsigned)blocks, kWColThreads, 0, st, pdl, P);
  return launch_dep(k_wcol_inv<CL, false, W>, (unsigned)blocks, kWColThreads, 0, st, pdl, P);
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
  if constexpr (sizeof(W) == 8 && !H) {
    if (use_lazy16<W>(P)) return cudaLaunchKernelEx(&cfg, k_wclu<MODE, H, W, CL, true>, P);
  }
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
  KParams Q = P;
  Q.pdl = 1;  // rows after the forward columns, inverse columns after the rows
  if (e == cudaSuccess) e = prows(Q);
  if (e == cudaSuccess) e = mark(pe, 2, st);
  if (e == cudaSuccess) e = wcol_inv<W>(Q, st);
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
    P.pdl = 1;
  }
  return wrows<MODE_FWD, W>(P, st);
}

template <typename W>
cudaError_t ntt_inv_wide_w(const KParams& P, cudaStream_t st) {
  if (P.nunits == 0) return cudaSuccess;
  if (clustered(P.logn, P.nunits)) return clu<MODE_INV, W>(P, st);
  cudaError_t e = wrows<MODE_INV, W>(P, st);
  if (e != cudaSuccess || P.logn == kWLog) return e;
  KParams Q = P;
  Q.pdl = 1;
  return wcol_inv<W>(Q, st);
}

template <bool H, typename W, int CL>
cudaError_t prepare_clu() {
  constexpr bool kLz = sizeof(W) == 8 && !H;  // the wide-range forms exist too
  const void* fns[] = {(const void*)k_wclu<MODE_POLYMUL, H, W, CL>,
                       (const void*)k_wclu<MODE_POLYMUL_FUSED, H, W, CL>,
                       (const void*)k_wclu<MODE_FWD, H, W, CL>,
                       (const void*)k_wclu<MODE_INV, H, W, CL>,
                       (const void*)k_wclu<MODE_POLYMUL, H, W, CL, kLz>,
                       (const void*)k_wclu<MODE_POLYMUL_FUSED, H, W, CL, kLz>,
                       (const void*)k_wclu<MODE_FWD, H, W, CL, kLz>,
                       (const void*)k_wclu<MODE_INV, H, W, CL, kLz>};
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
  constexpr bool kLz = sizeof(W) == 8 && !H;
  const void* fns[] = {(const void*)k_wclu<MODE_POLYMUL, H, W, 4>,
                       (const void*)k_wclu<MODE_POLYMUL_FUSED, H, W, 4>,
                       (const void*)k_wclu<MODE_FWD, H, W, 4>,
                       (const void*)k_wclu<MODE_INV, H, W, 4>,
                       (const void*)k_wclu<MODE_POLYMUL, H, W, 4, kLz>,
                       (const void*)k_wclu<MODE_POLYMUL_FUSED, H, W, 4, kLz>,
                       (const void*)k_wclu<MODE_FWD, H, W, 4, kLz>,
                       (const void*)k_wclu<MODE_INV, H, W, 4, kLz>};
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
