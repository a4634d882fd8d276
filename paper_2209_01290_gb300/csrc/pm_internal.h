// pm_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "pm_arith.cuh"

namespace pm {

// MODE_POLYMUL_FUSED: polymul by Algorithm 8 (truncated transforms around the
// Karatsuba pair step) instead of Eq. 2's full transforms.
enum Mode { MODE_POLYMUL = 0, MODE_FWD = 1, MODE_INV = 2, MODE_POLYMUL_FUSED = 3 };

// Kernel parameters for one batched call on one plan.
struct UnitDesc;

struct KParams {
  const uint64_t* a;     // operand a (device), [nunits][N]
  const uint64_t* b;     // operand b
  uint64_t* c;           // output / in-place buffer
  uint64_t* s;           // scratch [nunits][N] for the column-split path
  const TwPair* twf;     // [nlimbs][N] forward twiddles Psi_br with Shoup companions
  const TwPair* twi;     // [nlimbs][N] inverse twiddles Psi^-1_br * 1/2 with companions
  const LimbConst* lc;   // [nlimbs]
  uint32_t logn;
  uint32_t nlimbs;
  uint32_t nunits;       // npoly * nlimbs
  uint32_t halving;      // 1: per-stage 1/2 scaling (table holds w/2); 0: 1/N folded at the end
  uint32_t row_ops;      // row kernel: 1 = operands one after the other, 2 = together,
                         // 3 = 1024 threads per 4096-word row, 4 = 1024-word rows
  uint32_t fused;        // polymul by Algorithm 8; lc then has 2 nlimbs entries, the second
                         // half (2/N in place of 1/N) used by the polymul launchers
  uint32_t word32;       // 1: 32-bit words; a/b/c/s hold uint32_t, twf/twi TwPair32,
                         // lc LimbConst32 (the pointers are reinterpreted)
  uint32_t lazy16;       // 1: every q < 2^60 (64-bit words, no halving): the 1024-word
                         // split lets values grow to 16q between reductions
  const UnitDesc* desc;  // grouped launches (64-bit words): unit u's operands, output,
                         // scratch, tables and constants come from desc[u] instead
  int* err;              // device flag: set (to 1) by a CTA whose bounded wait for its
                         // staged twiddles gave up (NULL: not recorded)
  uint32_t inject_tx;    // test hook: extra bytes each row CTA's barrier expects (0)
  uint32_t tma_cols;     // 1024-word split, 64-bit words, 1/N folded: the column kernels
                         // load their tiles with 2-D tensor copies (pm_plan_tune row_ops 5)
  uint32_t pdl;          // launched with a programmatic dependency on the previous kernel
                         // of the stream: wait (griddepcontrol) before reading its output
};

// Optional profiling hook: when set, the launcher records ev[k] on the
// launch stream after phase k of a polymul (k < n).  Host-side only.
struct PhaseEvents {
  cudaEvent_t ev[4];
  int n;
};

// Persistent work-queue launch (pm_persist.cu).
struct PersistArgs {
  uint32_t* ctl;    // [0] ticket counter, [1] error flag, [4 + 2u] per-unit counters
  uint32_t F, W, I; // column-forward, row and column-inverse tasks per unit
  uint32_t lagF;    // ticket groups between a unit's column-forward and row tasks
  uint32_t lagI;    // ticket groups between a unit's column-forward and column-inverse tasks
  uint32_t ntasks;  // total tickets
  uint32_t withheld;  // fault injection: row tasks wait for this many extra signals (0)
  // Compact ticket order (1024-word persistent kernel): groups 0 .. nunits +
  // lagI - 1 fall into nseg segments; segment k covers groups seg_g[k] ..
  // seg_g[k+1] - 1, starts at ticket seg_t[k], and its groups hold the tasks
  // the bits of seg_mask[k] name (1: column-forward, 2: rows, 4: column-
  // inverse), so no ticket is empty.
  uint32_t nseg;
  uint32_t seg_g[8], seg_t[8], seg_mask[8];
};

// Uneven batch (pm_persist.cu): one descriptor per unit.
struct alignas(64) UnitDesc {
  const uint64_t* a;     // operand rows of this unit (device)
  const uint64_t* b;     // == a for a square
  uint64_t* c;           // output; also receives a's column-stage image
  uint64_t* s;           // scratch N words for b's image (== c for a square)
  const TwPair* twf;     // the unit's limb tables (its plan)
  const TwPair* twi;
  const LimbConst* lc;    // the fused constants for an Algorithm 8 plan
  uint32_t logn;
  uint32_t pad;
};

struct UnevenArgs {
  const UnitDesc* units;
  const uint32_t* pre_f;  // [nunits] exclusive prefix counts of column-forward tasks
  const uint32_t* pre_w;  // ... of row tasks
  const uint32_t* pre_i;  // ... of column-inverse tasks
  uint32_t* ctl;          // [0] ticket, [1] error flag, [4 + 2u] per-unit counters
  uint32_t nunits;
  uint32_t tf, tw, ti;    // tickets per section
  // 1024-word uneven kernel: blk[k][i] = the unit holding ticket i * 32 of
  // section k (section-relative), so a ticket's unit is found from there by
  // a short forward scan of the prefix counts
  const uint32_t* blk_f;
  const uint32_t* blk_w;
  const uint32_t* blk_i;
};

cudaError_t uneven_prepare();
cudaError_t launch_uneven(const UnevenArgs& A, bool halving, bool fused, int grid,
                          cudaStream_t st);

cudaError_t persist_prepare();
size_t persist_ctl_words(uint32_t nunits);
cudaError_t launch_polymul_persistent(const KParams& P, uint32_t* ctl, int grid, uint32_t lagF,
                                      uint32_t lagI, cudaStream_t st, uint32_t withheld = 0);

// Persistent launches over the 1024-word split (pm_wpersist.cu): 64-bit
// words, 1/N folded (no per-stage halving).
bool wpersist_ok(uint32_t logn);  // uniform batches: N = 2^13 .. 2^17
// resident CTAs per SM the kernel for N = 2^logn is built for (logn 0: the
// uneven kernel)
int wpersist_ctas_per_sm(uint32_t logn);
// Tasks of one uneven unit of N = 2^logn (2^12 .. 2^17): column-forward,
// row and column-inverse; returns their sum.
uint32_t wuneven_tasks(uint32_t logn, bool square, uint32_t* f, uint32_t* w, uint32_t* i);
cudaError_t wpersist_prepare();
cudaError_t launch_polymul_wpersistent(const KParams& P, uint32_t* ctl, int grid, uint32_t lagF,
                                       uint32_t lagI, cudaStream_t st, uint32_t withheld = 0);
cudaError_t launch_wuneven(const UnevenArgs& A, bool lazy16, bool fused, int grid,
                           cudaStream_t st);

cudaError_t kernels_prepare();
cudaError_t launch_polymul(const KParams& P, cudaStream_t st,
                           const PhaseEvents* pe = nullptr);
// Grouped uneven products (64-bit words): P.desc holds P.nunits unit
// descriptors of one N (logn >= 12), P.halving / P.fused as for their plans.
cudaError_t launch_polymul_grouped(const KParams& P, cudaStream_t st);
cudaError_t launch_ntt_fwd(const KParams& P, cudaStream_t st);
cudaError_t launch_ntt_inv(const KParams& P, cudaStream_t st);
cudaError_t launch_pointwise(const KParams& P, cudaStream_t st, int num_sms);

// The 1024-word split (pm_wide.cu), chosen with row_ops 4, for N = 2^10 ..
// 2^17: one launch up to N = 2^13 and for small N = 2^14 batches (a
// thread-block cluster per unit above 2^10, no scratch), otherwise three
// (the [nunits][N] scratch of the 4096-word split).
bool wide_polymul_ok(uint32_t logn);
// True when the 1024-word split runs this polymul batch as one launch
// (N = 2^10, or the cluster kernel), which uses no scratch.
bool wide_single_launch(uint32_t logn, uint32_t nunits);
bool wide_ntt_ok(uint32_t logn);
cudaError_t wide_prepare();
cudaError_t launch_polymul_wide(const KParams& P, cudaStream_t st, const PhaseEvents* pe);
cudaError_t launch_ntt_fwd_wide(const KParams& P, cudaStream_t st);
cudaError_t launch_ntt_inv_wide(const KParams& P, cudaStream_t st);
// Grouped uneven products of one N >= 2^13 (64-bit words, P.desc) through
// the 1024-word split.
cudaError_t launch_polymul_wide_grouped(const KParams& P, cudaStream_t st);
cudaError_t launch_check_reduced(const KParams& P, int* d_flag, cudaStream_t st, int num_sms);

// True when the polymul path for this N needs the [nunits][N] scratch.
inline bool polymul_needs_scratch(uint32_t logn) { return logn >= 14; }
// True when launch_polymul(P) writes P.s: the three-launch split of two
// distinct operands (a square keeps its one image in c).
bool polymul_writes_scratch(const KParams& P);

}  // namespace pm
