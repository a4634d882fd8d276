/*
 * pm.h -- C ABI of the GB300 (sm_103a) negacyclic polynomial multiplication
 * library: c = a * b in Z_q[X]/(X^N + 1), following arxiv 2209.01290.
 *
 * The hot path (Eq. 2 of the paper):
 *   c = NTT^{GS, psi^-1}_{bo->no, 1/2}( NTT^{CT, psi}_{no->bo}(a) . NTT^{CT, psi}_{no->bo}(b) )
 * i.e. a merged Cooley-Tukey forward NTT (Algorithm 6), a pointwise product
 * reduced with the paper's Barrett variant (Algorithm 4), and a merged
 * Gentleman-Sande inverse NTT (Algorithm 7) with the 1/N scaling folded into
 * its last stage (or, with PM_PLAN_HALVING, into every butterfly as the
 * halvings of Sec. III-A).  Many independent products (RNS limbs x
 * polynomials) run in one call.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Coefficients are uint64 words.  A batch is laid out [npoly][nlimbs][N],
 *   contiguous, row-major: unit u = p * nlimbs + l starts at word u * N and
 *   uses limb l's modulus q_l.
 * - Inputs must be reduced, 0 <= x < q_l (the REQUIRE of Algorithms 1 and 4).
 *   The fast path does not check this; pm_check_reduced() does.
 *   Outputs are always canonical, 0 <= x < q_l.
 * - "d_" pointers are device pointers (cudaMalloc / torch CUDA tensors) owned
 *   by the caller, 16-byte aligned.  "h_" pointers are host pointers.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Compute calls are asynchronous on that stream: argument errors
 *   are returned synchronously; errors from the device surface on the next
 *   call on the plan or from pm_plan_sync().
 * - Every call returns a pm_status; on failure pm_last_error() gives a
 *   human-readable message (thread-local).
 * - A plan may be used from several host threads on different streams at
 *   once; destroying it while work is in flight is the caller's error.
 * - For N >= 2^14, pm_polymul needs [npoly][nlimbs][N] words of device
 *   scratch.  The plan keeps one scratch area per stream and grows it on
 *   demand; growing allocates (cudaMalloc, and cudaFree of the old area,
 *   which synchronises the device).  Call pm_plan_reserve() first when the
 *   call must not allocate (for example inside CUDA graph capture).
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pm_status {
    PM_OK = 0,
    PM_ERR_ARG = -1,         /* null pointer, zero/oversized count, misaligned pointer */
    PM_ERR_N = -2,           /* N not a power of two in [2, 2^17] */
    PM_ERR_Q = -3,           /* q not prime, not = 1 mod 2N, or q >= 2^62 */
    PM_ERR_PSI = -4,         /* psi^N != -1 mod q (not a primitive 2N-th root) */
    PM_ERR_CUDA = -5,        /* a CUDA runtime call failed (message has the CUDA error) */
    PM_ERR_OOM = -6,         /* device allocation failed */
    PM_ERR_TIMEOUT = -7,     /* a bounded device-side wait gave up */
    PM_ERR_BUDGET = -8,      /* request exceeds the configured device-memory budget */
    PM_ERR_UNSUPPORTED = -9, /* this GPU cannot run the requested launch shape */
    PM_ERR_RANGE = -10       /* pm_check_reduced found a coefficient >= q */
} pm_status;

/* Opaque plan: owns the device twiddle tables, Barrett/Shoup constants and
 * the launch choices for one (N, {q_l}, {psi_l}). */
typedef struct pm_plan pm_plan;

/* Largest moduli for a given N (setup of Sec. III-A: q prime with 2N | q-1,
 * psi a primitive 2N-th root of unity).
 *   log2n   : log2 N, 1..17
 *   nlimbs  : number of moduli wanted (1..1024)
 *   qbits   : moduli are < 2^qbits, 3 <= qbits <= 62 (Algorithm 4 needs
 *             len(q) <= 64 - 2)
 *   q_out   : host[nlimbs], the nlimbs largest primes q < 2^qbits with
 *             q = 1 mod 2N, descending
 *   psi_out : host[nlimbs] or NULL; psi_l = x^((q_l-1)/2N) for the first
 *             x = 2, 3, ... with psi_l^N = q_l - 1
 * Returns PM_ERR_Q if fewer than nlimbs such primes exist. */
pm_status pm_find_params(uint32_t log2n, uint32_t nlimbs, uint32_t qbits,
                         uint64_t *q_out, uint64_t *psi_out);

/* Create a plan (twiddle-table setup, Sec. III-A and Sec. VI-A: tables are
 * precomputed on the host and kept on the device).
 *   out     : receives the plan
 *   log2n   : log2 N, 1..17
 *   nlimbs  : number of RNS limbs L (1..1024)
 *   q       : host[nlimbs] moduli; each prime, = 1 mod 2N, 3 < q < 2^62
 *   psi     : host[nlimbs] primitive 2N-th roots, or NULL to derive them
 *             with the rule of pm_find_params
 *   device  : CUDA device ordinal the plan lives on
 * The plan builds, per limb, Psi_br[i] = psi^br(i) and
 * Psi^-1_br[i] = psi^-br(i) with their Shoup companions floor(w 2^64 / q),
 * mu = floor(2^(2m+1)/q) of Algorithm 4, and N^-1 for the inverse scaling.
 * Device memory: 32 N + 128 bytes per limb (PM_PLAN_FUSED: 32 N + 256;
 * PM_PLAN_WORD32: 16 N + 64, or 16 N + 128 with PM_PLAN_FUSED).
 * Synchronous.
 * Errors: PM_ERR_N, PM_ERR_Q, PM_ERR_PSI, PM_ERR_OOM, PM_ERR_CUDA. */
pm_status pm_plan_create(pm_plan **out, uint32_t log2n, uint32_t nlimbs,
                         const uint64_t *q, const uint64_t *psi, int device);

/* Plan options (bit flags for pm_plan_create_ex). */
enum {
    /* Scale by 1/2 at every inverse butterfly output, as in the paper's Eq. 2
     * (Zhang et al.'s halving, Sec. III-A); the inverse table then holds
     * Psi^-1_br[i] / 2.  Without the flag the inverse butterflies are
     * unscaled and 1/N is folded into the last inverse stage (its sum output
     * times N^-1, its twiddle times N^-1).  Both give identical results; the
     * default is faster on this GPU. */
    PM_PLAN_HALVING = 1,
    /* Products by the fused polynomial multiplication of Sec. III-C,
     * Algorithm 8: both forward transforms stop before their last stage
     * (Algorithm 6 with m < N/2), each pair of bit-reversed positions
     * (2i, 2i+1) is combined by the Karatsuba step of Algorithm 8 (three
     * Algorithm 4 products and one product by Psi_br[N/4 + floor(i/2)]),
     * and the inverse transform starts at its second stage.  Results are
     * identical to the default (the product is unique); only pm_polymul and
     * the calls built on it (graphs, uneven batches, serving, host pipeline)
     * change; pm_ntt_fwd / pm_ntt_inv / pm_pointwise stay full transforms.
     * Needs N >= 4 (log2n >= 2): pm_plan_create_ex gives PM_ERR_N for N = 2. */
    PM_PLAN_FUSED = 2,
    /* 32-bit words: every q must be below 2^30 (Algorithm 4 with a 32-bit
     * word, m <= beta - 2), coefficients are uint32_t and the twiddle tables
     * hold 32-bit words with 32-bit Shoup companions (Table 4's 30-bit
     * setting).  Such a plan takes the *32 calls below (pm_ntt_fwd32,
     * pm_ntt_inv32, pm_pointwise32, pm_polymul32, pm_check_reduced32) and is
     * refused (PM_ERR_ARG) by the uint64_t calls, the persistent variant,
     * graphs, uneven batches, the server and the host pipeline; the
     * uint64_t calls refuse it the other way round.  Combines with
     * PM_PLAN_HALVING and PM_PLAN_FUSED. */
    PM_PLAN_WORD32 = 4
};

/* pm_plan_create with options: `flags` is a combination of PM_PLAN_*;
 * unknown bits give PM_ERR_ARG; PM_PLAN_FUSED with log2n < 2 gives PM_ERR_N. */
pm_status pm_plan_create_ex(pm_plan **out, uint32_t log2n, uint32_t nlimbs,
                            const uint64_t *q, const uint64_t *psi, int device,
                            uint32_t flags);

/* The flags the plan was created with. */
pm_status pm_plan_flags(const pm_plan *plan, uint32_t *flags);

/* Release the plan and its device memory.  NULL is accepted. */
pm_status pm_plan_destroy(pm_plan *plan);

/* Pre-size the stream's scratch area for batches of up to npoly
 * polynomials (N >= 2^14 only; a no-op otherwise).  Synchronous. */
pm_status pm_plan_reserve(pm_plan *plan, uint32_t npoly, void *stream);

/* Plan facts: N, L, and the plan's moduli/psi (host[nlimbs] each, either
 * may be NULL). */
pm_status pm_plan_info(const pm_plan *plan, uint32_t *log2n, uint32_t *nlimbs,
                       uint64_t *q_out, uint64_t *psi_out);

/* Forward merged CT NTT (Algorithm 6), in place, for every unit of a batch:
 *   d_x[u*N + j] <- sum_i x_i psi_l^{i (2 br(j) + 1)} mod q_l
 * i.e. normal order in, bit-reversed order out (no->bo).  npoly >= 1. */
pm_status pm_ntt_fwd(const pm_plan *plan, uint64_t *d_x, uint32_t npoly, void *stream);

/* Inverse merged GS NTT (Algorithm 7 with the psi^-1 table, Eq. 1/Eq. 2),
 * in place: the exact inverse of pm_ntt_fwd (bit-reversed order in, normal
 * order out, 1/N applied -- folded into the last stage, or as 1/2 at every
 * butterfly with PM_PLAN_HALVING). */
pm_status pm_ntt_inv(const pm_plan *plan, uint64_t *d_x, uint32_t npoly, void *stream);

/* Pointwise (Hadamard) product d_c = d_a . d_b mod q_l, reduced with
 * Algorithm 4 (at most one correction).  d_c may alias d_a or d_b. */
pm_status pm_pointwise(const pm_plan *plan, const uint64_t *d_a, const uint64_t *d_b,
                       uint64_t *d_c, uint32_t npoly, void *stream);

/* Negacyclic product of every unit (Eq. 2): forward NTT of a and b,
 * pointwise product, inverse NTT with 1/N folded in.  N <= 2^13 (and small
 * batches at N = 2^14) run as one launch; larger N run as three launches on
 * `stream` (the forward column stages of a and b, one kernel that fuses the
 * in-row forward stages, the pointwise product and the in-row inverse
 * stages, then the inverse column stages), or as one persistent launch when
 * pm_plan_tune selects it.  d_a, d_b, d_c: device [npoly][nlimbs][N].  d_c
 * may alias d_a or d_b (each unit reads all of its inputs before it writes
 * any output). */
pm_status pm_polymul(const pm_plan *plan, const uint64_t *d_a, const uint64_t *d_b,
                     uint64_t *d_c, uint32_t npoly, void *stream);

/* ---- 32-bit words (plans created with PM_PLAN_WORD32, q < 2^30).
 * The same operations as pm_ntt_fwd, pm_ntt_inv, pm_pointwise, pm_polymul
 * and pm_check_reduced (same layout [npoly][nlimbs][N], same ownership,
 * aliasing and error rules) on uint32_t arrays; 16-byte aligned device
 * pointers.  A 64-bit plan gives PM_ERR_ARG. */
pm_status pm_ntt_fwd32(const pm_plan *plan, uint32_t *d_x, uint32_t npoly, void *stream);
pm_status pm_ntt_inv32(const pm_plan *plan, uint32_t *d_x, uint32_t npoly, void *stream);
pm_status pm_pointwise32(const pm_plan *plan, const uint32_t *d_a, const uint32_t *d_b,
                         uint32_t *d_c, uint32_t npoly, void *stream);
pm_status pm_polymul32(const pm_plan *plan, const uint32_t *d_a, const uint32_t *d_b,
                       uint32_t *d_c, uint32_t npoly, void *stream);
pm_status pm_check_reduced32(const pm_plan *plan, const uint32_t *d_x, uint32_t npoly,
                             void *stream);

/* Same product as pm_polymul, for callers that must not allocate device
 * memory: code running while another memory manager owns the device pool,
 * or latency-critical paths that cannot take the device-wide synchronisation
 * of cudaFree.  The paper has no counterpart; this is a deployment variant.
 * The caller still provides a, b and c.  Products of two distinct operands
 * at N >= 2^14 that run as three launches need scratch for b's column
 * image: it is a fixed 16 MiB array inside the library (2^21 words, held on
 * every device that loads the library until the process exits), so such a
 * batch must satisfy npoly * nlimbs * N <= 2^21; larger ones are rejected
 * with PM_ERR_ARG.  Squares (d_a == d_b), N < 2^14 and the one-launch
 * cluster batches use no scratch and have no such limit.  No cudaMalloc,
 * cudaFree or other allocating call is made.  The first call on a device
 * that needs the scratch looks up the array's device address
 * (cudaGetSymbolAddress) once and caches it per device ordinal; make that
 * first call before any stream capture, and do not rely on the cache across
 * cudaDeviceReset (the address belongs to the context that looked it up).
 * The launch choice is the plan's split path (a persistent tuning is not
 * used).  All calls share the one array and the scratch needs no clearing
 * (every word is written before it is read within a call), so calls that
 * overlap on the GPU -- on different streams or from several threads --
 * race on it: issue them on one stream. */
pm_status pm_polymul_noalloc(const pm_plan *plan, const uint64_t *d_a, const uint64_t *d_b,
                             uint64_t *d_c, uint32_t npoly, void *stream);

/* Same product from and to HOST memory: copies h_a, h_b to the device
 * buffers d_a, d_b, runs pm_polymul into d_c and copies d_c back to h_c, all
 * on `stream`, in chunks so that copies and compute of successive chunks
 * overlap (the plan's internal side streams and events order them).  Host
 * buffers should be pinned (cudaHostAlloc) for full copy speed.  The call
 * returns once h_c holds the result (it synchronises `stream`). */
pm_status pm_polymul_host(const pm_plan *plan, const uint64_t *h_a, const uint64_t *h_b,
                          uint64_t *h_c, uint64_t *d_a, uint64_t *d_b, uint64_t *d_c,
                          uint32_t npoly, void *stream);

/* ---- CUDA graphs: pm_polymul for fixed buffers, captured once and
 * replayed with one cudaGraphLaunch.  The graph owns its own scratch and
 * control block (allocated at creation), so replays allocate nothing.
 * Replays of one graph must not overlap on the device (they share its
 * scratch); the captured launch choice is the plan's tuning at creation. */
typedef struct pm_graph pm_graph;
pm_status pm_graph_create_polymul(pm_graph **out, const pm_plan *plan, const uint64_t *d_a,
                                  const uint64_t *d_b, uint64_t *d_c, uint32_t npoly);
pm_status pm_graph_launch(pm_graph *g, void *stream);
pm_status pm_graph_destroy(pm_graph *g);

/* ---- Uneven batches: many products of different N and limb counts in
 * one persistent launch (a work queue over all units).
 * A job is npoly polynomials of one plan (its N, limbs and tables), laid
 * out [npoly][nlimbs][N] as for pm_polymul; c may alias a or b. */
typedef struct pm_job {
    const pm_plan *plan;
    const uint64_t *a;
    const uint64_t *b;
    uint64_t *c;
    uint32_t npoly;
} pm_job;

/* Reusable context for uneven launches: device descriptor tables, the
 * column-stage scratch (one N-word area per unit of N >= 2^13) and the
 * control block, grown on demand (allocation only when growing). */
typedef struct pm_queue pm_queue;
pm_status pm_queue_create(pm_queue **out, int device);
pm_status pm_queue_destroy(pm_queue *q);
/* Pre-size for up to `units` units and `scratch_words` scratch words. */
pm_status pm_queue_reserve(pm_queue *q, uint64_t units, uint64_t scratch_words);

/* All jobs' products in one launch on `stream`.  Jobs with N >= 4096 share
 * the launch: each CTA takes column and row tasks of any unit from a ticket
 * counter (all column-forward tasks first, then rows, then column-inverse
 * tasks), waiting (bounded) on per-unit counters.  Jobs with N <= 2048 run
 * through their plan's own kernel on the same stream.  All plans must be on
 * the queue's device and agree on PM_PLAN_HALVING and on PM_PLAN_FUSED
 * (PM_ERR_ARG otherwise; jobs with N <= 2048 are exempt).  Calls on one queue must
 * be serialised on one stream (they share its buffers). */
pm_status pm_polymul_uneven(pm_queue *q, const pm_job *jobs, uint32_t njobs, void *stream);

/* How pm_polymul_uneven runs the jobs with N >= 4096:
 *   PM_UNEVEN_PERSISTENT: one persistent work-queue launch (above);
 *   PM_UNEVEN_GROUPED: the units grouped by N, each group through the column
 *     and row kernels of pm_polymul (rows of 1024 words for N >= 2^13, whole
 *     4096-word rows for N = 2^12; up to three launches per distinct N,
 *     every unit's pointers and tables from a descriptor table) -- no
 *     dependency waits, the throughput kernels;
 *   PM_UNEVEN_AUTO (default): GROUPED when the batch has at least 8 rows of
 *     4096 words per SM, else PERSISTENT.
 * Results are identical; PM_ERR_ARG for another value. */
enum { PM_UNEVEN_AUTO = 0, PM_UNEVEN_PERSISTENT = 1, PM_UNEVEN_GROUPED = 2 };
pm_status pm_queue_set_mode(pm_queue *q, int mode);

/* Synchronise `stream` and report PM_ERR_TIMEOUT if an uneven launch on this
 * queue gave up waiting for a dependency. */
pm_status pm_queue_sync(pm_queue *q, void *stream);

/* ---- Serving: a continuous-batching request loop.
 * Clients submit products whose operands are already on the device; a
 * worker thread forms batches from queued requests in arrival order,
 * admitting a request only when its output (npoly * nlimbs * N words) and
 * column-stage scratch (as many words again for N >= 2^13 unless a == b)
 * fit in the remaining budget of a device arena allocated once at creation,
 * and runs each batch as one uneven persistent launch (a batch holds plans
 * of one kind -- the same PM_PLAN_HALVING and PM_PLAN_FUSED bits; the first
 * request of another kind closes it).  Up to max_inflight
 * batches are on the device at once (one stream each), so requests arriving
 * while others run are admitted as soon as a slot and memory free up.
 * A request's output stays in the arena until pm_server_release(). */
typedef struct pm_server pm_server;
typedef struct pm_server_config {
    uint64_t hbm_budget_bytes;  /* arena size: the admission cap */
    uint32_t max_batch;         /* requests per launch, 0 = no cap */
    uint32_t max_inflight;      /* batches on the device at once, 1..8 */
    uint64_t min_batch_rows;    /* while a batch runs, launch the next only once
                                   the queue holds this many 4096-word rows of
                                   work; 0 = 4 x 3 x SM count.  An idle device
                                   always takes what is queued. */
} pm_server_config;
typedef struct pm_server_stats {
    uint64_t submitted, completed, batches, batched_requests, max_batch;
    uint64_t arena_peak_bytes, arena_used_bytes;
    /* batches launched while others were still unretired, at most (host view) */
    uint64_t max_inflight;
    /* the most batches in flight on the device at one instant (device
     * intervals: a timing event before and after each launch on its slot's
     * stream; swept over the last 16 batches at each retirement) */
    uint64_t max_device_overlap;
} pm_server_stats;

pm_status pm_server_create(pm_server **out, int device, const pm_server_config *cfg);
/* Drains queued and running requests, then frees everything; a queued
 * request that cannot fit beside the outputs clients still hold is failed
 * (PM_ERR_BUDGET) instead of waited for. */
pm_status pm_server_destroy(pm_server *s);
/* Queue one request (npoly products of `plan`); PM_ERR_BUDGET if it could
 * never fit.  d_a, d_b must stay valid until the request is done. */
pm_status pm_server_submit(pm_server *s, const pm_plan *plan, const uint64_t *d_a,
                           const uint64_t *d_b, uint32_t npoly, uint64_t *id_out);
/* Block until request `id` is done (PM_ERR_TIMEOUT after timeout_ms); gives
 * its device output [npoly][nlimbs][N] and submit-to-completion latency. */
pm_status pm_server_wait(pm_server *s, uint64_t id, uint32_t timeout_ms, uint64_t **d_c_out,
                         double *latency_us);
/* Return a done request's output memory to the arena. */
pm_status pm_server_release(pm_server *s, uint64_t id);
pm_status pm_server_get_stats(pm_server *s, pm_server_stats *out);

/* Checks 0 <= x < q_l for every coefficient of d_x [npoly][nlimbs][N];
 * returns PM_ERR_RANGE if one is out of range.  Synchronous. */
pm_status pm_check_reduced(const pm_plan *plan, const uint64_t *d_x, uint32_t npoly,
                           void *stream);

/* How pm_polymul is launched (a performance choice only; the results are
 * identical):
 *   PM_VARIANT_SPLIT      : the transform split into rows and columns: up to
 *                           three launches -- forward column stages, in-row
 *                           stages with the pointwise product, inverse column
 *                           stages (row kernel and row length: row_ops);
 *   PM_VARIANT_PERSISTENT : one persistent launch whose CTAs take column and
 *                           row tasks of all units from a work queue in a
 *                           software-pipelined order (lag_fwd / lag_inv are
 *                           the pipeline distances in units, ctas_per_sm the
 *                           resident CTAs per SM, 1..4, capped at what the
 *                           kernel holds: 4 for the 1024-word tasks up to
 *                           N = 2^16, else 3).  The tasks are those of the
 *                           1024-word split (row_ops 0 or 4, no per-stage
 *                           halving, N >= 2^13) or of 4096-word rows.  Uses
 *                           a control block of 16 + 8 * units bytes in the
 *                           stream's scratch.
 * row_ops (SPLIT; for PERSISTENT the task size as above):
 *   1..3: the transform as rows of 4096 words (N >= 4096):
 *   1 = 256 threads per row, a transformed before b (3 CTAs per SM);
 *   2 = 256 threads per row, a and b together sharing twiddle loads
 *       (2 CTAs per SM);
 *   3 = 1024 threads per row in radix-4 passes (1 CTA per SM);
 *   4 = the transform as N/1024 rows of 1024 words (N >= 1024): 256
 *       threads per row in radix-4 passes with the row's twiddles staged in
 *       shared memory, up to 4 CTAs per SM; for N = 2^11 .. 2^13, and N =
 *       2^14 batches of up to 16 units where the device runs clusters of 16
 *       CTAs, one launch (a thread-block cluster of N/1024 CTAs per unit
 *       exchanging the column stages through distributed shared memory),
 *       otherwise three launches (column stages, rows, column stages);
 *   5 = 4 with the column stages' tiles moved by 2-D tensor copies (64-bit
 *       words, 1/N folded; else as 4);
 *   0 = by N, word size and batch size (measured on GB300): 4 for 64-bit
 *       words, except N = 2^12 batches above 64 units; 4 for 32-bit words
 *       in batches of up to 2^20 words; otherwise 3 while the batch has at
 *       most (SM count) rows of 4096 words, else 2 (pm_ntt_fwd/inv: 1).
 *   Sizes a choice does not cover keep their own kernels (N <= 2^11 without
 *   4: one CTA per unit; N = 2^13 without 4: one CTA of 512 threads).
 * pm_plan_autotune() picks these by timing; without it a plan uses SPLIT,
 * row_ops 0 (persistent settings: 3 CTAs per SM, lags 8 and 64). */
enum { PM_VARIANT_SPLIT = 0, PM_VARIANT_PERSISTENT = 1 };
typedef struct pm_tuning {
    int32_t variant;
    uint32_t ctas_per_sm;
    uint32_t lag_fwd;
    uint32_t lag_inv;
    uint32_t row_ops;
} pm_tuning;

/* Autotuner: time every launch choice for batches of `npoly` polynomials
 * (the split path with each row kernel, the persistent launch with a few
 * pipeline distances) on temporary device buffers, keep the fastest in the
 * plan and return it (and its median time in ms).  Allocates, synchronises
 * `stream`; call it at setup, not on a hot path. */
pm_status pm_plan_autotune(pm_plan *plan, uint32_t npoly, void *stream, pm_tuning *best_out,
                           float *best_ms_out);

/* Set / read the plan's launch choice.  PM_ERR_ARG for out-of-range values. */
pm_status pm_plan_tune(pm_plan *plan, const pm_tuning *t);
pm_status pm_plan_get_tuning(const pm_plan *plan, pm_tuning *t);

/* The launch choice a pm_polymul (or pm_ntt_fwd / pm_ntt_inv) of npoly
 * polynomials on this plan makes: the plan's tuning with row_ops 0 replaced
 * by the row kernel the rule above picks for that batch (1..4).  No device
 * work.  PM_ERR_ARG for a NULL tuning or an invalid batch size. */
pm_status pm_plan_resolve_tuning(const pm_plan *plan, uint32_t npoly, pm_tuning *t);

/* Test hook: fault injection on the host side of the next polymul launch
 * on this plan (kind 0 clears it).
 *   PM_FAULT_WITHHOLD_SIGNAL : (next persistent launch) the row tasks wait
 *     for one more "column stage done" signal than will ever arrive, so
 *     their bounded waits run out (about a second); pm_plan_sync then
 *     reports PM_ERR_TIMEOUT and the results of that call are invalid.
 *   PM_FAULT_SHORT_TWIDDLES : (next split launch with 64-bit words, N >=
 *     2^10) every row CTA's barrier expects 16 bytes more than its bulk
 *     twiddle copies deliver, so its bounded wait runs out (about a second
 *     per CTA, twice); pm_plan_sync reports PM_ERR_TIMEOUT and the results of
 *     that call are invalid.
 * Nothing faults on the device and later calls work normally. */
enum { PM_FAULT_WITHHOLD_SIGNAL = 1, PM_FAULT_SHORT_TWIDDLES = 2 };
pm_status pm_plan_inject_fault(pm_plan *plan, int kind);

/* Profiling hook for pm_polymul: with n > 0, each later pm_polymul on this
 * plan records events[k] (cudaEvent_t, created by the caller) on its stream
 * after phase k: k = 0 before the first kernel, then after each kernel
 * (column forward, rows, column inverse for N >= 2^14; the single fused
 * kernel otherwise).  n = 0 turns it off.  n <= 4. */
pm_status pm_plan_set_phase_events(pm_plan *plan, void *const *events, int n);

/* Wait for all work the plan's calls queued on `stream` and report any
 * device-side error, including PM_ERR_TIMEOUT when a persistent launch on
 * that stream gave up waiting for a dependency (its results are then not
 * valid).  Each device-side wait is bounded (about a second). */
pm_status pm_plan_sync(const pm_plan *plan, void *stream);

/* Message for the last failing call on this host thread ("" if none). */
const char *pm_last_error(void);

/* Copy of pm_last_error() into buf[n] (always NUL-terminated when n > 0). */
pm_status pm_last_error_string(char *buf, size_t n);

/* Roofline denominators for this integer path, measured on `device`:
 *   mulmod_per_s : register-resident rate of the lazy Shoup 64-bit modular
 *                  product (60-bit q) used by the NTT butterflies
 *   imad_per_s   : 32-bit integer multiply-add rate
 * Runs two short kernels (tens of milliseconds) and synchronises the device.
 * The paper measures reductions the same way (Sec. II-B, register-resident
 * microbenchmarks of one reduction per operation). */
pm_status pm_measure_peaks(int device, double *mulmod_per_s, double *imad_per_s);

/* ---- Modular-reduction study (Sec. II-B, Fig. 4) on this GPU.
 * Variants of reducing a*b mod q for a, b < q, q odd, 4 < q < 2^62:
 *   PM_RED_BUILTIN    the C '%' operator on the 128-bit product
 *   PM_RED_ALG2       classical Barrett, Algorithm 2 (up to two corrections)
 *   PM_RED_ALG3       Dhem-Quisquater, Algorithm 3 (needs len(q) <= 60)
 *   PM_RED_ALG4       the paper's Barrett variant, Algorithm 4
 *   PM_RED_SHOUP      Shoup's product (b a constant with a precomputed
 *                     companion), fully reduced
 *   PM_RED_MONTGOMERY Montgomery REDC with R = 2^64 (b in Montgomery form) */
enum {
    PM_RED_BUILTIN = 0, PM_RED_ALG2 = 1, PM_RED_ALG3 = 2, PM_RED_ALG4 = 3,
    PM_RED_SHOUP = 4, PM_RED_MONTGOMERY = 5, PM_RED_COUNT = 6
};

/* Register-resident throughput of each variant (reductions/s) for modulus q;
 * rates[PM_RED_ALG3] = 0 when len(q) > 60.  Runs short kernels, synchronous. */
pm_status pm_reduction_rates(int device, uint64_t q, double *rates);

/* d_c[i] = a[i] * b[i] mod q computed with `variant`, n elements on the
 * current device (for checking each variant; the constants a variant needs
 * are derived per element). */
pm_status pm_reduction_apply(int variant, uint64_t q, const uint64_t *d_a, const uint64_t *d_b,
                             uint64_t *d_c, uint64_t n, void *stream);

/* Library version string. */
const char *pm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PM_H */
