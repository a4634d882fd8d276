// pm_capi.cu -- the C ABI declared in include/pm.h: plan lifetime, argument
// validation, error reporting and dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pm.h"
#include "pm_internal.h"
#include "pm_params.h"

#define PM_VERSION "0.1.0"

namespace {

thread_local char g_err[512] = "";

pm_status fail(pm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

pm_status ok() {
  g_err[0] = '\0';
  return PM_OK;
}

pm_status cuda_fail(cudaError_t e, const char* what) {
  const pm_status st = (e == cudaErrorMemoryAllocation) ? PM_ERR_OOM : PM_ERR_CUDA;
  return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Makes `dev` current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

std::mutex g_prep_mu;
std::vector<int> g_prepared;  // devices on which kernels_prepare() ran

cudaError_t prepare_device(int dev) {
  std::lock_guard<std::mutex> lk(g_prep_mu);
  for (int d : g_prepared)
    if (d == dev) return cudaSuccess;
  cudaError_t e = pm::kernels_prepare();
  if (e == cudaSuccess) g_prepared.push_back(dev);
  return e;
}

constexpr uint32_t kMaxLog2N = 17;
constexpr uint32_t kMaxLimbs = 1024;
constexpr int kHostChunks = 8;

}  // namespace

struct pm_plan {
  int device = 0;
  int num_sms = 0;
  uint32_t logn = 0, nlimbs = 0;
  uint32_t flags = 0;
  // every q < 2^60, 64-bit words, 1/N folded: the 1024-word split may let
  // values grow to 16q between reductions (KParams::lazy16)
  bool lazy16 = false;
  std::vector<uint64_t> q, psi;
  pm::LimbConst* d_lc = nullptr;
  pm::TwPair* d_twf = nullptr;
  pm::TwPair* d_twi = nullptr;
  int* d_flag = nullptr;
  int* d_err = nullptr;  // set by a row CTA whose bounded wait for its twiddles gave up
  std::mutex mu;  // guards the scratch list and the host-pipeline objects
  // Scratch for the column-split polymul path, one area per stream so that
  // calls on different streams never share it (calls on one stream are
  // ordered by the stream).
  struct Scratch {
    cudaStream_t stream;
    uint64_t* ptr;      // [units][N] words
    uint64_t units;
    uint32_t* ctl;      // persistent-kernel control block
    size_t ctl_words;
  };
  std::vector<Scratch> scratch;
  // Launch choice for polymul (set by pm_plan_tune / pm_plan_autotune).
  pm_tuning tune{};
  // Fault injection for tests (pm_plan_inject_fault): consumed by the next
  // persistent launch.
  int inject = 0;
  cudaStream_t side_in = nullptr, side_out = nullptr;
  cudaEvent_t ev_in[kHostChunks] = {}, ev_done[kHostChunks] = {}, ev_start = nullptr,
              ev_end = nullptr;
  pm::PhaseEvents phase{};  // profiling hook (pm_plan_set_phase_events)
};

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

pm_status check_plan(const pm_plan* p) {
  if (!p) return fail(PM_ERR_ARG, "plan is NULL");
  return PM_OK;
}

bool is_word32(const pm_plan* p) { return (p->flags & PM_PLAN_WORD32) != 0; }

// The calls on 64-bit words and their *32 counterparts each take plans of
// their own word size only.
pm_status check_word(const pm_plan* p, bool word32, const char* fn) {
  if (is_word32(p) != word32)
    return fail(PM_ERR_ARG, "%s: the plan uses %d-bit words", fn, is_word32(p) ? 32 : 64);
  return PM_OK;
}

pm_status check_plan_word(const pm_plan* p, bool word32, const char* fn) {
  pm_status s = check_plan(p);
  return s != PM_OK ? s : check_word(p, word32, fn);
}

pm::KParams base_params(const pm_plan* p, uint32_t npoly) {
  pm::KParams P{};
  P.twf = p->d_twf;
  P.twi = p->d_twi;
  P.lc = p->d_lc;
  P.logn = p->logn;
  P.nlimbs = p->nlimbs;
  P.nunits = npoly * p->nlimbs;
  P.halving = (p->flags & PM_PLAN_HALVING) ? 1 : 0;
  // row kernel: 1 = k_rows, 2 = k_rows2, 3 = k_rows_lat, 4 = the 1024-word
  // rows of pm_wide.cu; 0 = by N, word size and batch size, as measured on
  // GB300: the 1024-word rows for 64-bit words at every N >= 2^10 except
  // N = 2^12 batches above 64 units, and for 32-bit words in batches of up
  // to 2^20 words; otherwise the 4096-word rows, the 1024-thread latency
  // rows up to one row per SM and the two-operand throughput rows above
  const uint64_t words = (uint64_t)P.nunits << p->logn;
  const bool wide = p->logn >= 10 && (is_word32(p) ? words <= (1ull << 20)
                                                   : !(p->logn == 12 && P.nunits > 64));
  const uint64_t row_ctas = p->logn >= 12 ? (uint64_t)P.nunits << (p->logn - 12) : 0;
  // row_ops 5: the 1024-word split with tensor-copy column tiles
  P.tma_cols = (p->tune.row_ops == 5 && !is_word32(p) && !(p->flags & PM_PLAN_HALVING)) ? 1 : 0;
  P.row_ops = p->tune.row_ops == 5 ? 4u
              : p->tune.row_ops ? p->tune.row_ops
              : wide          ? 4u
                              : (row_ctas <= (uint64_t)p->num_sms ? 3u : 2u);
  P.fused = (p->flags & PM_PLAN_FUSED) ? 1 : 0;  // read by the polymul launchers only
  P.word32 = is_word32(p) ? 1 : 0;
  P.lazy16 = p->lazy16 ? 1 : 0;
  P.err = p->d_err;
  return P;
}

pm_status check_batch(const pm_plan* p, uint32_t npoly) {
  if (npoly == 0) return fail(PM_ERR_ARG, "npoly must be >= 1");
  const uint64_t units = (uint64_t)npoly * p->nlimbs;
  if (units > 0x7fffffffull >> (p->logn > 12 ? p->logn - 12 : 0))
    return fail(PM_ERR_ARG, "batch too large: %llu units", (unsigned long long)units);
  return PM_OK;
}

// The stream's scratch area, grown to at least `units` polynomials (caller
// holds p->mu).  Growing frees the old area (cudaFree synchronises the
// device) and allocates a new one.  With `ctl`, also the persistent kernel's
// control block for `units` units.
pm_status ensure_scratch(pm_plan* p, cudaStream_t st, uint64_t units, uint64_t** out,
                         uint32_t** ctl = nullptr) {
  pm_plan::Scratch* sc = nullptr;
  for (auto& s : p->scratch)
    if (s.stream == st) sc = &s;
  if (!sc) {
    p->scratch.push_back(pm_plan::Scratch{st, nullptr, 0, nullptr, 0});
    sc = &p->scratch.back();
  }
  if (ctl) {
    const size_t words = pm::persist_ctl_words((uint32_t)units);
    if (words > sc->ctl_words) {
      if (sc->ctl) {
        cudaError_t e = cudaFree(sc->ctl);
        sc->ctl = nullptr;
        sc->ctl_words = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(ctl)");
      }
      cudaError_t e = cudaMalloc(&sc->ctl, words * 4);
      if (e != cudaSuccess) {
        sc->ctl = nullptr;
        return cuda_fail(e, "cudaMalloc(ctl)");
      }
      e = cudaMemset(sc->ctl, 0, words * 4);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(ctl)");
      sc->ctl_words = words;
    }
    *ctl = sc->ctl;
  }
  if (units > sc->units) {
    if (sc->ptr) {
      cudaError_t e = cudaFree(sc->ptr);
      sc->ptr = nullptr;
      sc->units = 0;
      if (e != cudaSuccess) return cuda_fail(e, "cudaFree(scratch)");
    }
    cudaError_t e = cudaMalloc(&sc->ptr, (size_t)units << p->logn << 3);
    if (e != cudaSuccess) {
      sc->ptr = nullptr;
      return cuda_fail(e, "cudaMalloc(scratch)");
    }
    sc->units = units;
  }
  *out = sc->ptr;
  return PM_OK;
}

void destroy_plan(pm_plan* p) {
  if (!p) return;
  DeviceGuard g(p->device);
  cudaFree(p->d_lc);
  cudaFree(p->d_twf);
  cudaFree(p->d_twi);
  cudaFree(p->d_flag);
  cudaFree(p->d_err);
  for (auto& sc : p->scratch) {
    cudaFree(sc.ptr);
    cudaFree(sc.ctl);
  }
  if (p->side_in) cudaStreamDestroy(p->side_in);
  if (p->side_out) cudaStreamDestroy(p->side_out);
  for (int i = 0; i < kHostChunks; ++i) {
    if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
    if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
  }
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_end) cudaEventDestroy(p->ev_end);
  delete p;
}

bool use_persistent(const pm_plan* p) {
  return p->tune.variant == PM_VARIANT_PERSISTENT && p->logn >= 13 && !is_word32(p);
}

// One persistent launch with the plan's tuning: the 1024-word tasks (row
// kernel choice 4, 1/N folded, N >= 2^13) or the 4096-word ones.
cudaError_t launch_persistent(const pm_plan* p, const pm::KParams& P, uint32_t* ctl,
                              cudaStream_t st, uint32_t withheld) {
  if (P.row_ops == 4 && !P.halving && pm::wpersist_ok(p->logn)) {
    const int ctas = std::min((int)p->tune.ctas_per_sm, pm::wpersist_ctas_per_sm(p->logn));
    return pm::launch_polymul_wpersistent(P, ctl, p->num_sms * ctas, p->tune.lag_fwd,
                                          p->tune.lag_inv, st, withheld);
  }
  const int ctas = std::min((int)p->tune.ctas_per_sm, 3);
  return pm::launch_polymul_persistent(P, ctl, p->num_sms * ctas, p->tune.lag_fwd,
                                       p->tune.lag_inv, st, withheld);
}

pm_status polymul_impl(pm_plan* p, const uint64_t* d_a, const uint64_t* d_b, uint64_t* d_c,
                       uint32_t npoly, cudaStream_t st) {
  pm::KParams P = base_params(p, npoly);
  P.a = d_a;
  P.b = d_b;
  P.c = d_c;
  const pm::PhaseEvents* pe = p->phase.n ? &p->phase : nullptr;
  cudaError_t e;
  if (use_persistent(p)) {
    uint32_t* ctl = nullptr;
    pm_status s = ensure_scratch(p, st, P.nunits, &P.s, &ctl);
    if (s != PM_OK) return s;
    if (pe && pe->n > 0 && (e = cudaEventRecord(pe->ev[0], st)) != cudaSuccess)
      return cuda_fail(e, "event");
    const uint32_t withheld = (p->inject == PM_FAULT_WITHHOLD_SIGNAL) ? 1u : 0u;
    p->inject = 0;
    e = launch_persistent(p, P, ctl, st, withheld);
    if (e != cudaSuccess) return cuda_fail(e, "persistent polymul launch");
    for (int k = 1; pe && k < pe->n; ++k)
      if ((e = cudaEventRecord(pe->ev[k], st)) != cudaSuccess) return cuda_fail(e, "event");
    return PM_OK;
  }
  if (pm::polymul_needs_scratch(p->logn)) {
    pm_status s = ensure_scratch(p, st, P.nunits, &P.s);
    if (s != PM_OK) return s;
  }
  if (p->inject == PM_FAULT_SHORT_TWIDDLES) {
    P.inject_tx = 16;
    p->inject = 0;
  }
  e = pm::launch_polymul(P, st, pe);
  if (e != cudaSuccess) return cuda_fail(e, "polymul launch");
  return PM_OK;
}

}  // namespace

extern "C" {

const char* pm_version(void) { return PM_VERSION; }

const char* pm_last_error(void) { return g_err; }

pm_status pm_last_error_string(char* buf, size_t n) {
  if (!buf || n == 0) return PM_ERR_ARG;
  snprintf(buf, n, "%s", g_err);
  return PM_OK;
}

pm_status pm_find_params(uint32_t log2n, uint32_t nlimbs, uint32_t qbits, uint64_t* q_out,
                         uint64_t* psi_out) {
  if (log2n < 1 || log2n > kMaxLog2N) return fail(PM_ERR_N, "log2n=%u outside [1,17]", log2n);
  if (nlimbs < 1 || nlimbs > kMaxLimbs) return fail(PM_ERR_ARG, "nlimbs=%u outside [1,1024]", nlimbs);
  if (qbits < 3 || qbits > 62 || qbits <= log2n + 1)
    return fail(PM_ERR_Q, "qbits=%u invalid for log2n=%u (need log2n+1 < qbits <= 62)", qbits, log2n);
  if (!q_out) return fail(PM_ERR_ARG, "q_out is NULL");
  std::vector<uint64_t> qs(nlimbs);
  const int got = pm::host::largest_ntt_primes(log2n, qbits, nlimbs, qs.data());
  if (got < (int)nlimbs)
    return fail(PM_ERR_Q, "only %d primes q < 2^%u with q = 1 mod 2^%u", got, qbits, log2n + 1);
  for (uint32_t i = 0; i < nlimbs; ++i) {
    q_out[i] = qs[i];
    if (psi_out) {
      psi_out[i] = pm::host::default_psi(qs[i], log2n);
      if (!psi_out[i]) return fail(PM_ERR_PSI, "no psi found for q=%llu", (unsigned long long)qs[i]);
    }
  }
  return ok();
}

pm_status pm_plan_create(pm_plan** out, uint32_t log2n, uint32_t nlimbs, const uint64_t* q,
                         const uint64_t* psi, int device) {
  return pm_plan_create_ex(out, log2n, nlimbs, q, psi, device, 0);
}

pm_status pm_plan_create_ex(pm_plan** out, uint32_t log2n, uint32_t nlimbs, const uint64_t* q,
                            const uint64_t* psi, int device, uint32_t flags) {
  if (!out) return fail(PM_ERR_ARG, "out is NULL");
  if (flags & ~(uint32_t)(PM_PLAN_HALVING | PM_PLAN_FUSED | PM_PLAN_WORD32))
    return fail(PM_ERR_ARG, "unknown plan flags 0x%x", flags);
  const bool word32 = (flags & PM_PLAN_WORD32) != 0;
  *out = nullptr;
  if (log2n < 1 || log2n > kMaxLog2N) return fail(PM_ERR_N, "log2n=%u outside [1,17]", log2n);
  if ((flags & PM_PLAN_FUSED) && log2n < 2)
    return fail(PM_ERR_N, "PM_PLAN_FUSED needs N >= 4 (Algorithm 8)");
  if (nlimbs < 1 || nlimbs > kMaxLimbs) return fail(PM_ERR_ARG, "nlimbs=%u outside [1,1024]", nlimbs);
  if (!q) return fail(PM_ERR_ARG, "q is NULL");
  const uint64_t n = (uint64_t)1 << log2n;
  std::vector<uint64_t> psis(nlimbs);
  for (uint32_t l = 0; l < nlimbs; ++l) {
    const uint64_t ql = q[l];
    if (ql <= 3 || ql >= ((uint64_t)1 << 62))
      return fail(PM_ERR_Q, "limb %u: q=%llu outside (3, 2^62)", l, (unsigned long long)ql);
    if (word32 && ql >= ((uint64_t)1 << 30))
      return fail(PM_ERR_Q, "limb %u: q=%llu is not below 2^30 (PM_PLAN_WORD32)", l,
                  (unsigned long long)ql);
    if ((ql - 1) % (2 * n))
      return fail(PM_ERR_Q, "limb %u: q=%llu is not 1 mod 2N (N=%llu)", l, (unsigned long long)ql,
                  (unsigned long long)n);
    if (!pm::host::is_prime_u64(ql))
      return fail(PM_ERR_Q, "limb %u: q=%llu is not prime", l, (unsigned long long)ql);
    if (psi) {
      const uint64_t p = psi[l];
      if (p == 0 || p >= ql || pm::host::pow_mod(p, n, ql) != ql - 1)
        return fail(PM_ERR_PSI, "limb %u: psi=%llu is not a primitive 2N-th root mod q", l,
                    (unsigned long long)p);
      psis[l] = p;
    } else {
      psis[l] = pm::host::default_psi(ql, log2n);
      if (!psis[l]) return fail(PM_ERR_PSI, "limb %u: no psi found", l);
    }
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(PM_ERR_ARG, "device %d not present (%d devices)", device, ndev);
  DeviceGuard g(device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_plan* p = new (std::nothrow) pm_plan();
  if (!p) return fail(PM_ERR_OOM, "host allocation failed");
  p->device = device;
  p->flags = flags;
  p->tune.variant = PM_VARIANT_SPLIT;
  p->tune.ctas_per_sm = 3;
  p->tune.lag_fwd = 8;
  p->tune.lag_inv = 64;
  p->tune.row_ops = 0;
  p->logn = log2n;
  p->nlimbs = nlimbs;
  p->q.assign(q, q + nlimbs);
  p->psi = psis;
  e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  e = prepare_device(device);
  if (e == cudaSuccess) e = pm::persist_prepare();
  if (e == cudaSuccess) e = pm::wpersist_prepare();
  if (e != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e, "kernel attributes");
  }
  // limb constants: [0, L) plain; for PM_PLAN_FUSED, [L, 2L) the constants
  // of Algorithm 8's truncated inverse (2/N in place of 1/N).  With
  // PM_PLAN_WORD32 the tables hold the 32-bit types (the device pointers are
  // reinterpreted by the kernels).
  const uint32_t nlc = (flags & PM_PLAN_FUSED) ? 2 * nlimbs : nlimbs;
  const bool halving = (flags & PM_PLAN_HALVING) != 0;
  p->lazy16 = !word32 && !halving;
  for (uint32_t l = 0; l < nlimbs; ++l)
    if (q[l] >> 60) p->lazy16 = false;
  std::vector<pm::LimbConst> lc;
  std::vector<pm::TwPair> twf, twi;
  std::vector<pm::LimbConst32> lc32;
  std::vector<pm::TwPair32> twf32, twi32;
  const void *h_lc, *h_twf, *h_twi;
  size_t lc_bytes, tw_bytes;
  if (word32) {
    lc32.resize(nlc);
    twf32.resize((size_t)nlimbs * n);
    twi32.resize((size_t)nlimbs * n);
    for (uint32_t l = 0; l < nlimbs; ++l)
      pm::host::build_limb32(log2n, q[l], psis[l], halving, &lc32[l], &twf32[(size_t)l * n],
                             &twi32[(size_t)l * n]);
    for (uint32_t l = nlimbs; l < nlc; ++l) pm::host::fused_limb32(lc32[l - nlimbs], &lc32[l]);
    h_lc = lc32.data();
    h_twf = twf32.data();
    h_twi = twi32.data();
    lc_bytes = nlc * sizeof(pm::LimbConst32);
    tw_bytes = (size_t)nlimbs * n * sizeof(pm::TwPair32);
  } else {
    lc.resize(nlc);
    twf.resize((size_t)nlimbs * n);
    twi.resize((size_t)nlimbs * n);
    for (uint32_t l = 0; l < nlimbs; ++l)
      pm::host::build_limb(log2n, q[l], psis[l], halving, &lc[l], &twf[(size_t)l * n],
                           &twi[(size_t)l * n]);
    for (uint32_t l = nlimbs; l < nlc; ++l) pm::host::fused_limb(lc[l - nlimbs], &lc[l]);
    h_lc = lc.data();
    h_twf = twf.data();
    h_twi = twi.data();
    lc_bytes = nlc * sizeof(pm::LimbConst);
    tw_bytes = (size_t)nlimbs * n * sizeof(pm::TwPair);
  }
  void *d_lc = nullptr, *d_twf = nullptr, *d_twi = nullptr;
  e = cudaMalloc(&d_lc, lc_bytes);
  p->d_lc = (pm::LimbConst*)d_lc;
  if (e == cudaSuccess) e = cudaMalloc(&d_twf, tw_bytes);
  p->d_twf = (pm::TwPair*)d_twf;
  if (e == cudaSuccess) e = cudaMalloc(&d_twi, tw_bytes);
  p->d_twi = (pm::TwPair*)d_twi;
  if (e == cudaSuccess) e = cudaMalloc(&p->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e, "cudaMalloc(plan tables)");
  }
  if ((e = cudaMemcpy(d_lc, h_lc, lc_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d_twf, h_twf, tw_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d_twi, h_twi, tw_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e, "cudaMemcpy(plan tables)");
  }
  *out = p;
  return ok();
}

pm_status pm_plan_destroy(pm_plan* plan) {
  destroy_plan(plan);
  return ok();
}

pm_status pm_plan_flags(const pm_plan* plan, uint32_t* flags) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (!flags) return fail(PM_ERR_ARG, "flags is NULL");
  *flags = plan->flags;
  return ok();
}

pm_status pm_plan_info(const pm_plan* plan, uint32_t* log2n, uint32_t* nlimbs, uint64_t* q_out,
                       uint64_t* psi_out) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (log2n) *log2n = plan->logn;
  if (nlimbs) *nlimbs = plan->nlimbs;
  for (uint32_t l = 0; l < plan->nlimbs; ++l) {
    if (q_out) q_out[l] = plan->q[l];
    if (psi_out) psi_out[l] = plan->psi[l];
  }
  return ok();
}

pm_status pm_plan_reserve(pm_plan* plan, uint32_t npoly, void* stream) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  if (!pm::polymul_needs_scratch(plan->logn)) return ok();
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  std::lock_guard<std::mutex> lk(plan->mu);
  uint64_t* ptr = nullptr;
  s = ensure_scratch(plan, (cudaStream_t)stream, (uint64_t)npoly * plan->nlimbs, &ptr);
  return s == PM_OK ? ok() : s;
}

pm_status pm_ntt_fwd(const pm_plan* plan, uint64_t* d_x, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_ntt_fwd");
  if (s != PM_OK) return s;
  if (!d_x || !aligned16(d_x)) return fail(PM_ERR_ARG, "d_x NULL or not 16-byte aligned");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm::KParams P = base_params(plan, npoly);
  P.a = d_x;
  P.c = d_x;
  cudaError_t e = pm::launch_ntt_fwd(P, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ntt_fwd launch");
  return ok();
}

pm_status pm_ntt_inv(const pm_plan* plan, uint64_t* d_x, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_ntt_inv");
  if (s != PM_OK) return s;
  if (!d_x || !aligned16(d_x)) return fail(PM_ERR_ARG, "d_x NULL or not 16-byte aligned");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm::KParams P = base_params(plan, npoly);
  P.a = d_x;
  P.c = d_x;
  cudaError_t e = pm::launch_ntt_inv(P, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ntt_inv launch");
  return ok();
}

pm_status pm_pointwise(const pm_plan* plan, const uint64_t* d_a, const uint64_t* d_b,
                       uint64_t* d_c, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_pointwise");
  if (s != PM_OK) return s;
  if (!d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm::KParams P = base_params(plan, npoly);
  P.a = d_a;
  P.b = d_b;
  P.c = d_c;
  cudaError_t e = pm::launch_pointwise(P, (cudaStream_t)stream, plan->num_sms);
  if (e != cudaSuccess) return cuda_fail(e, "pointwise launch");
  return ok();
}

pm_status pm_polymul(const pm_plan* plan, const uint64_t* d_a, const uint64_t* d_b,
                     uint64_t* d_c, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_polymul");
  if (s != PM_OK) return s;
  if (!d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_plan* p = const_cast<pm_plan*>(plan);
  std::lock_guard<std::mutex> lk(p->mu);
  s = polymul_impl(p, d_a, d_b, d_c, npoly, (cudaStream_t)stream);
  return s == PM_OK ? ok() : s;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free polymul.  Callers that must not allocate device memory
// (for example code running while another component owns the device
// memory pool, or latency-critical code that cannot accept the device-wide
// synchronisation of cudaFree) use this entry point instead of pm_polymul:
// the column-split path's scratch lives in the fixed array below, which is
// part of the library image and exists on every device that loads it.
constexpr uint64_t kNoAllocScratchWords = (uint64_t)1 << 21;  // 16 MiB

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocScratchWords];

namespace {

std::mutex g_noalloc_mu;
std::vector<std::pair<int, uint64_t*>> g_noalloc_ptr;  // device -> device address

// Device address of g_noalloc_scratch on the current device `dev`, looked up
// once per device.  In host code the array's name is only a host-side
// stand-in, so the kernels must be given this looked-up address.
pm_status noalloc_scratch(int dev, uint64_t** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  for (auto& e : g_noalloc_ptr)
    if (e.first == dev) {
      *out = e.second;
      return PM_OK;
    }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  g_noalloc_ptr.emplace_back(dev, (uint64_t*)ptr);
  *out = (uint64_t*)ptr;
  return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_polymul_noalloc(const pm_plan* plan, const uint64_t* d_a, const uint64_t* d_b,
                             uint64_t* d_c, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_polymul_noalloc");
  if (s != PM_OK) return s;
  if (!d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  pm::KParams P;
  {
    // the launch choice (plan->tune) is read under the plan's lock, since
    // pm_plan_tune / pm_plan_autotune may rewrite it from another thread
    std::lock_guard<std::mutex> lk(const_cast<pm_plan*>(plan)->mu);
    P = base_params(plan, npoly);
  }
  P.a = d_a;
  P.b = d_b;
  P.c = d_c;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if (pm::polymul_writes_scratch(P)) {
    const uint64_t words = (uint64_t)P.nunits << plan->logn;
    if (words > kNoAllocScratchWords)
      return fail(PM_ERR_ARG,
                  "pm_polymul_noalloc: batch needs %llu scratch words, the static area holds "
                  "%llu (npoly * nlimbs * N <= 2^21)",
                  (unsigned long long)words, (unsigned long long)kNoAllocScratchWords);
    s = noalloc_scratch(plan->device, &P.s);
    if (s != PM_OK) return s;
  }
  cudaError_t e = pm::launch_polymul(P, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "polymul launch");
  return ok();
}

pm_status pm_polymul_host(const pm_plan* plan, const uint64_t* h_a, const uint64_t* h_b,
                          uint64_t* h_c, uint64_t* d_a, uint64_t* d_b, uint64_t* d_c,
                          uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_polymul_host");
  if (s != PM_OK) return s;
  if (!h_a || !h_b || !h_c || !d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) ||
      !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_plan* p = const_cast<pm_plan*>(plan);
  std::lock_guard<std::mutex> lk(p->mu);
  cudaError_t e;
  if (!p->side_in) {
    if ((e = cudaStreamCreateWithFlags(&p->side_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&p->side_out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->ev_end, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "pipeline streams");
    for (int i = 0; i < kHostChunks; ++i)
      if ((e = cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "pipeline events");
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t* scratch = nullptr;
  if (pm::polymul_needs_scratch(p->logn)) {
    s = ensure_scratch(p, st, (uint64_t)npoly * p->nlimbs, &scratch);
    if (s != PM_OK) return s;
  }
  const size_t poly_words = (size_t)p->nlimbs << p->logn;
  const uint32_t nchunks = npoly < (uint32_t)kHostChunks ? npoly : (uint32_t)kHostChunks;
  // the side streams start after work already queued on `st`
  if ((e = cudaEventRecord(p->ev_start, st)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(p->side_in, p->ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(p->side_out, p->ev_start, 0)) != cudaSuccess)
    return cuda_fail(e, "pipeline start");
  uint32_t done = 0;
  for (uint32_t k = 0; k < nchunks; ++k) {
    const uint32_t cnt = (npoly - done) / (nchunks - k);
    const size_t off = (size_t)done * poly_words, bytes = (size_t)cnt * poly_words * 8;
    if ((e = cudaMemcpyAsync(d_a + off, h_a + off, bytes, cudaMemcpyHostToDevice, p->side_in)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(d_b + off, h_b + off, bytes, cudaMemcpyHostToDevice, p->side_in)) !=
            cudaSuccess ||
        (e = cudaEventRecord(p->ev_in[k], p->side_in)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, p->ev_in[k], 0)) != cudaSuccess)
      return cuda_fail(e, "pipeline copy-in");
    // the scratch is indexed from unit 0 of each launch; chunks run in order on `st`
    (void)scratch;
    if ((s = polymul_impl(p, d_a + off, d_b + off, d_c + off, cnt, st)) != PM_OK) return s;
    if ((e = cudaEventRecord(p->ev_done[k], st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->side_out, p->ev_done[k], 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h_c + off, d_c + off, bytes, cudaMemcpyDeviceToHost, p->side_out)) !=
            cudaSuccess)
      return cuda_fail(e, "pipeline copy-out");
    done += cnt;
  }
  if ((e = cudaEventRecord(p->ev_end, p->side_out)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, p->ev_end, 0)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "pipeline end");
  return ok();
}

pm_status pm_check_reduced(const pm_plan* plan, const uint64_t* d_x, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, false, "pm_check_reduced");
  if (s != PM_OK) return s;
  if (!d_x) return fail(PM_ERR_ARG, "d_x is NULL");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_plan* p = const_cast<pm_plan*>(plan);
  std::lock_guard<std::mutex> lk(p->mu);
  cudaStream_t st = (cudaStream_t)stream;
  pm::KParams P = base_params(p, npoly);
  P.a = d_x;
  int flag = 0;
  cudaError_t e;
  if ((e = cudaMemsetAsync(p->d_flag, 0, sizeof(int), st)) != cudaSuccess ||
      (e = pm::launch_check_reduced(P, p->d_flag, st, p->num_sms)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "check_reduced");
  if (flag) return fail(PM_ERR_RANGE, "a coefficient is >= its modulus");
  return ok();
}

// ---- 32-bit words (PM_PLAN_WORD32): the same calls on uint32_t arrays.
pm_status pm_ntt_fwd32(const pm_plan* plan, uint32_t* d_x, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, true, "pm_ntt_fwd32");
  if (s != PM_OK) return s;
  if (!d_x || !aligned16(d_x)) return fail(PM_ERR_ARG, "d_x NULL or not 16-byte aligned");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm::KParams P = base_params(plan, npoly);
  P.a = reinterpret_cast<const uint64_t*>(d_x);
  P.c = reinterpret_cast<uint64_t*>(d_x);
  cudaError_t e = pm::launch_ntt_fwd(P, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ntt_fwd32 launch");
  return ok();
}

pm_status pm_ntt_inv32(const pm_plan* plan, uint32_t* d_x, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, true, "pm_ntt_inv32");
  if (s != PM_OK) return s;
  if (!d_x || !aligned16(d_x)) return fail(PM_ERR_ARG, "d_x NULL or not 16-byte aligned");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm::KParams P = base_params(plan, npoly);
  P.a = reinterpret_cast<const uint64_t*>(d_x);
  P.c = reinterpret_cast<uint64_t*>(d_x);
  cudaError_t e = pm::launch_ntt_inv(P, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ntt_inv32 launch");
  return ok();
}

pm_status pm_pointwise32(const pm_plan* plan, const uint32_t* d_a, const uint32_t* d_b,
                         uint32_t* d_c, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, true, "pm_pointwise32");
  if (s != PM_OK) return s;
  if (!d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm::KParams P = base_params(plan, npoly);
  P.a = reinterpret_cast<const uint64_t*>(d_a);
  P.b = reinterpret_cast<const uint64_t*>(d_b);
  P.c = reinterpret_cast<uint64_t*>(d_c);
  cudaError_t e = pm::launch_pointwise(P, (cudaStream_t)stream, plan->num_sms);
  if (e != cudaSuccess) return cuda_fail(e, "pointwise32 launch");
  return ok();
}

pm_status pm_polymul32(const pm_plan* plan, const uint32_t* d_a, const uint32_t* d_b,
                       uint32_t* d_c, uint32_t npoly, void* stream) {
  pm_status s = check_plan_word(plan, true, "pm_polymul32");
  if (s != PM_OK) return s;
  if (!d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_plan* p = const_cast<pm_plan*>(plan);
  std::lock_guard<std::mutex> lk(p->mu);
  s = polymul_impl(p, reinterpret_cast<const uint64_t*>(d_a),
                   reinterpret_cast<const uint64_t*>(d_b), reinterpret_cast<uint64_t*>(d_c), npoly,
                   (cudaStream_t)stream);
  return s == PM_OK ? ok() : s;
}

pm_status pm_check_reduced32(const pm_plan* plan, const uint32_t* d_x, uint32_t npoly,
                             void* stream) {
  pm_status s = check_plan_word(plan, true, "pm_check_reduced32");
  if (s != PM_OK) return s;
  if (!d_x) return fail(PM_ERR_ARG, "d_x is NULL");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_plan* p = const_cast<pm_plan*>(plan);
  std::lock_guard<std::mutex> lk(p->mu);
  cudaStream_t st = (cudaStream_t)stream;
  pm::KParams P = base_params(p, npoly);
  P.a = reinterpret_cast<const uint64_t*>(d_x);
  int flag = 0;
  cudaError_t e;
  if ((e = cudaMemsetAsync(p->d_flag, 0, sizeof(int), st)) != cudaSuccess ||
      (e = pm::launch_check_reduced(P, p->d_flag, st, p->num_sms)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "check_reduced32");
  if (flag) return fail(PM_ERR_RANGE, "a coefficient is >= its modulus");
  return ok();
}

pm_status pm_plan_set_phase_events(pm_plan* plan, void* const* events, int n) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (n < 0 || n > 4 || (n > 0 && !events)) return fail(PM_ERR_ARG, "n must be 0..4");
  std::lock_guard<std::mutex> lk(plan->mu);
  plan->phase.n = n;
  for (int k = 0; k < n; ++k) plan->phase.ev[k] = (cudaEvent_t)events[k];
  return ok();
}

pm_status pm_plan_sync(const pm_plan* plan, void* stream) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "device error");
  // a persistent launch on this stream that gave up waiting leaves a flag
  pm_plan* p = const_cast<pm_plan*>(plan);
  std::lock_guard<std::mutex> lk(p->mu);
  int rflag = 0;
  if ((e = cudaMemcpy(&rflag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read status");
  if (rflag) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return fail(PM_ERR_TIMEOUT, "a row kernel gave up waiting for its staged twiddles");
  }
  for (auto& sc : p->scratch) {
    if (sc.stream != (cudaStream_t)stream || !sc.ctl) continue;
    uint32_t flag = 0;
    if ((e = cudaMemcpy(&flag, sc.ctl + 1, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "read status");
    if (flag) {
      cudaMemset(sc.ctl + 1, 0, 4);
      return fail(PM_ERR_TIMEOUT, "a persistent launch gave up waiting for a dependency");
    }
  }
  return ok();
}

pm_status pm_plan_tune(pm_plan* plan, const pm_tuning* t) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (!t) return fail(PM_ERR_ARG, "tuning is NULL");
  if (t->variant != PM_VARIANT_SPLIT && t->variant != PM_VARIANT_PERSISTENT)
    return fail(PM_ERR_ARG, "unknown variant %d", t->variant);
  if (t->row_ops > 5) return fail(PM_ERR_ARG, "row_ops must be 0..5");
  if (t->variant == PM_VARIANT_PERSISTENT && is_word32(plan))
    return fail(PM_ERR_ARG, "the persistent variant takes 64-bit plans");
  if (t->variant == PM_VARIANT_PERSISTENT &&
      (t->ctas_per_sm < 1 || t->ctas_per_sm > 4 || t->lag_fwd < 1 || t->lag_inv <= t->lag_fwd ||
       t->lag_inv > 4096))
    return fail(PM_ERR_ARG, "persistent tuning needs 1 <= ctas_per_sm <= 4, 1 <= lag_fwd < lag_inv <= 4096");
  std::lock_guard<std::mutex> lk(plan->mu);
  plan->tune = *t;
  return ok();
}

pm_status pm_plan_autotune(pm_plan* plan, uint32_t npoly, void* stream, pm_tuning* best_out,
                           float* best_ms_out) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard g(plan->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  // candidates: the split path with each row kernel (4096-word rows: the
  // two-operand, one-operand and 1024-thread kernels; 1024-word rows), the
  // persistent launch with a few pipeline distances
  std::vector<pm_tuning> cand;
  cand.push_back(pm_tuning{PM_VARIANT_SPLIT, 3, 8, 64, 2});
  if (plan->logn >= 12 && plan->logn != 13) {
    cand.push_back(pm_tuning{PM_VARIANT_SPLIT, 3, 8, 64, 1});
    cand.push_back(pm_tuning{PM_VARIANT_SPLIT, 3, 8, 64, 3});
  }
  if (pm::wide_polymul_ok(plan->logn)) cand.push_back(pm_tuning{PM_VARIANT_SPLIT, 3, 8, 64, 4});
  if (plan->logn >= 13 && !is_word32(plan)) {
    cand.push_back(pm_tuning{PM_VARIANT_PERSISTENT, 3, 8, 64, 1});
    cand.push_back(pm_tuning{PM_VARIANT_PERSISTENT, 3, 16, 128, 1});
    if (pm::wpersist_ok(plan->logn) && !(plan->flags & PM_PLAN_HALVING)) {
      cand.push_back(pm_tuning{PM_VARIANT_PERSISTENT, 4, 8, 32, 4});
      cand.push_back(pm_tuning{PM_VARIANT_PERSISTENT, 4, 32, 64, 4});
    }
  }
  const size_t words = (size_t)npoly * plan->nlimbs << plan->logn;
  uint64_t *a = nullptr, *b = nullptr, *c = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  pm_tuning best = plan->tune;
  float best_ms = 1e30f;
  if ((e = cudaMalloc(&a, words * 8)) != cudaSuccess || (e = cudaMalloc(&b, words * 8)) != cudaSuccess ||
      (e = cudaMalloc(&c, words * 8)) != cudaSuccess || (e = cudaMemsetAsync(a, 0, words * 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b, 0, words * 8, st)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
      (e = cudaEventCreate(&e1)) != cudaSuccess) {
    s = cuda_fail(e, "autotune buffers");
  } else {
    std::lock_guard<std::mutex> lk(plan->mu);
    const pm_tuning saved = plan->tune;
    for (const pm_tuning& t : cand) {
      plan->tune = t;
      float times[5];
      for (int r = 0; r < 7 && s == PM_OK; ++r) {
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { s = cuda_fail(e, "event"); break; }
        if ((s = polymul_impl(plan, a, b, c, npoly, st)) != PM_OK) break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
          s = cuda_fail(e, "event");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r >= 2) times[r - 2] = ms;  // two warm-up runs
      }
      if (s != PM_OK) break;
      std::sort(times, times + 5);
      if (times[2] < best_ms) {
        best_ms = times[2];
        best = t;
      }
    }
    plan->tune = (s == PM_OK) ? best : saved;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  cudaFree(c);
  if (s != PM_OK) return s;
  if (best_out) *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return ok();
}

pm_status pm_plan_inject_fault(pm_plan* plan, int kind) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (kind != 0 && kind != PM_FAULT_WITHHOLD_SIGNAL && kind != PM_FAULT_SHORT_TWIDDLES)
    return fail(PM_ERR_ARG, "unknown fault %d", kind);
  std::lock_guard<std::mutex> lk(plan->mu);
  plan->inject = kind;
  return ok();
}

pm_status pm_plan_get_tuning(const pm_plan* plan, pm_tuning* t) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (!t) return fail(PM_ERR_ARG, "tuning is NULL");
  *t = plan->tune;
  return ok();
}

pm_status pm_plan_resolve_tuning(const pm_plan* plan, uint32_t npoly, pm_tuning* t) {
  pm_status s = check_plan(plan);
  if (s != PM_OK) return s;
  if (!t) return fail(PM_ERR_ARG, "tuning is NULL");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  *t = plan->tune;
  t->row_ops = base_params(plan, npoly).row_ops;  // the same rule as the launch
  return ok();
}


}  // extern "C"

// ---------------------------------------------------------------- uneven batch

// Uneven batches with at least this many 4096-word rows per SM take the
// grouped split launches under PM_UNEVEN_AUTO.
constexpr uint64_t kGroupedMinRows = 8;

struct pm_queue {
  int device = 0;
  int num_sms = 0;
  std::mutex mu;
  pm::UnitDesc* d_units = nullptr;
  uint32_t* d_pre = nullptr;  // [3][cap]
  uint32_t* d_ctl = nullptr;  // [4 + 2 cap]
  size_t cap = 0;
  uint64_t* d_scratch = nullptr;
  size_t scratch_words = 0;
  pm::UnitDesc* h_units = nullptr;  // pinned staging
  uint32_t* h_pre = nullptr;
  size_t h_cap = 0;
  cudaEvent_t staged = nullptr;  // the last upload from the staging buffers
  bool staged_used = false;
  int mode = 0;  // PM_UNEVEN_AUTO / _PERSISTENT / _GROUPED
};

namespace {

void destroy_queue(pm_queue* q) {
  if (!q) return;
  DeviceGuard g(q->device);
  cudaFree(q->d_units);
  cudaFree(q->d_pre);
  cudaFree(q->d_ctl);
  cudaFree(q->d_scratch);
  cudaFreeHost(q->h_units);
  cudaFreeHost(q->h_pre);
  if (q->staged) cudaEventDestroy(q->staged);
  delete q;
}

// Words of the prefix buffer per unit of capacity: three prefix counts, then
// the 1024-word kernel's block tables (one entry per 32 tickets of a
// section: at most 224 tickets per unit, 7 entries, plus one per section).
constexpr size_t kPreWords = 3 + 8;

pm_status queue_reserve(pm_queue* q, size_t units, size_t scratch_words) {
  cudaError_t e;
  if (units > q->cap) {
    if (q->staged_used && (e = cudaEventSynchronize(q->staged)) != cudaSuccess)
      return cuda_fail(e, "queue staging");
    cudaFree(q->d_units);
    cudaFree(q->d_pre);
    cudaFree(q->d_ctl);
    cudaFreeHost(q->h_units);
    cudaFreeHost(q->h_pre);
    q->d_units = nullptr;
    q->d_pre = q->d_ctl = nullptr;
    q->h_units = nullptr;
    q->h_pre = nullptr;
    q->cap = q->h_cap = 0;
    const size_t cap = units < 256 ? 256 : units;
    if ((e = cudaMalloc(&q->d_units, cap * sizeof(pm::UnitDesc))) != cudaSuccess ||
        (e = cudaMalloc(&q->d_pre, kPreWords * cap * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc(&q->d_ctl, (4 + 2 * cap) * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMallocHost(&q->h_units, cap * sizeof(pm::UnitDesc))) != cudaSuccess ||
        (e = cudaMallocHost(&q->h_pre, kPreWords * cap * sizeof(uint32_t))) != cudaSuccess)
      return cuda_fail(e, "queue buffers");
    if ((e = cudaMemset(q->d_ctl, 0, (4 + 2 * cap) * sizeof(uint32_t))) != cudaSuccess)
      return cuda_fail(e, "queue ctl");
    q->cap = q->h_cap = cap;
    q->staged_used = false;
  }
  if (scratch_words > q->scratch_words) {
    cudaFree(q->d_scratch);
    q->d_scratch = nullptr;
    q->scratch_words = 0;
    if ((e = cudaMalloc(&q->d_scratch, scratch_words * 8)) != cudaSuccess)
      return cuda_fail(e, "queue scratch");
    q->scratch_words = scratch_words;
  }
  return PM_OK;
}

}  // namespace

// The uneven launch.  ext_scratch[j], when given, is job j's own column-stage
// scratch (npoly * nlimbs * N words, for N >= 2^13 and a != b); otherwise the
// queue's scratch is used.  The caller holds q->mu with q's device current.
pm_status uneven_impl(pm_queue* q, const pm_job* jobs, uint32_t njobs, uint64_t* const* ext_scratch,
                      cudaStream_t st) {
  if (!q) return fail(PM_ERR_ARG, "queue is NULL");
  if (njobs == 0) return ok();
  if (!jobs) return fail(PM_ERR_ARG, "jobs is NULL");
  // validate and size
  uint64_t units = 0, scratch = 0;
  int halving = -1, fused = -1;
  bool lazy16 = true;
  for (uint32_t j = 0; j < njobs; ++j) {
    const pm_job& J = jobs[j];
    if (!J.plan) return fail(PM_ERR_ARG, "job %u: plan is NULL", j);
    if (J.plan->device != q->device)
      return fail(PM_ERR_ARG, "job %u: plan on device %d, queue on %d", j, J.plan->device, q->device);
    if (is_word32(J.plan)) return fail(PM_ERR_ARG, "job %u: uneven batches take 64-bit plans", j);
    if (J.npoly == 0) return fail(PM_ERR_ARG, "job %u: npoly is 0", j);
    if (!J.a || !J.b || !J.c || !aligned16(J.a) || !aligned16(J.b) || !aligned16(J.c))
      return fail(PM_ERR_ARG, "job %u: NULL or misaligned pointer", j);
    if (J.plan->logn < 12) continue;  // run through the plan's own path below
    const int h = (J.plan->flags & PM_PLAN_HALVING) ? 1 : 0;
    if (halving >= 0 && h != halving)
      return fail(PM_ERR_ARG, "jobs mix PM_PLAN_HALVING and default plans");
    halving = h;
    const int f = (J.plan->flags & PM_PLAN_FUSED) ? 1 : 0;
    if (fused >= 0 && f != fused)
      return fail(PM_ERR_ARG, "jobs mix PM_PLAN_FUSED and default plans");
    fused = f;
    lazy16 = lazy16 && J.plan->lazy16;
    const uint64_t u = (uint64_t)J.npoly * J.plan->nlimbs;
    units += u;
    // N = 2^12 units need b's image too on the 1024-word persistent path
    if (J.plan->logn >= 12 && J.a != J.b && !(ext_scratch && ext_scratch[j]))
      scratch += u << J.plan->logn;
  }
  if (units > 0x3fffffffull) return fail(PM_ERR_ARG, "too many units (%llu)", (unsigned long long)units);
  cudaError_t e;
  // small-N jobs: their plan's own path, on the same stream
  for (uint32_t j = 0; j < njobs; ++j) {
    const pm_job& J = jobs[j];
    if (J.plan->logn >= 12) continue;
    pm_plan* p = const_cast<pm_plan*>(J.plan);
    std::lock_guard<std::mutex> lp(p->mu);
    pm_status s2 = polymul_impl(p, J.a, J.b, J.c, J.npoly, st);
    if (s2 != PM_OK) return s2;
  }
  if (units == 0) return ok();
  pm_status s = queue_reserve(q, units, scratch ? scratch : 1);
  if (s != PM_OK) return s;
  // grouped split launches for large batches (each N's units through the
  // column and row kernels of the uniform path), the persistent work queue
  // for small ones (its overlap of the three phases matters there)
  uint64_t rows_total = 0;
  for (uint32_t j = 0; j < njobs; ++j)
    if (jobs[j].plan->logn >= 12)
      rows_total += ((uint64_t)jobs[j].npoly * jobs[j].plan->nlimbs) << (jobs[j].plan->logn - 12);
  const bool grouped = q->mode == PM_UNEVEN_GROUPED ||
                       (q->mode == PM_UNEVEN_AUTO && rows_total >= kGroupedMinRows * (uint64_t)q->num_sms);
  // one persistent launch: the 1024-word tasks unless the plans halve at
  // every inverse stage (then the 4096-word tasks)
  const bool wide = !grouped && halving != 1;
  if (q->staged_used && (e = cudaEventSynchronize(q->staged)) != cudaSuccess)
    return cuda_fail(e, "queue staging");
  // unit descriptors and section prefix counts
  uint32_t* pf = q->h_pre;
  uint32_t* pw = q->h_pre + units;
  uint32_t* pi = q->h_pre + 2 * units;
  uint32_t tf = 0, tw = 0, ti = 0;
  uint64_t soff = 0;
  size_t u = 0;
  for (uint32_t j = 0; j < njobs; ++j) {
    const pm_job& J = jobs[j];
    const pm_plan* p = J.plan;
    if (p->logn < 12) continue;
    const uint64_t n = (uint64_t)1 << p->logn;
    const bool split = p->logn > 12 || wide;
    const bool square = J.a == J.b;
    uint64_t* own = (ext_scratch && ext_scratch[j]) ? ext_scratch[j] : nullptr;
    for (uint32_t k = 0; k < J.npoly * p->nlimbs; ++k, ++u) {
      pm::UnitDesc& D = q->h_units[u];
      const uint32_t limb = k % p->nlimbs;
      D.a = J.a + k * n;
      D.b = J.b + k * n;
      D.c = J.c + k * n;
      if (split && !square) {
        if (own) {
          D.s = own + k * n;
        } else {
          D.s = q->d_scratch + soff;
          soff += n;
        }
        if (J.c == J.b) std::swap(D.a, D.b);  // b's image stays in place in c
      } else {
        D.s = D.c;
      }
      D.twf = p->d_twf + ((size_t)limb << p->logn);
      D.twi = p->d_twi + ((size_t)limb << p->logn);
      D.lc = p->d_lc + limb + ((p->flags & PM_PLAN_FUSED) ? p->nlimbs : 0);
      D.logn = p->logn;
      D.pad = 0;
      pf[u] = tf;
      pw[u] = tw;
      pi[u] = ti;
      if (wide) {
        uint32_t f, w, i;
        pm::wuneven_tasks(p->logn, square, &f, &w, &i);
        tf += f;
        tw += w;
        ti += i;
      } else {
        tf += split ? (square ? 1u : 2u) * 16u : 0u;
        tw += (uint32_t)(n >> 12);
        ti += split ? 16u : 0u;
      }
    }
  }
  if (grouped) {
    // units sorted by N (stable), one grouped launch per N
    std::vector<pm::UnitDesc> sorted(units);
    uint32_t count[18] = {0}, start[18] = {0};
    for (size_t i = 0; i < units; ++i) count[q->h_units[i].logn]++;
    for (int L = 13; L < 18; ++L) start[L] = start[L - 1] + count[L - 1];
    for (size_t i = 0; i < units; ++i) sorted[start[q->h_units[i].logn]++] = q->h_units[i];
    std::copy(sorted.begin(), sorted.end(), q->h_units);
    if ((e = cudaMemcpyAsync(q->d_units, q->h_units, units * sizeof(pm::UnitDesc),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaEventRecord(q->staged, st)) != cudaSuccess)
      return cuda_fail(e, "queue upload");
    q->staged_used = true;
    size_t first = 0;
    for (int L = 12; L < 18; ++L) {
      if (!count[L]) continue;
      pm::KParams P{};
      P.desc = q->d_units + first;
      P.nunits = count[L];
      P.nlimbs = 1;
      P.logn = (uint32_t)L;
      P.halving = (uint32_t)halving;
      P.fused = (uint32_t)fused;
      P.lazy16 = lazy16 ? 1 : 0;
      P.err = reinterpret_cast<int*>(q->d_ctl + 1);  // reported by pm_queue_sync
      // N >= 2^13: the 1024-word split (measured faster at every batch
      // size); N = 2^12: whole 4096-word rows with the two-operand kernel
      P.row_ops = L >= 13 ? 4 : 2;
      if ((e = pm::launch_polymul_grouped(P, st)) != cudaSuccess)
        return cuda_fail(e, "grouped uneven launch");
      first += count[L];
    }
    return ok();
  }
  // the 1024-word kernel's block tables: per section, the unit holding every
  // 32nd ticket (all units have tickets in every section)
  size_t nblk[3] = {0, 0, 0};
  if (wide) {
    const uint32_t* pres[3] = {pf, pw, pi};
    const uint32_t tot[3] = {tf, tw, ti};
    uint32_t* blk = q->h_pre + 3 * units;
    for (int sec = 0; sec < 3; ++sec) {
      nblk[sec] = (tot[sec] + 31) / 32;
      size_t uu = 0;
      for (size_t i = 0; i < nblk[sec]; ++i) {
        const uint32_t x = (uint32_t)(32 * i);
        while (uu + 1 < units && pres[sec][uu + 1] <= x) ++uu;
        blk[i] = (uint32_t)uu;
      }
      blk += nblk[sec];
    }
  }
  const size_t pre_words = 3 * units + nblk[0] + nblk[1] + nblk[2];
  // the prefix arrays (f, w, i) and block tables are uploaded contiguously
  if ((e = cudaMemcpyAsync(q->d_units, q->h_units, units * sizeof(pm::UnitDesc),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(q->d_pre, q->h_pre, pre_words * sizeof(uint32_t), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess ||
      (e = cudaEventRecord(q->staged, st)) != cudaSuccess)
    return cuda_fail(e, "queue upload");
  q->staged_used = true;
  pm::UnevenArgs A{};
  A.units = q->d_units;
  A.pre_f = q->d_pre;
  A.pre_w = q->d_pre + units;
  A.pre_i = q->d_pre + 2 * units;
  A.ctl = q->d_ctl;
  A.nunits = (uint32_t)units;
  A.tf = tf;
  A.tw = tw;
  A.ti = ti;
  A.blk_f = q->d_pre + 3 * units;
  A.blk_w = A.blk_f + nblk[0];
  A.blk_i = A.blk_w + nblk[1];
  if (wide)
    e = pm::launch_wuneven(A, lazy16, fused == 1, q->num_sms * pm::wpersist_ctas_per_sm(0), st);
  else
    e = pm::launch_uneven(A, halving == 1, fused == 1, q->num_sms * 3, st);
  if (e != cudaSuccess) return cuda_fail(e, "uneven launch");
  return ok();
}


extern "C" {

pm_status pm_queue_create(pm_queue** out, int device) {
  if (!out) return fail(PM_ERR_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(PM_ERR_ARG, "device %d not present", device);
  DeviceGuard g(device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_queue* q = new (std::nothrow) pm_queue();
  if (!q) return fail(PM_ERR_OOM, "host allocation failed");
  q->device = device;
  if ((e = cudaDeviceGetAttribute(&q->num_sms, cudaDevAttrMultiProcessorCount, device)) !=
          cudaSuccess ||
      (e = prepare_device(device)) != cudaSuccess || (e = pm::persist_prepare()) != cudaSuccess ||
      (e = pm::uneven_prepare()) != cudaSuccess || (e = pm::wpersist_prepare()) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&q->staged, cudaEventDisableTiming)) != cudaSuccess) {
    destroy_queue(q);
    return cuda_fail(e, "queue setup");
  }
  *out = q;
  return ok();
}

pm_status pm_queue_set_mode(pm_queue* q, int mode) {
  if (!q) return fail(PM_ERR_ARG, "queue is NULL");
  if (mode < PM_UNEVEN_AUTO || mode > PM_UNEVEN_GROUPED) return fail(PM_ERR_ARG, "mode must be 0..2");
  std::lock_guard<std::mutex> lk(q->mu);
  q->mode = mode;
  return ok();
}

pm_status pm_queue_destroy(pm_queue* q) {
  destroy_queue(q);
  return ok();
}

pm_status pm_queue_reserve(pm_queue* q, uint64_t units, uint64_t scratch_words) {
  if (!q) return fail(PM_ERR_ARG, "queue is NULL");
  DeviceGuard g(q->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  std::lock_guard<std::mutex> lk(q->mu);
  pm_status s = queue_reserve(q, units, scratch_words);
  return s == PM_OK ? ok() : s;
}

pm_status pm_polymul_uneven(pm_queue* q, const pm_job* jobs, uint32_t njobs, void* stream) {
  if (!q) return fail(PM_ERR_ARG, "queue is NULL");
  DeviceGuard g(q->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  std::lock_guard<std::mutex> lk(q->mu);
  return uneven_impl(q, jobs, njobs, nullptr, (cudaStream_t)stream);
}

pm_status pm_queue_sync(pm_queue* q, void* stream) {
  if (!q) return fail(PM_ERR_ARG, "queue is NULL");
  DeviceGuard g(q->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  std::lock_guard<std::mutex> lk(q->mu);
  if (q->d_ctl) {
    uint32_t flag = 0;
    if ((e = cudaMemcpy(&flag, q->d_ctl + 1, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "read status");
    if (flag) {
      cudaMemset(q->d_ctl + 1, 0, 4);
      return fail(PM_ERR_TIMEOUT, "the uneven launch gave up waiting for a dependency");
    }
  }
  return ok();
}

}  // extern "C"

// ----------------------------------------------------------------- graphs

struct pm_graph {
  int device = 0;
  uint64_t* scratch = nullptr;
  uint32_t* ctl = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
void destroy_graph(pm_graph* g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFree(g->scratch);
  cudaFree(g->ctl);
  delete g;
}
}  // namespace

extern "C" {

pm_status pm_graph_create_polymul(pm_graph** out, const pm_plan* plan, const uint64_t* d_a,
                                  const uint64_t* d_b, uint64_t* d_c, uint32_t npoly) {
  if (!out) return fail(PM_ERR_ARG, "out is NULL");
  *out = nullptr;
  pm_status s = check_plan_word(plan, false, "pm_graph_create_polymul");
  if (s != PM_OK) return s;
  if (!d_a || !d_b || !d_c || !aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c))
    return fail(PM_ERR_ARG, "NULL or misaligned pointer");
  if ((s = check_batch(plan, npoly)) != PM_OK) return s;
  DeviceGuard dg(plan->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  pm_graph* g = new (std::nothrow) pm_graph();
  if (!g) return fail(PM_ERR_OOM, "host allocation failed");
  g->device = plan->device;
  pm::KParams P = base_params(plan, npoly);
  P.a = d_a;
  P.b = d_b;
  P.c = d_c;
  const bool persistent = use_persistent(plan);
  cudaError_t e = cudaSuccess;
  if (pm::polymul_needs_scratch(plan->logn) || (persistent && plan->logn >= 13)) {
    if ((e = cudaMalloc(&g->scratch, (size_t)P.nunits << plan->logn << 3)) != cudaSuccess) {
      destroy_graph(g);
      return cuda_fail(e, "cudaMalloc(graph scratch)");
    }
    P.s = g->scratch;
  }
  if (persistent &&
      (e = cudaMalloc(&g->ctl, pm::persist_ctl_words(P.nunits) * 4)) != cudaSuccess) {
    destroy_graph(g);
    return cuda_fail(e, "cudaMalloc(graph ctl)");
  }
  cudaStream_t cap = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
    destroy_graph(g);
    return cuda_fail(e, "capture stream");
  }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le =
        persistent ? launch_persistent(plan, P, g->ctl, cap, 0) : pm::launch_polymul(P, cap);
    e = cudaStreamEndCapture(cap, &g->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    destroy_graph(g);
    return cuda_fail(e, "graph capture");
  }
  *out = g;
  return ok();
}

pm_status pm_graph_launch(pm_graph* g, void* stream) {
  if (!g) return fail(PM_ERR_ARG, "graph is NULL");
  DeviceGuard dg(g->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return ok();
}

pm_status pm_graph_destroy(pm_graph* g) {
  destroy_graph(g);
  return ok();
}

}  // extern "C"

// ---------------------------------------------------------------- serving
//
// A continuous-batching request loop.  Clients submit products whose
// operands already live on the device; a worker thread forms batches from
// the queued requests in arrival order, admitting each one only if its
// output and column-stage scratch fit in the remaining device-memory budget
// (an arena allocated once), and runs every batch as one uneven persistent
// launch.  Up to `max_inflight` batches are on the device at once (one
// stream and work queue each), so requests that arrive while others run are
// admitted as soon as a slot and memory free up.  Outputs stay in the arena
// until the client releases the request.

namespace {

double now_us() {
  using namespace std::chrono;
  return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) in 256-byte granules.
struct Arena {
  std::map<uint64_t, uint64_t> free_;  // offset -> length
  uint64_t used = 0, peak = 0;
  void init(uint64_t size) {
    free_.clear();
    free_[0] = size;
    used = peak = 0;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = (bytes + 255) & ~(uint64_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes;
        const uint64_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        used += bytes;
        if (used > peak) peak = used;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~(uint64_t)255;
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Request {
  const pm_plan* plan;
  const uint64_t* a;
  const uint64_t* b;
  uint32_t npoly;
  uint64_t c_off = 0, c_bytes = 0, s_off = 0, s_bytes = 0;
  double t_submit = 0, t_done = 0;
  int state = RQ_QUEUED;
  pm_status status = PM_OK;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;  // timing events around each launch
  pm_queue* queue = nullptr;
  bool busy = false;
  std::vector<uint64_t> ids;
};

}  // namespace

struct pm_server {
  int device = 0;
  pm_server_config cfg{};
  uint8_t* arena_base = nullptr;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queued;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t queued_rows = 0;   // row tasks (4096-word rows) of the queued requests
  uint64_t min_rows = 0;      // launch threshold while another batch runs
  pm_server_stats stats{};
  cudaEvent_t t0 = nullptr;  // time origin of the batches' device intervals
  std::deque<std::pair<float, float>> recent;  // device intervals (ms) of the last 16 batches
  pm_status worker_status = PM_OK;
  char worker_msg[256] = "";
};

namespace {

uint64_t request_scratch_bytes(const pm_plan* p, uint32_t npoly, bool square) {
  // N >= 2^12 (the 1024-word split keeps b's column image for N = 2^12 too)
  if (p->logn < 12 || square) return 0;
  return (uint64_t)npoly * p->nlimbs << p->logn << 3;
}

// Work of a request in 4096-word rows (a request of smaller N counts as one).
uint64_t request_rows(const pm_plan* p, uint32_t npoly) {
  const uint64_t per = p->logn > 12 ? ((uint64_t)1 << (p->logn - 12)) : 1;
  return (uint64_t)npoly * p->nlimbs * per;
}

// Worker: retire finished batches, then launch a new one on a free slot.
void server_loop(pm_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progress = false;
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const double t = now_us();
      pm_status st = PM_OK;
      if (q != cudaSuccess) {
        st = PM_ERR_CUDA;
      } else {
        uint32_t flag = 0;
        if (sl.queue->d_ctl && cudaMemcpy(&flag, sl.queue->d_ctl + 1, 4, cudaMemcpyDeviceToHost) == cudaSuccess && flag) {
          st = PM_ERR_TIMEOUT;
          cudaMemset(sl.queue->d_ctl + 1, 0, 4);
        }
        // the batch's device interval; the most batches running at one
        // instant among the last 16 (a sweep over their end points)
        float b0 = 0.f, b1 = 0.f;
        if (cudaEventElapsedTime(&b0, S->t0, sl.start) == cudaSuccess &&
            cudaEventElapsedTime(&b1, S->t0, sl.done) == cudaSuccess) {
          S->recent.emplace_back(b0, b1);
          if (S->recent.size() > 16) S->recent.pop_front();
          std::vector<std::pair<float, int>> ends;
          for (const auto& iv : S->recent) {
            ends.emplace_back(iv.first, 1);
            ends.emplace_back(iv.second, -1);
          }
          std::sort(ends.begin(), ends.end());  // at equal times an end (-1) comes first
          int run = 0;
          for (const auto& e : ends) {
            run += e.second;
            if ((uint64_t)run > S->stats.max_device_overlap) S->stats.max_device_overlap = run;
          }
        }
      }
      for (uint64_t id : sl.ids) {
        Request& r = S->reqs[id];
        r.state = RQ_DONE;
        r.status = st;
        r.t_done = t;
        if (r.s_bytes) S->arena.release(r.s_off, r.s_bytes);
        r.s_bytes = 0;
        S->stats.completed++;
      }
      sl.ids.clear();
      sl.busy = false;
      progress = true;
      S->cv_done.notify_all();
    }
    Slot* free_slot = nullptr;
    bool running = false;
    for (auto& sl : S->slots) {
      if (sl.busy)
        running = true;
      else if (!free_slot)
        free_slot = &sl;
    }
    // An idle device takes whatever is queued; while a batch runs, the next
    // one waits until it has enough rows to keep the GPU full on its own.
    if (free_slot && !S->queued.empty() && (!running || S->queued_rows >= S->min_rows)) {
      std::vector<pm_job> jobs;
      std::vector<uint64_t*> scr;
      std::vector<uint64_t> ids;
      // one uneven launch serves plans of one kind (PM_PLAN_HALVING and
      // PM_PLAN_FUSED agree); a request of another kind starts the next batch
      uint32_t kind = ~0u;
      while (!S->queued.empty() && (!S->cfg.max_batch || ids.size() < S->cfg.max_batch)) {
        const uint64_t id = S->queued.front();
        Request& r = S->reqs[id];
        if (r.plan->logn >= 12) {
          const uint32_t k = r.plan->flags & (PM_PLAN_HALVING | PM_PLAN_FUSED);
          if (kind != ~0u && k != kind) break;
          kind = k;
        }
        const bool square = r.a == r.b;
        const uint64_t cb = (uint64_t)r.npoly * r.plan->nlimbs << r.plan->logn << 3;
        const uint64_t sb = request_scratch_bytes(r.plan, r.npoly, square);
        uint64_t coff = 0, soff = 0;
        if (!S->arena.alloc(cb, &coff)) break;
        if (sb && !S->arena.alloc(sb, &soff)) {
          S->arena.release(coff, cb);
          break;
        }
        r.c_off = coff;
        r.c_bytes = cb;
        r.s_off = soff;
        r.s_bytes = sb;
        r.state = RQ_RUNNING;
        S->queued.pop_front();
        S->queued_rows -= request_rows(r.plan, r.npoly);
        jobs.push_back(pm_job{r.plan, r.a, r.b, (uint64_t*)(S->arena_base + coff), r.npoly});
        scr.push_back(sb ? (uint64_t*)(S->arena_base + soff) : nullptr);
        ids.push_back(id);
      }
      if (!ids.empty()) {
        pm_status st = PM_OK;
        if (cudaEventRecord(free_slot->start, free_slot->stream) != cudaSuccess) st = PM_ERR_CUDA;
        if (st == PM_OK) {
          std::lock_guard<std::mutex> lq(free_slot->queue->mu);
          st = uneven_impl(free_slot->queue, jobs.data(), (uint32_t)jobs.size(), scr.data(),
                           free_slot->stream);
        }
        if (st == PM_OK && cudaEventRecord(free_slot->done, free_slot->stream) != cudaSuccess)
          st = PM_ERR_CUDA;
        if (st != PM_OK) {
          S->worker_status = st;
          snprintf(S->worker_msg, sizeof(S->worker_msg), "%s", g_err);
          for (uint64_t id : ids) {
            Request& r = S->reqs[id];
            r.state = RQ_DONE;
            r.status = st;
            r.t_done = now_us();
            if (r.s_bytes) S->arena.release(r.s_off, r.s_bytes);
            r.s_bytes = 0;
          }
          S->cv_done.notify_all();
        } else {
          free_slot->ids = ids;
          free_slot->busy = true;
          uint64_t busy = 0;
          for (auto& sl : S->slots) busy += sl.busy ? 1 : 0;
          if (busy > S->stats.max_inflight) S->stats.max_inflight = busy;
          S->stats.batches++;
          S->stats.batched_requests += ids.size();
          if (ids.size() > S->stats.max_batch) S->stats.max_batch = ids.size();
        }
        progress = true;
      } else if (S->stop && !running) {
        // stopping, nothing on the device, and the head request does not fit
        // beside the outputs clients still hold: it never will, so fail the
        // rest of the queue instead of waiting for releases
        for (uint64_t id : S->queued) {
          Request& r = S->reqs[id];
          r.state = RQ_DONE;
          r.status = PM_ERR_BUDGET;
          r.t_done = now_us();
        }
        S->queued.clear();
        S->queued_rows = 0;
        snprintf(S->worker_msg, sizeof(S->worker_msg), "server stopped with the arena full");
        S->cv_done.notify_all();
        progress = true;
      }
    }
    S->stats.arena_peak_bytes = S->arena.peak;
    bool any_busy = false;
    for (auto& sl : S->slots) any_busy |= sl.busy;
    if (S->stop && !any_busy && S->queued.empty()) break;
    if (!progress) {
      if (any_busy)
        S->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

void destroy_server(pm_server* S) {
  if (!S) return;
  if (S->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    S->worker.join();
  }
  DeviceGuard g(S->device);
  for (auto& sl : S->slots) {
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    destroy_queue(sl.queue);
  }
  if (S->t0) cudaEventDestroy(S->t0);
  cudaFree(S->arena_base);
  delete S;
}

}  // namespace

extern "C" {

pm_status pm_server_create(pm_server** out, int device, const pm_server_config* cfg) {
  if (!out || !cfg) return fail(PM_ERR_ARG, "out or cfg is NULL");
  *out = nullptr;
  if (cfg->hbm_budget_bytes < (1u << 20)) return fail(PM_ERR_ARG, "budget below 1 MiB");
  if (cfg->max_inflight < 1 || cfg->max_inflight > 8) return fail(PM_ERR_ARG, "max_inflight must be 1..8");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(PM_ERR_ARG, "device %d not present", device);
  DeviceGuard g(device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  pm_server* S = new (std::nothrow) pm_server();
  if (!S) return fail(PM_ERR_OOM, "host allocation failed");
  S->device = device;
  S->cfg = *cfg;
  if ((e = cudaMalloc(&S->arena_base, cfg->hbm_budget_bytes)) != cudaSuccess) {
    destroy_server(S);
    return cuda_fail(e, "cudaMalloc(serving arena)");
  }
  S->arena.init(cfg->hbm_budget_bytes);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  S->min_rows = cfg->min_batch_rows ? cfg->min_batch_rows : (uint64_t)sms * 3 * 4;
  S->slots.resize(cfg->max_inflight);
  for (auto& sl : S->slots) {
    pm_status st = pm_queue_create(&sl.queue, device);
    if (st != PM_OK) {
      destroy_server(S);
      return st;
    }
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&sl.start)) != cudaSuccess ||
        (e = cudaEventCreate(&sl.done)) != cudaSuccess) {
      destroy_server(S);
      return cuda_fail(e, "serving streams");
    }
  }
  // the time origin: recorded (and complete) before any batch is launched
  if ((e = cudaEventCreate(&S->t0)) != cudaSuccess ||
      (e = cudaEventRecord(S->t0, S->slots[0].stream)) != cudaSuccess ||
      (e = cudaEventSynchronize(S->t0)) != cudaSuccess) {
    destroy_server(S);
    return cuda_fail(e, "serving time origin");
  }
  S->worker = std::thread(server_loop, S);
  *out = S;
  return ok();
}

pm_status pm_server_destroy(pm_server* S) {
  destroy_server(S);
  return ok();
}

pm_status pm_server_submit(pm_server* S, const pm_plan* plan, const uint64_t* d_a,
                           const uint64_t* d_b, uint32_t npoly, uint64_t* id_out) {
  if (!S || !plan || !id_out) return fail(PM_ERR_ARG, "NULL argument");
  if (!d_a || !d_b || !aligned16(d_a) || !aligned16(d_b)) return fail(PM_ERR_ARG, "NULL or misaligned operand");
  if (plan->device != S->device) return fail(PM_ERR_ARG, "plan on another device");
  if (is_word32(plan)) return fail(PM_ERR_ARG, "the server takes 64-bit plans");
  pm_status s = check_batch(plan, npoly);
  if (s != PM_OK) return s;
  const uint64_t need = ((uint64_t)npoly * plan->nlimbs << plan->logn << 3) +
                        request_scratch_bytes(plan, npoly, d_a == d_b) + 512;
  if (need > S->cfg.hbm_budget_bytes)
    return fail(PM_ERR_BUDGET, "request needs %llu bytes, budget is %llu", (unsigned long long)need,
                (unsigned long long)S->cfg.hbm_budget_bytes);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(PM_ERR_ARG, "server is stopping");
    const uint64_t id = S->next_id++;
    Request r;
    r.plan = plan;
    r.a = d_a;
    r.b = d_b;
    r.npoly = npoly;
    r.t_submit = now_us();
    S->reqs.emplace(id, r);
    S->queued.push_back(id);
    S->queued_rows += request_rows(plan, npoly);
    S->stats.submitted++;
    *id_out = id;
  }
  S->cv_work.notify_one();
  return ok();
}

pm_status pm_server_wait(pm_server* S, uint64_t id, uint32_t timeout_ms, uint64_t** d_c_out,
                         double* latency_us) {
  if (!S) return fail(PM_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(PM_ERR_ARG, "unknown request %llu", (unsigned long long)id);
  // find, not operator[]: a request released by another thread meanwhile
  // must not be re-created as a fresh queued entry
  const bool ready = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    const auto jt = S->reqs.find(id);
    return jt == S->reqs.end() || jt->second.state == RQ_DONE;
  });
  if (!ready) return fail(PM_ERR_TIMEOUT, "request %llu not done within %u ms", (unsigned long long)id, timeout_ms);
  it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(PM_ERR_ARG, "request %llu was released", (unsigned long long)id);
  Request& r = it->second;
  if (r.status != PM_OK) return fail(r.status, "request %llu failed: %s", (unsigned long long)id, S->worker_msg);
  if (d_c_out) *d_c_out = (uint64_t*)(S->arena_base + r.c_off);
  if (latency_us) *latency_us = r.t_done - r.t_submit;
  return ok();
}

pm_status pm_server_release(pm_server* S, uint64_t id) {
  if (!S) return fail(PM_ERR_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return fail(PM_ERR_ARG, "unknown request %llu", (unsigned long long)id);
    if (it->second.state != RQ_DONE) return fail(PM_ERR_ARG, "request %llu still running", (unsigned long long)id);
    if (it->second.c_bytes) S->arena.release(it->second.c_off, it->second.c_bytes);
    S->reqs.erase(it);
  }
  S->cv_work.notify_one();
  return ok();
}

pm_status pm_server_get_stats(pm_server* S, pm_server_stats* out) {
  if (!S || !out) return fail(PM_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->arena_used_bytes = S->arena.used;
  return ok();
}

}  // extern "C"
