// pm_reduce.cu -- the modular-reduction study of Sec. II-B (Fig. 4) on this
// GPU: reductions of a product a*b (a, b < q) by
//   PM_RED_BUILTIN    : the C '%' operator on a 128-bit product,
//   PM_RED_ALG2       : classical Barrett (Algorithm 2, up to two corrections),
//   PM_RED_ALG3       : Dhem-Quisquater alpha=N+3, beta=-2 (Algorithm 3, m <= 60),
//   PM_RED_ALG4       : the paper's variant (Algorithm 4, m <= 62),
//   PM_RED_SHOUP      : Shoup's product with a precomputed companion of b
//                       (b is a constant such as a twiddle), fully reduced,
//   PM_RED_MONTGOMERY : Montgomery's REDC with R = 2^64 (b in Montgomery form).
// Each has a throughput kernel (register-resident chains) and an elementwise
// kernel used by the tests to check it against exact arithmetic.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pm.h"
#include "pm_arith.cuh"

namespace pm {
namespace {

struct RedConst {
  uint64_t q;
  uint32_t m;
  uint64_t mu2;   // Algorithm 2: floor(2^(2m) / q)
  uint64_t mu3;   // Algorithm 3: floor(2^(2m+3) / q)   (m <= 60)
  uint64_t mu4;   // Algorithm 4: floor(2^(2m+1) / q)
  uint64_t qinv;  // Montgomery: -q^-1 mod 2^64
};

// 128-bit value (hi:lo) shifted right by s, 0 < s < 128.
__device__ __forceinline__ uint64_t shr128(uint64_t hi, uint64_t lo, uint32_t s) {
  if (s >= 64) return hi >> (s - 64);
  return (lo >> s) | (hi << (64 - s));
}

__device__ __forceinline__ uint64_t red_builtin(uint64_t a, uint64_t b, const RedConst& k) {
  const unsigned __int128 x = (unsigned __int128)a * b;
  return (uint64_t)(x % k.q);
}

// Algorithm 2: c = x >> (m-1); quot = (c*mu) >> (m+1); rem = x - quot*q; <= 2 corrections.
__device__ __forceinline__ uint64_t red_alg2(uint64_t a, uint64_t b, const RedConst& k) {
  const uint64_t lo = a * b, hi = __umul64hi(a, b);
  const uint64_t c = shr128(hi, lo, k.m - 1);
  const uint64_t plo = c * k.mu2, phi = __umul64hi(c, k.mu2);
  const uint64_t quot = shr128(phi, plo, k.m + 1);
  uint64_t r = lo - quot * k.q;
  r = csub(r, k.q);
  return csub(r, k.q);
}

// Algorithm 3: c = x >> (m-2); quot = (c*mu) >> (m+5); one correction.
__device__ __forceinline__ uint64_t red_alg3(uint64_t a, uint64_t b, const RedConst& k) {
  const uint64_t lo = a * b, hi = __umul64hi(a, b);
  const uint64_t c = shr128(hi, lo, k.m - 2);
  const uint64_t plo = c * k.mu3, phi = __umul64hi(c, k.mu3);
  const uint64_t quot = shr128(phi, plo, k.m + 5);
  return csub(lo - quot * k.q, k.q);
}

__device__ __forceinline__ uint64_t red_alg4(uint64_t a, uint64_t b, const RedConst& k) {
  const uint64_t lo = a * b, hi = __umul64hi(a, b);
  const uint64_t c = shr128(hi, lo, k.m - 2);
  const uint64_t plo = c * k.mu4, phi = __umul64hi(c, k.mu4);
  const uint64_t quot = shr128(phi, plo, k.m + 3);
  return csub(lo - quot * k.q, k.q);
}

// Shoup: w*y mod q with wp = floor(w 2^64 / q), one correction.
__device__ __forceinline__ uint64_t red_shoup(uint64_t y, uint64_t w, uint64_t wp,
                                              const RedConst& k) {
  return csub(mul_shoup_lazy(y, w, wp, k.q), k.q);
}

// Montgomery REDC: returns a * bm * 2^-64 mod q for bm < q (bm = b 2^64 mod q
// gives a*b mod q).  t = a*bm; m = t_lo * (-q^-1); u = (t + m q) / 2^64.
__device__ __forceinline__ uint64_t red_mont(uint64_t a, uint64_t bm, const RedConst& k) {
  const uint64_t tlo = a * bm, thi = __umul64hi(a, bm);
  const uint64_t mm = tlo * k.qinv;
  const uint64_t mlo = mm * k.q, mhi = __umul64hi(mm, k.q);
  // (tlo + mlo) is 0 mod 2^64; its carry is 1 unless both are 0
  const uint64_t carry = (tlo != 0) ? 1 : 0;
  (void)mlo;
  const uint64_t u = thi + mhi + carry;  // < 2q for q < 2^63
  return csub(u, k.q);
}

template <int V>
__device__ __forceinline__ uint64_t red_any(uint64_t a, uint64_t b, uint64_t bp,
                                            const RedConst& k) {
  if constexpr (V == PM_RED_BUILTIN) return red_builtin(a, b, k);
  if constexpr (V == PM_RED_ALG2) return red_alg2(a, b, k);
  if constexpr (V == PM_RED_ALG3) return red_alg3(a, b, k);
  if constexpr (V == PM_RED_ALG4) return red_alg4(a, b, k);
  if constexpr (V == PM_RED_SHOUP) return red_shoup(a, b, bp, k);
  return red_mont(a, b, k);
}

template <int V>
__global__ void __launch_bounds__(256) k_red_rate(uint64_t* sink, RedConst k, uint64_t b,
                                                  uint64_t bp, int iters) {
  uint64_t x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = (threadIdx.x * 977u + i * 131u + blockIdx.x) % k.q;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = red_any<V>(x[i], b, bp, k);
  }
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s ^= x[i];
  if (s == 0x9e3779b97f4a7c15ull) sink[0] = s;
}

// Elementwise: c[i] = reduce(a[i] * b[i]).  For Shoup and Montgomery the
// per-element constant (companion / Montgomery form of b[i]) is derived with
// 128-bit arithmetic first, since b varies here.
template <int V>
__global__ void __launch_bounds__(256) k_red_apply(const uint64_t* a, const uint64_t* b,
                                                   uint64_t* c, size_t n, RedConst k) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    uint64_t bb = b[i], bp = 0;
    if constexpr (V == PM_RED_SHOUP)
      bp = (uint64_t)((((unsigned __int128)bb) << 64) / k.q);
    if constexpr (V == PM_RED_MONTGOMERY)
      bb = (uint64_t)((((unsigned __int128)bb) << 64) % k.q);
    c[i] = red_any<V>(a[i], bb, bp, k);
  }
}

uint32_t bitlen64(uint64_t x) {
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

bool make_const(uint64_t q, RedConst* k) {
  if (q < 5 || q >= ((uint64_t)1 << 62) || !(q & 1)) return false;
  k->q = q;
  k->m = bitlen64(q);
  using u128 = unsigned __int128;
  k->mu2 = (uint64_t)((((u128)1) << (2 * k->m)) / q);
  k->mu3 = k->m <= 60 ? (uint64_t)((((u128)1) << (2 * k->m + 3)) / q) : 0;
  k->mu4 = (uint64_t)((((u128)1) << (2 * k->m + 1)) / q);
  uint64_t inv = 1;  // q^-1 mod 2^64 by Newton iteration (q odd)
  for (int i = 0; i < 7; i++) inv *= 2 - q * inv;
  k->qinv = 0 - inv;
  return true;
}

template <int V>
cudaError_t rate_one(const RedConst& k, int sms, uint64_t* sink, double* out) {
  const int blocks = sms * 8, threads = 256, iters = 1024;
  const uint64_t b = (0x0123456789abcdefull % k.q) | 1;
  const uint64_t bp = (uint64_t)((((unsigned __int128)b) << 64) / k.q);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < 3; r++) {
    cudaEventRecord(e0);
    k_red_rate<V><<<blocks, threads>>>(sink, k, b, bp, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = (double)blocks * threads * 8 * iters / (best * 1e-3);
  return cudaGetLastError();
}

}  // namespace
}  // namespace pm

extern "C" pm_status pm_reduction_rates(int device, uint64_t q, double* rates) {
  pm::RedConst k;
  if (!rates || !pm::make_const(q, &k)) return PM_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return PM_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  uint64_t* sink = nullptr;
  pm_status st = PM_OK;
  if (cudaMalloc(&sink, 64) != cudaSuccess) {
    cudaSetDevice(prev);
    return PM_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  if (!e) e = pm::rate_one<PM_RED_BUILTIN>(k, sms, sink, &rates[PM_RED_BUILTIN]);
  if (!e) e = pm::rate_one<PM_RED_ALG2>(k, sms, sink, &rates[PM_RED_ALG2]);
  if (!e) {
    if (k.m <= 60)
      e = pm::rate_one<PM_RED_ALG3>(k, sms, sink, &rates[PM_RED_ALG3]);
    else
      rates[PM_RED_ALG3] = 0.0;  // Algorithm 3 needs len(q) <= 60 for 64-bit words
  }
  if (!e) e = pm::rate_one<PM_RED_ALG4>(k, sms, sink, &rates[PM_RED_ALG4]);
  if (!e) e = pm::rate_one<PM_RED_SHOUP>(k, sms, sink, &rates[PM_RED_SHOUP]);
  if (!e) e = pm::rate_one<PM_RED_MONTGOMERY>(k, sms, sink, &rates[PM_RED_MONTGOMERY]);
  if (e != cudaSuccess) st = PM_ERR_CUDA;
  cudaFree(sink);
  cudaSetDevice(prev);
  return st;
}

extern "C" pm_status pm_reduction_apply(int variant, uint64_t q, const uint64_t* d_a,
                                        const uint64_t* d_b, uint64_t* d_c, uint64_t n,
                                        void* stream) {
  pm::RedConst k;
  if (!d_a || !d_b || !d_c || !pm::make_const(q, &k)) return PM_ERR_ARG;
  if (variant == PM_RED_ALG3 && k.m > 60) return PM_ERR_ARG;
  if (n == 0) return PM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256);
  switch (variant) {
    case PM_RED_BUILTIN: pm::k_red_apply<PM_RED_BUILTIN><<<blocks, 256, 0, st>>>(d_a, d_b, d_c, n, k); break;
    case PM_RED_ALG2: pm::k_red_apply<PM_RED_ALG2><<<blocks, 256, 0, st>>>(d_a, d_b, d_c, n, k); break;
    case PM_RED_ALG3: pm::k_red_apply<PM_RED_ALG3><<<blocks, 256, 0, st>>>(d_a, d_b, d_c, n, k); break;
    case PM_RED_ALG4: pm::k_red_apply<PM_RED_ALG4><<<blocks, 256, 0, st>>>(d_a, d_b, d_c, n, k); break;
    case PM_RED_SHOUP: pm::k_red_apply<PM_RED_SHOUP><<<blocks, 256, 0, st>>>(d_a, d_b, d_c, n, k); break;
    case PM_RED_MONTGOMERY: pm::k_red_apply<PM_RED_MONTGOMERY><<<blocks, 256, 0, st>>>(d_a, d_b, d_c, n, k); break;
    default: return PM_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}
