// pm_microbench.cu -- throughput microbenchmarks that give the roofline
// denominators for this integer-arithmetic path:
//   * the register-resident rate of the cheapest exact 60-bit modular product
//     used on the path (the lazy Shoup product of pm_arith.cuh), and
//   * the 32-bit integer multiply-add (IMAD) rate it is built from.
// Both kernels keep every operand in registers with 8 independent chains per
// thread and a grid of 8 CTAs x 256 threads per SM.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pm.h"
#include "pm_arith.cuh"

namespace pm {

__global__ void __launch_bounds__(256) k_peak_shoup(uint64_t* sink, uint64_t w, uint64_t wp,
                                                    uint64_t q, int iters) {
  uint64_t x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 977u + i * 131u + blockIdx.x;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = mul_shoup_lazy(x[i], w, wp, q);
  }
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s ^= x[i];
  if (s == 0x9e3779b97f4a7c15ull) sink[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_imad(uint32_t* sink, uint32_t a, uint32_t b,
                                                   int iters) {
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = threadIdx.x + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = x[i] * a + b;
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s ^= x[i];
  if (s == 0x9e3779b9u) sink[0] = s;
}

}  // namespace pm

extern "C" pm_status pm_measure_peaks(int device, double* mulmod_per_s, double* imad_per_s) {
  if (!mulmod_per_s || !imad_per_s) return PM_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return PM_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  uint64_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pm_status st = PM_OK;
  if (cudaMalloc(&sink, 64) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = PM_ERR_CUDA;
  } else {
    const uint64_t q = 0xffffffffffc0001ull;  // a 60-bit NTT prime
    const uint64_t w = 0x0123456789abcdeull % q;
    const uint64_t wp = (uint64_t)((((unsigned __int128)w) << 64) / q);
    const int blocks = sms * 8, threads = 256, iters = 2048;
    const double n = (double)blocks * threads * 8 * iters;
    float ms = 0.f, best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {  // first repetition warms up clocks
      cudaEventRecord(e0);
      pm::k_peak_shoup<<<blocks, threads>>>(sink, w, wp, q, iters);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    *mulmod_per_s = n / (best * 1e-3);
    best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
      cudaEventRecord(e0);
      pm::k_peak_imad<<<blocks, threads>>>((uint32_t*)sink, 3u, 7u, iters * 4);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    *imad_per_s = n * 4 / (best * 1e-3);
    if (cudaGetLastError() != cudaSuccess) st = PM_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  return st;
}
