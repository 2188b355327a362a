// FMA-throughput measurement used as the ALU roofline denominator: every thread runs
// eight independent FMA chains, enough warps per SM to fill the FP64 / FP32 pipes.
#include <algorithm>

#include "common.h"

namespace vef {

template <typename T>
__global__ void fma_chain_kernel(T* out, int iters) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
  const T b = (T)0.999999, c = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
static vef_status measure(int iters, double* rate) {
  int dev = 0, sms = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  VEF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  VEF_CUDA_TRY(cudaMalloc(&out, sizeof(T) * blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chain_kernel<T><<<blocks, threads>>>(out, iters / 8);
  cudaEventRecord(e0);
  fma_chain_kernel<T><<<blocks, threads>>>(out, iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return cuda_fail(err, "fma peak kernel");
  *rate = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return VEF_OK;
}

}  // namespace vef

extern "C" vef_status vef_measure_fma_peak(int precision, double* flops_per_s) {
  if (!flops_per_s) { vef::set_last_error("flops_per_s is NULL"); return VEF_ERR_INVALID_ARG; }
  if (precision == VEF_FP64) return vef::measure<double>(4096, flops_per_s);
  if (precision == VEF_MIXED) return vef::measure<float>(65536, flops_per_s);
  vef::set_last_error("precision must be VEF_FP64 or VEF_MIXED");
  return VEF_ERR_INVALID_ARG;
}
