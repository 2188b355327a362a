// FMA-throughput measurement used as the ALU roofline denominator: every thread runs
// eight independent FMA chains, enough warps per SM to fill the FP64 / FP32 pipes.
#include <algorithm>

#include "common.h"
#include "device.cuh"

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

// Failure-detection self-test.  One thread polls, in the bounded form the sweep's waits
// take, for something that is already complete (satisfied != 0) or that nothing completes:
// kind 0 an acquire load of a global flag (with a short sleep between polls, like the wait
// for a band of the fused apply), kind 1 the parity of a shared-memory mbarrier phase (like
// the wait for a staged chunk).  After `polls` failed polls it sets the timeout bit of the
// status word and returns; the loop count is the only bound, so the kernel always ends.
__global__ void wait_selftest_kernel(int kind, int satisfied, uint32_t polls, const int* flag,
                                     unsigned int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  uint32_t n = 0;
  if (kind == 0) {
    while (ld_acquire_gpu(flag) == 0 && ++n < polls) __nanosleep(64);
  } else {
    mbar_init(&bar, 1);
    mbar_fence_init();
    if (satisfied) mbar_arrive(&bar);
    while (!mbar_try_wait(&bar, 0) && ++n < polls) {
    }
  }
  if (n >= polls) atomicOr(status, kDevTimeout);
}

}  // namespace vef

extern "C" vef_status vef_wait_selftest(int kind, int satisfied, long long polls, void* stream) {
  using namespace vef;
  if (kind != 0 && kind != 1) { set_last_error("kind must be 0 (global flag) or 1 (mbarrier)"); return VEF_ERR_INVALID_ARG; }
  if (polls < 1 || polls > (1LL << 24)) { set_last_error("polls must be in 1..2^24"); return VEF_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  int* buf = nullptr;   // [0] the flag, [1] the status word
  VEF_CUDA_TRY(cudaMalloc(&buf, 2 * sizeof(int)));
  cudaError_t err = cudaMemsetAsync(buf, 0, 2 * sizeof(int), s);
  if (err == cudaSuccess && satisfied && kind == 0) err = cudaMemsetAsync(buf, 1, 1, s);
  if (err == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(kind, satisfied ? 1 : 0, (uint32_t)polls, buf,
                                          reinterpret_cast<unsigned int*>(buf + 1));
    err = cudaGetLastError();
  }
  unsigned int bits = 0;
  if (err == cudaSuccess) err = cudaMemcpyAsync(&bits, buf + 1, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (err != cudaSuccess) return cuda_fail(err, "wait self-test");
  if (bits & kDevTimeout) { set_last_error("the bounded wait ran out and reported a timeout"); return VEF_ERR_TIMEOUT; }
  return VEF_OK;
}

extern "C" vef_status vef_measure_fma_peak(int precision, double* flops_per_s) {
  if (!flops_per_s) { vef::set_last_error("flops_per_s is NULL"); return VEF_ERR_INVALID_ARG; }
  if (precision == VEF_FP64) return vef::measure<double>(4096, flops_per_s);
  if (precision == VEF_MIXED) return vef::measure<float>(65536, flops_per_s);
  vef::set_last_error("precision must be VEF_FP64 or VEF_MIXED");
  return VEF_ERR_INVALID_ARG;
}

// Failure-detection test hook: OR status bits into a mesh handle's device status word from a
// one-thread kernel on `stream`, as a device-side wait that ran out would.
namespace vef {
__global__ void inject_status_kernel(unsigned int* status, unsigned int bits) { atomicOr(status, bits); }
}  // namespace vef

static_assert((unsigned)VEF_STATUS_TIMEOUT == (unsigned)vef::kDevTimeout &&
                  (unsigned)VEF_STATUS_NOT_CONVERGED == (unsigned)vef::kDevNotConverged &&
                  (unsigned)VEF_STATUS_NONPOSITIVE == (unsigned)vef::kDevNonpositive &&
                  (unsigned)VEF_STATUS_SINGULAR == (unsigned)vef::kDevSingular &&
                  (unsigned)VEF_STATUS_BOUNDS == (unsigned)vef::kDevBounds,
              "public status bits match the device status word");

extern "C" vef_status vef_mesh_inject_status(vef_mesh mesh, unsigned int bits, void* stream) {
  if (!mesh) { vef::set_last_error("mesh is NULL"); return VEF_ERR_INVALID_ARG; }
  if (bits == 0 || (bits & ~0x1fu)) { vef::set_last_error("bits must be a non-empty set of VEF_STATUS_* values"); return VEF_ERR_INVALID_ARG; }
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != mesh->impl.device) { vef::set_last_error("mesh belongs to another device"); return VEF_ERR_INVALID_ARG; }
  vef::inject_status_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(mesh->impl.dev_status, bits);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

namespace vef {
namespace {

// pivot_rcp against the correctly rounded reciprocal over n inputs spread across the
// normal range (exponents -500..500 and hashed mantissas, both signs): the largest
// relative difference, as a non-negative double's bit pattern (ordered like an integer)
__global__ void rcp_selftest_kernel(long long n, unsigned long long* worst64, unsigned int* worst32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    const double m = 1.0 + (double)(h >> 12) * 0x1.0p-52;   // [1, 2)
    const int ex = (int)(i % 1001) - 500;
    const double x = ((i & 1) ? -1.0 : 1.0) * ldexp(m, ex);
    const double r = pivot_rcp(x), q = 1.0 / x;
    const double d = fabs(r - q) / fabs(q);
    atomicMax(worst64, (unsigned long long)__double_as_longlong(d));
    const float xf = (float)ldexp(m, ex % 100);
    const float rf = pivot_rcp(xf), qf = 1.0f / xf;
    const float df = fabsf(rf - qf) / fabsf(qf);
    atomicMax(worst32, (unsigned int)__float_as_int(df));
  }
}

}  // namespace
}  // namespace vef

extern "C" vef_status vef_rcp_selftest(long long n, double* max_rel_err, double* max_rel_err_f32) {
  if (n < 1 || n > (1LL << 30) || !max_rel_err || !max_rel_err_f32) {
    vef::set_last_error("n must be in 1..2^30 and both outputs given");
    return VEF_ERR_INVALID_ARG;
  }
  unsigned long long* w = nullptr;
  VEF_CUDA_TRY(cudaMalloc(&w, 16));
  cudaError_t e = cudaMemset(w, 0, 16);
  if (e == cudaSuccess) {
    vef::rcp_selftest_kernel<<<256, 256>>>(n, w, reinterpret_cast<unsigned int*>(w + 1));
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, w, 16, cudaMemcpyDeviceToHost);
  cudaFree(w);
  if (e != cudaSuccess) return vef::cuda_fail(e, "vef_rcp_selftest");
  *max_rel_err = __builtin_bit_cast(double, h[0]);
  const unsigned int f = (unsigned int)h[1];
  *max_rel_err_f32 = (double)__builtin_bit_cast(float, f);
  return VEF_OK;
}
