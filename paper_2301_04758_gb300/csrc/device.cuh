// Device helpers shared by the sweep, moment and adjoint kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"

namespace vef {

// floats per factor record of one (element, direction): A^{-1} (n x n) followed by the
// four inflow-coupling maps W_f (n x (p+1) each)
template <int P>
__host__ __device__ constexpr int rec_size() {
  return (P + 1) * (P + 1) * (P + 1) * (P + 1) + 4 * (P + 1) * (P + 1) * (P + 1);
}

template <typename T> __host__ __device__ constexpr T tiny_pivot();
template <> __host__ __device__ constexpr double tiny_pivot<double>() { return 1e-300; }
template <> __host__ __device__ constexpr float tiny_pivot<float>() { return 1e-37f; }

// face-node -> element-dof maps (GLL nodes on the face, in increasing reference coordinate)
template <int P>
__host__ __device__ __forceinline__ int face_dof(int f, int t) {
  constexpr int Q = P + 1;
  return f == 0 ? t : (f == 1 ? P + Q * t : (f == 2 ? t + Q * P : Q * t));
}

__device__ __forceinline__ int nb_elem(int nx, int ny, int e, int f) {
  const int i = e % nx, j = e / nx;
  return f == 0 ? (j > 0 ? e - nx : -1)
       : f == 1 ? (i < nx - 1 ? e + 1 : -1)
       : f == 2 ? (j < ny - 1 ? e + nx : -1)
                : (i > 0 ? e - 1 : -1);
}

// boundary face index of face f of element e (valid only when nb_elem(...) < 0)
__device__ __forceinline__ int bface(int nx, int ny, int e, int f) {
  const int i = e % nx, j = e / nx;
  return f == 0 ? i : f == 1 ? nx + j : f == 2 ? nx + ny + i : 2 * nx + ny + j;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin (bounded) until *flag == epoch.  Returns false if the wait ran out (records
// kDevTimeout and raises the abort word) or another warp aborted.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
constexpr uint32_t kWaitLimitIters = 200000000u;
__device__ __forceinline__ bool wait_epoch(const uint32_t* flag, uint32_t epoch,
                                           unsigned int* status) {
  if (ld_acquire(flag) == epoch) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < kWaitLimitIters; ++it) {
    if (ld_acquire(flag) == epoch) return true;
    if ((it & 63u) == 0) {
      if (*((volatile unsigned int*)(status + 1)) != 0u) return false;
      if (global_ns() - t0 > kWaitLimitNs) break;
    }
  }
  atomicOr(status, kDevTimeout);
  atomicExch(status + 1, 1u);
  return false;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// Table of 1D Lagrange values for kernels templated on the real type.
template <typename T>
struct FaceTab {
  T l[kMaxP + 1][kMaxNq];  // l_a(s_k)
  T w[kMaxNq];             // face Gauss weights
};

template <typename T>
inline FaceTab<T> make_facetab(const Tab1D& t) {
  FaceTab<T> f{};
  for (int a = 0; a <= t.p; ++a)
    for (int k = 0; k < t.nq; ++k) f.l[a][k] = (T)t.l[a][k];
  for (int k = 0; k < t.nq; ++k) f.w[k] = (T)t.glw[k];
  return f;
}

}  // namespace vef
