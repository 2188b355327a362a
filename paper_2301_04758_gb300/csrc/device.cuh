// Device helpers shared by the sweep, moment and adjoint kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"

namespace vef {

// Bounds-checked build (compiled with -DVEF_CHECKED into libvef_checked.so):
// VEF_IN_RANGE(i, n, status) is false when i lies outside [0, n), after setting kDevBounds in
// the device status word, and the access it guards is skipped; in the normal build it is the
// constant true and the guard compiles away.
#ifdef VEF_CHECKED
__device__ __forceinline__ bool in_range_checked(long long i, long long n, unsigned int* status) {
  if (i >= 0 && i < n) return true;
  atomicOr(status, kDevBounds);
  return false;
}
#define VEF_IN_RANGE(i, n, status) ::vef::in_range_checked((long long)(i), (long long)(n), (status))
#else
#define VEF_IN_RANGE(i, n, status) true
#endif

// Factor records of all (element, direction) pairs, in schedule order, as two arrays of
// 16-byte-aligned blocks so the sweep can stage a run of consecutive tasks with one bulk
// copy:
//   staged array S, per task: [info: element, face bits, face of each W slot (4 x u8),
//                               pad: 16 bytes][W slots 0, 1: n x (p+1) each, column-major]
//   extra array X, per task:  [W slots 2, 3][A^{-1}: n x n column-major]
// W slot s holds W_f = A^{-1} Cin_f for the s-th interior inflow face f (in face order);
// slots 2 and 3 exist only on curved meshes (a face partly inflow).
template <int P, typename T>
struct Rec {
  static constexpr int Q = P + 1, N = Q * Q;
  static constexpr int r16(int b) { return (b + 15) / 16 * 16; }
  static constexpr int kSlot = N * Q;                                   // elements per W slot
  static constexpr int kStaged = r16(16 + 2 * kSlot * (int)sizeof(T));  // bytes per task in S
  static constexpr int kExtra = r16(2 * kSlot * (int)sizeof(T));
  static constexpr int kAinv = r16(N * N * (int)sizeof(T));
  static constexpr int kX = kExtra + kAinv;                             // bytes per task in X
  static constexpr int kYBytes = r16(N * (int)sizeof(T));               // padded y row
  static constexpr int kYStride = kYBytes / (int)sizeof(T);
  __host__ __device__ static const char* s_at(const void* S, long long m) {
    return (const char*)S + m * (long long)kStaged;
  }
  __host__ __device__ static char* s_at(void* S, long long m) { return (char*)S + m * (long long)kStaged; }
  __host__ __device__ static const char* x_at(const void* X, long long m) {
    return (const char*)X + m * (long long)kX;
  }
  __host__ __device__ static char* x_at(void* X, long long m) { return (char*)X + m * (long long)kX; }
  // W slot s of the task whose staged block is at s_rec and extra block at x_rec
  __host__ __device__ static const T* slot(const char* s_rec, const char* x_rec, int s) {
    return (const T*)(s < 2 ? s_rec + 16 + s * kSlot * (int)sizeof(T) : x_rec + (s - 2) * kSlot * (int)sizeof(T));
  }
  __host__ __device__ static T* slot(char* s_rec, char* x_rec, int s) {
    return (T*)(s < 2 ? s_rec + 16 + s * kSlot * (int)sizeof(T) : x_rec + (s - 2) * kSlot * (int)sizeof(T));
  }
  __host__ __device__ static const T* ainv(const char* x_rec) { return (const T*)(x_rec + kExtra); }
  __host__ __device__ static T* ainv(char* x_rec) { return (T*)(x_rec + kExtra); }
};

// slot holding face f according to the record's face list (info.z bytes), or -1
__host__ __device__ __forceinline__ int rec_slot_of(unsigned faces, int f) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (((faces >> (8 * s)) & 0xffu) == (unsigned)f) return s;
  return -1;
}

template <typename T> __host__ __device__ constexpr T tiny_pivot();
template <> __host__ __device__ constexpr double tiny_pivot<double>() { return 1e-300; }
template <> __host__ __device__ constexpr float tiny_pivot<float>() { return 1e-37f; }

// Reciprocal of an elimination pivot: the approximate reciprocal instruction
// (rcp.approx.ftz.f64) refined by two Newton-Raphson steps r <- r + r (1 - x r), each of
// which squares the relative error, so the result is within an ulp or two of 1/x for
// normal x, at five FP64-pipe operations instead of a correctly rounded division.  The
// unpivoted eliminations use it; a pivot the guard rejects (tiny, huge or not finite) goes
// to the partial-pivoting path, which divides.  vef_rcp_selftest measures it against 1/x.
__device__ __forceinline__ double pivot_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float pivot_rcp(float x) { return __frcp_rn(x); }

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

// barrier over all threads of the thread-block cluster, release / acquire at cluster scope
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// mbarrier and bulk-copy (TMA) helpers for staging records into shared memory
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// barrier `id` (1..15) over the first `threads` threads of the CTA (a multiple of 32);
// orders the participants' shared and global memory accesses like __syncthreads
__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for staged data: polls the mbarrier phase up to `iters` times and gives up
// early, every 16 polls, once `status` carries the timeout bit (another wait ran out, or
// the call started with an uncollected timeout).  Returns whether the phase completed; a
// consumer that gets false must not use the staged buffer (it may never have been filled).
__device__ __forceinline__ bool mbar_wait_data(uint64_t* bar, unsigned parity, uint32_t iters,
                                               const unsigned int* status) {
  uint32_t n = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++n >= iters) return false;
    if ((n & 15u) == 0 && (*(const volatile unsigned int*)status & kDevTimeout)) return false;
  }
  return true;
}
// 1D bulk copy global -> this CTA's shared memory, completion counted on bar (bytes and
// both addresses must be multiples of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// flag published / read at GPU scope (release / acquire)
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// order this thread's earlier generic-proxy view of global memory before later bulk copies
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// bring the 128-byte line holding p into L2 (no register result)
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
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
