// Eddington tensor without any device allocation.
//
// vef_moments computes E = P / phi at the volume Gauss points in two kernels that pass
// the nodal moments phi, P_xx, P_xy, P_yy through scratch memory owned by the mesh
// handle.  Some callers cannot allocate device memory at all: an application that
// reserves the whole GPU for its own pool at start-up, or a time-stepping loop that
// must not hit the device-wide synchronisation that cudaMalloc / cudaFree can imply.
// They also cannot create a mesh handle, which allocates its geometry.  This file gives
// them vef_eddington_noalloc: the same two-phase computation, with the scratch in a
// file-scope device array of fixed size and the direction set passed by value, so the
// call allocates nothing.
#include <cmath>
#include <mutex>

#include "common.h"

namespace vef {

// 2^21 doubles = 16 MiB: the four nodal moment fields, so E * (p+1)^2 <= 2^19.
constexpr long long kNoAllocScratchDoubles = 1LL << 21;
constexpr int kNoAllocMaxD = 256;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

struct DirSet {
  int D;
  double mu[kNoAllocMaxD];
  double eta[kNoAllocMaxD];
  double w[kNoAllocMaxD];
};

// one thread per (e, i): phi and the second moment at the DG nodes, into the scratch
__global__ void noalloc_nodal_kernel(long long En, DirSet ds, const double* __restrict__ psi,
                                     double* __restrict__ scratch) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= En) return;
  double s0 = 0, sxx = 0, sxy = 0, syy = 0;
  for (int d = 0; d < ds.D; ++d) {
    const double v = ds.w[d] * psi[(size_t)d * En + t];
    const double mu = ds.mu[d], eta = ds.eta[d];
    s0 += v;
    sxx += mu * mu * v;
    sxy += mu * eta * v;
    syy += eta * eta * v;
  }
  scratch[t] = s0;
  scratch[En + t] = sxx;
  scratch[2 * En + t] = sxy;
  scratch[3 * En + t] = syy;
}

// one thread per (e, q): interpolate phi and P to the Gauss point and divide
__global__ void noalloc_eddington_kernel(long long E, Tab1D tab, const double* __restrict__ scratch,
                                         double* __restrict__ Eten) {
  const int np1 = tab.np1, n = np1 * np1, nq = tab.nq, nq2 = nq * nq;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * nq2) return;
  const long long e = t / nq2;
  const int q = (int)(t % nq2), k1 = q % nq, k2 = q / nq;
  const long long En = E * n;
  double f = 0, a = 0, b = 0, c = 0;
  for (int j = 0; j < n; ++j) {
    const double B = tab.l[j % np1][k1] * tab.l[j / np1][k2];
    const size_t o = (size_t)e * n + j;
    f += B * scratch[o];
    a += B * scratch[En + o];
    b += B * scratch[2 * En + o];
    c += B * scratch[3 * En + o];
  }
  const size_t Eq = (size_t)E * nq2;
  if (f > 1e-300) {
    Eten[t] = a / f;
    Eten[Eq + t] = b / f;
    Eten[2 * Eq + t] = c / f;
  } else {
    Eten[t] = Eten[Eq + t] = Eten[2 * Eq + t] = nan("");
  }
}

// Device address of the scratch array, looked up once per device (with that device
// current) by cudaGetSymbolAddress; the host-side name of the array is not a device
// address and is never passed to a kernel.  The table is filled under a mutex, so host
// threads making their first calls at the same time do not race on it.
constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

static vef_status scratch_address(double** out) {
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("device ordinal out of range for the no-allocation scratch table");
    return VEF_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(no-allocation scratch)");
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return VEF_OK;
}

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_eddington_noalloc(const double* psi, const double* omega,
                                            const double* weights, int D, long long E, int p,
                                            double* Eten, void* stream) {
  if (!psi || !omega || !weights || !Eten) {
    set_last_error("psi, omega, weights and Eten are required");
    return VEF_ERR_INVALID_ARG;
  }
  if (p < 1 || p > kMaxP || E < 1) {
    set_last_error("p must be in 1..4 and E >= 1");
    return VEF_ERR_INVALID_ARG;
  }
  if (D < 1 || D > kNoAllocMaxD) {
    set_last_error("vef_eddington_noalloc: D must be in 1..256");
    return VEF_ERR_INVALID_ARG;
  }
  const long long n = (long long)(p + 1) * (p + 1);
  if (E > kNoAllocScratchDoubles / (4 * n)) {
    set_last_error("vef_eddington_noalloc: E * (p+1)^2 exceeds the fixed scratch limit of 524288 "
                   "nodal values (16 MiB); use vef_moments for larger meshes");
    return VEF_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  vef_status st = scratch_address(&scratch);
  if (st != VEF_OK) return st;
  DirSet ds{};
  ds.D = D;
  for (int d = 0; d < D; ++d) {
    ds.mu[d] = omega[2 * d];
    ds.eta[d] = omega[2 * d + 1];
    ds.w[d] = weights[d];
  }
  const Tab1D tab = make_tab1d(p);
  cudaStream_t s = (cudaStream_t)stream;
  const long long En = E * n;
  // every scratch entry the second kernel reads is written by the first in this call
  noalloc_nodal_kernel<<<(unsigned)((En + 255) / 256), 256, 0, s>>>(En, ds, psi, scratch);
  const long long Eq = E * (p + 2) * (p + 2);
  noalloc_eddington_kernel<<<(unsigned)((Eq + 255) / 256), 256, 0, s>>>(E, tab, scratch, Eten);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}
