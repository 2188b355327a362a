// VEF fixed-point iteration (paper Sec. "VEF Algorithm"): invert the transport equation with
// the current scattering source, form the Eddington tensor, boundary factor and inflow
// partial current from its angular flux, solve the VEF equations (hybridized RT,
// vef_hrt_solve), take their scalar flux as the next iterate; stop when the max norm of the
// difference of successive iterates is below the tolerance (the criterion the paper's
// fixed-point solver uses).  Every step runs in the library's kernels; this file only
// sequences them.  The transport factorisation is formed once (sigma_t does not change).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "device.cuh"

namespace vef {
namespace {

__global__ void scale_kernel(long long n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x ? a * x[i] : 0.0;
}

// out = max |a - b| (non-negative doubles order like their bit patterns)
__global__ void vef_maxdiff_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                                   unsigned long long* out) {
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[t] - b[t]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace
}  // namespace vef

using namespace vef;

extern "C" vef_status vef_vef_iterate(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                      const double* source, const double* inflow, const double* omega,
                                      const double* weights, int D, const double* phi0, int max_outer,
                                      double tol, double hrt_tol, int hrt_max_iter, const vef_opts* opts,
                                      double* phi_out, double* J_out, double* psi, double* dphi,
                                      vef_vef_info* info, void* stream) {
  if (!mesh || !sigma_t || !sigma_s || !omega || !weights || !phi_out || !psi) {
    set_last_error("mesh, sigma_t, sigma_s, omega, weights, phi_out and psi are required");
    return VEF_ERR_INVALID_ARG;
  }
  if (max_outer < 1 || !(tol >= 0.0) || !(hrt_tol > 0.0) || hrt_max_iter < 1) {
    set_last_error("max_outer >= 1, tol >= 0, hrt_tol > 0 and hrt_max_iter >= 1 are required");
    return VEF_ERR_INVALID_ARG;
  }
  Mesh& M = mesh->impl;
  cudaStream_t s = (cudaStream_t)stream;
  const long long En = M.E * M.n, nb = M.nbf * M.nq;
  const long long nJ = M.E * 2LL * (M.p + 2) * (M.p + 1);
  // iterates, transport moments and closures, the zeroth source moment, a J scratch, max-diff word
  const size_t need = (size_t)(2 * En + 4 * En + 2 * nb + En + (J_out ? 0 : nJ) + 1) * sizeof(double);
  vef_status st = ensure_buffer(&M.vef_work, &M.vef_work_cap, need);
  if (st != VEF_OK) return st;
  double* cur = (double*)M.vef_work;
  double* nxt = cur + En;
  double* phi_tr = nxt + En;
  double* P = phi_tr + En;
  double* Eb = P + 3 * En;
  double* Jin = Eb + nb;
  double* Q0 = Jin + nb;
  double* Jbuf = Q0 + En;
  double* J = J_out ? J_out : Jbuf;
  unsigned long long* md = (unsigned long long*)(Jbuf + (J_out ? 0 : nJ));
  const unsigned bl = (unsigned)((En + 255) / 256);
  // Q0 = int q dOmega = 4 pi q for the isotropic source (per steradian)
  scale_kernel<<<bl, 256, 0, s>>>(En, kFourPi, source, Q0);
  if (phi0) VEF_CUDA_TRY(cudaMemcpyAsync(cur, phi0, En * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else VEF_CUDA_TRY(cudaMemsetAsync(cur, 0, En * sizeof(double), s));
  VEF_CUDA_TRY(cudaGetLastError());
  vef_opts o{};
  if (opts) o = *opts;
  else { o.precision = VEF_FP64; }
  int k = 0, converged = 0, hrt_its = 0;
  double change = -1.0;
  for (; k < max_outer; ++k) {
    vef_opts ok = o;
    if (k > 0) ok.flags |= VEF_REUSE_FACTORS;   // sigma_t unchanged: keep the factorisation
    if ((st = vef_sweep(mesh, sigma_t, sigma_s, cur, source, 0, inflow, omega, weights, D, &ok, psi, nullptr,
                        stream)) != VEF_OK)
      return st;
    if ((st = vef_moments(mesh, psi, omega, weights, D, inflow, phi_tr, nullptr, P, nullptr, Eb, Jin, stream)) !=
        VEF_OK)
      return st;
    vef_hrt_info hi{};
    if ((st = vef_hrt_solve(mesh, sigma_t, sigma_s, phi_tr, P, Eb, Jin, Q0, nullptr, hrt_tol, hrt_max_iter, nxt, J,
                            nullptr, &hi, stream)) != VEF_OK)
      return st;
    hrt_its += hi.iterations;
    VEF_CUDA_TRY(cudaMemsetAsync(md, 0, sizeof(unsigned long long), s));
    vef_maxdiff_kernel<<<std::min<unsigned>(bl, 1024u), 256, 0, s>>>(En, nxt, cur, md);
    VEF_CUDA_TRY(cudaGetLastError());
    unsigned long long bits = 0;
    VEF_CUDA_TRY(cudaMemcpyAsync(&bits, md, sizeof(bits), cudaMemcpyDeviceToHost, s));
    VEF_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(&change, &bits, sizeof(change));
    if (dphi) VEF_CUDA_TRY(cudaMemcpyAsync(dphi + k, &change, sizeof(double), cudaMemcpyHostToDevice, s));
    std::swap(cur, nxt);
    if (change <= tol) { converged = 1; ++k; break; }
  }
  VEF_CUDA_TRY(cudaMemcpyAsync(phi_out, cur, En * sizeof(double), cudaMemcpyDeviceToDevice, s));
  VEF_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iterations = k;
    info->converged = converged;
    info->last_change = change;
    info->hrt_iterations = hrt_its;
  }
  st = collect_status(M, s, nullptr);
  if (st != VEF_OK) return st;
  if (!converged) {
    set_last_error("VEF fixed-point iteration reached max_outer before its tolerance");
    return VEF_ERR_NOT_CONVERGED;
  }
  return VEF_OK;
}
