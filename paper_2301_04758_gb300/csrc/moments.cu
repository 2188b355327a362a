// Angular moments and VEF closures (paper Eq. vef_disc; E_b and J_in as defined after
// Eq. mlbc).  All sums over directions accumulate in FP64.
//
//   phi = sum_d w_d psi_d,  J = sum_d w_d Omega_d psi_d,  P = sum_d w_d Omega_d (x) Omega_d psi_d
// are DG functions (nodal coefficients, since the sums are linear in psi).  The
// Eddington tensor is the ratio P/phi evaluated pointwise at the volume Gauss points;
// the boundary factor E_b = sum w |Omega.n_hat| psi / sum w psi uses the interior trace
// at the boundary face Gauss points, and J_in = sum_{Omega.n<0} w (Omega.n_hat) psi_bar.
#include <cmath>
#include <cstdint>

#include "device.cuh"

namespace vef {

__device__ __forceinline__ int face_dof_rt(int p, int f, int t) {
  const int q = p + 1;
  return f == 0 ? t : (f == 1 ? p + q * t : (f == 2 ? t + q * p : q * t));
}

// Nodal moments: the six sums over directions are a (6 x D) by (D x E n) product with the
// per-direction coefficients w, w mu, w eta, w mu^2, w mu eta, w eta^2, kept in shared
// memory.  Every psi value costs its six FP64 FMAs and nothing else: at 1.5 flop per byte
// read the pass is bound by FP64 issue on this GPU, not by HBM.  A thread takes two
// consecutive dofs (one 16-byte load per direction, coalesced across the warp) and keeps
// twelve FP64 accumulators; four directions are loaded ahead to keep loads in flight.
constexpr int kMomBlock = 256;
__global__ void __launch_bounds__(kMomBlock)
moments_nodal_kernel(int D, long long En, const double* __restrict__ om, const double* __restrict__ w,
                     const double* __restrict__ psi, double* __restrict__ phi, double* __restrict__ J,
                     double* __restrict__ P) {
  extern __shared__ double cw[];   // [D][6]
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    const double wd = w[d], mu = om[2 * d], eta = om[2 * d + 1];
    cw[6 * d + 0] = wd;
    cw[6 * d + 1] = wd * mu;
    cw[6 * d + 2] = wd * eta;
    cw[6 * d + 3] = wd * mu * mu;
    cw[6 * d + 4] = wd * mu * eta;
    cw[6 * d + 5] = wd * eta * eta;
  }
  __syncthreads();
  const long long t = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  if (t >= En) return;
  // 16-byte aligned pairs: E n even and psi itself 16-byte aligned
  const bool pair = t + 1 < En && (En & 1) == 0 && (reinterpret_cast<uintptr_t>(psi) & 15) == 0;
  double a[6] = {0, 0, 0, 0, 0, 0}, b[6] = {0, 0, 0, 0, 0, 0};
  int d = 0;
  if (pair) {
    const double2* p2 = reinterpret_cast<const double2*>(psi + t);
    const long long stride2 = En / 2;
    for (; d + 4 <= D; d += 4) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldcs(p2 + (size_t)(d + u) * stride2);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double* c = cw + 6 * (d + u);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          a[k] = fma(c[k], v[u].x, a[k]);
          b[k] = fma(c[k], v[u].y, b[k]);
        }
      }
    }
    for (; d < D; ++d) {
      const double2 v = __ldcs(p2 + (size_t)d * stride2);
      const double* c = cw + 6 * d;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        a[k] = fma(c[k], v.x, a[k]);
        b[k] = fma(c[k], v.y, b[k]);
      }
    }
  } else {
    for (; d < D; ++d) {
      const double* c = cw + 6 * d;
      const double v0 = psi[(size_t)d * En + t];
      const double v1 = t + 1 < En ? psi[(size_t)d * En + t + 1] : 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        a[k] = fma(c[k], v0, a[k]);
        b[k] = fma(c[k], v1, b[k]);
      }
    }
  }
  const bool two = t + 1 < En;
  if (phi) { phi[t] = a[0]; if (two) phi[t + 1] = b[0]; }
  if (J) {
    J[t] = a[1]; J[En + t] = a[2];
    if (two) { J[t + 1] = b[1]; J[En + t + 1] = b[2]; }
  }
  if (P) {
    P[t] = a[3]; P[En + t] = a[4]; P[2 * En + t] = a[5];
    if (two) { P[t + 1] = b[3]; P[En + t + 1] = b[4]; P[2 * En + t + 1] = b[5]; }
  }
}

// one thread per (e, q): E = P(x_q) / phi(x_q)
__global__ void eddington_kernel(long long E, Tab1D tab, const double* __restrict__ phi,
                                 const double* __restrict__ P, double* __restrict__ Eten,
                                 unsigned int* status) {
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
    f += B * phi[o];
    a += B * P[o];
    b += B * P[En + o];
    c += B * P[2 * En + o];
  }
  const size_t Eq = (size_t)E * nq2;
  if (f > 1e-300) {
    Eten[t] = a / f;
    Eten[Eq + t] = b / f;
    Eten[2 * Eq + t] = c / f;
  } else {
    Eten[t] = Eten[Eq + t] = Eten[2 * Eq + t] = nan("");
    atomicOr(status, kDevNonpositive);
  }
}

// one thread per (boundary face, point)
__global__ void boundary_kernel(int D, int nx, int ny, long long E, Tab1D tab,
                                const double* __restrict__ om, const double* __restrict__ w,
                                const double* __restrict__ psi, const double* __restrict__ nds,
                                const double* __restrict__ inflow, double* __restrict__ Eb,
                                double* __restrict__ Jin, unsigned int* status) {
  const int nq = tab.nq, p = tab.p, n = tab.np1 * tab.np1;
  const long long nbf = 2LL * nx + 2LL * ny;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nbf * nq) return;
  const int bf = (int)(t / nq), k = (int)(t % nq);
  int e, f;
  if (bf < nx) { e = bf; f = 0; }
  else if (bf < nx + ny) { e = (bf - nx) * nx + nx - 1; f = 1; }
  else if (bf < 2 * nx + ny) { e = (ny - 1) * nx + (bf - nx - ny); f = 2; }
  else { e = (bf - 2 * nx - ny) * nx; f = 3; }
  const double* v = nds + (((size_t)e * 4 + f) * nq + k) * 2;
  const double len = sqrt(v[0] * v[0] + v[1] * v[1]);
  const double nxh = v[0] / len, nyh = v[1] / len;
  double num = 0, den = 0, jin = 0;
  for (int d = 0; d < D; ++d) {
    const double* pe = psi + ((size_t)d * E + e) * n;
    double tr = 0;
    for (int a = 0; a <= p; ++a) tr += tab.l[a][k] * pe[face_dof_rt(p, f, a)];
    const double on = om[2 * d] * nxh + om[2 * d + 1] * nyh;
    num += w[d] * fabs(on) * tr;
    den += w[d] * tr;
    if (inflow && on < 0.0) jin += w[d] * on * inflow[((size_t)d * nbf + bf) * nq + k];
  }
  if (Eb) {
    if (den > 1e-300) Eb[t] = num / den;
    else { Eb[t] = nan(""); atomicOr(status, kDevNonpositive); }
  }
  if (Jin) Jin[t] = jin;
}

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_moments(vef_mesh mesh, const double* psi, const double* omega,
                                  const double* weights, int D, const double* inflow, double* phi,
                                  double* J, double* P, double* Eten, double* Eb, double* Jin,
                                  void* stream) {
  if (!mesh || !psi || !omega || !weights) { set_last_error("mesh, psi, omega, weights are required"); return VEF_ERR_INVALID_ARG; }
  if (D < 1 || D > kMaxD) { set_last_error("D must be in 1..1023"); return VEF_ERR_INVALID_ARG; }
  Mesh& M = mesh->impl;
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != M.device) { set_last_error("mesh belongs to another device"); return VEF_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  vef_status st;
  Schedule* S = get_schedule(&M, omega, weights, D, s, &st);  // device copies of omega / weights
  if (!S) return st;
  const long long En = M.E * M.n;
  double* phiw = phi;
  double* Pw = P;
  if (Eten && (!phi || !P)) {
    if ((st = ensure_buffer((void**)&M.work, &M.work_cap, (size_t)4 * En * sizeof(double))) != VEF_OK)
      return st;
    if (!phiw) phiw = M.work;
    if (!Pw) Pw = M.work + En;
  }
  KTimer kt(&M, VEF_K_MOMENTS, s);   // the whole closure pass counts as one launch
  if (phiw || J || Pw) {
    moments_nodal_kernel<<<nblk((En + 1) / 2, kMomBlock), kMomBlock, (size_t)6 * D * sizeof(double), s>>>(
        D, En, S->omega_dev, S->weights_dev, psi, phiw, J, Pw);
  }
  if (Eten) {
    eddington_kernel<<<nblk(M.E * M.nq * M.nq, 256), 256, 0, s>>>(M.E, M.tab, phiw, Pw, Eten,
                                                                  M.dev_status);
  }
  if (Eb || Jin) {
    boundary_kernel<<<nblk(M.nbf * M.nq, 128), 128, 0, s>>>(D, M.nx, M.ny, M.E, M.tab, S->omega_dev,
                                                           S->weights_dev, psi, M.nds, inflow, Eb,
                                                           Jin, M.dev_status);
  }
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}
