// Angular moments and VEF closures (paper Eq. vef_disc; E_b and J_in as defined after
// Eq. mlbc).  All sums over directions accumulate in FP64.
//
//   phi = sum_d w_d psi_d,  J = sum_d w_d Omega_d psi_d,  P = sum_d w_d Omega_d (x) Omega_d psi_d
// are DG functions (nodal coefficients, since the sums are linear in psi).  The
// Eddington tensor is the ratio P/phi evaluated pointwise at the volume Gauss points;
// the boundary factor E_b = sum w |Omega.n_hat| psi / sum w psi uses the interior trace
// at the boundary face Gauss points, and J_in = sum_{Omega.n<0} w (Omega.n_hat) psi_bar.
#include <cmath>

#include "device.cuh"

namespace vef {

__device__ __forceinline__ int face_dof_rt(int p, int f, int t) {
  const int q = p + 1;
  return f == 0 ? t : (f == 1 ? p + q * t : (f == 2 ? t + q * p : q * t));
}

// one thread per (e, i): six FP64 accumulators over the directions
__global__ void moments_nodal_kernel(int D, long long En, const double* __restrict__ om,
                                     const double* __restrict__ w, const double* __restrict__ psi,
                                     double* __restrict__ phi, double* __restrict__ J,
                                     double* __restrict__ P) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= En) return;
  double s0 = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
  for (int d = 0; d < D; ++d) {
    const double v = w[d] * psi[(size_t)d * En + t];
    const double mu = om[2 * d], eta = om[2 * d + 1];
    s0 += v;
    sx += mu * v;
    sy += eta * v;
    sxx += mu * mu * v;
    sxy += mu * eta * v;
    syy += eta * eta * v;
  }
  if (phi) phi[t] = s0;
  if (J) { J[t] = sx; J[En + t] = sy; }
  if (P) { P[t] = sxx; P[En + t] = sxy; P[2 * En + t] = syy; }
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
  if (phiw || J || Pw) {
    KTimer kt(&M, VEF_K_MOMENTS, s);
    moments_nodal_kernel<<<nblk(En, 256), 256, 0, s>>>(D, En, S->omega_dev, S->weights_dev, psi,
                                                        phiw, J, Pw);
  }
  if (Eten) {
    KTimer kt(&M, VEF_K_MOMENTS, s);
    eddington_kernel<<<nblk(M.E * M.nq * M.nq, 256), 256, 0, s>>>(M.E, M.tab, phiw, Pw, Eten,
                                                                  M.dev_status);
  }
  if (Eb || Jin) {
    KTimer kt(&M, VEF_K_MOMENTS, s);
    boundary_kernel<<<nblk(M.nbf * M.nq, 128), 128, 0, s>>>(D, M.nx, M.ny, M.E, M.tab, S->omega_dev,
                                                           S->weights_dev, psi, M.nds, inflow, Eb,
                                                           Jin, M.dev_status);
  }
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}
