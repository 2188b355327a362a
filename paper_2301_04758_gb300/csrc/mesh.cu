// Mesh creation and geometric factors (paper Sec. "Description of the Mesh" and
// "Integration Transformations").
//
// Each element is the Q_m image of [0,1]^2 through (m+1)^2 Gauss-Lobatto control points.
// Per element the kernels here compute, once, the direction-independent matrices of
// the upwind DG operator (test index i, trial index j, tensor GLL-Lagrange basis):
//   M_ij  = sum_q w_q J_q l_i l_j                              (mass)
//   Gx_ij = sum_q w_q [adj(F)_00 dl_i/dxi + adj(F)_10 dl_i/deta] l_j
//   Gy_ij = sum_q w_q [adj(F)_01 dl_i/dxi + adj(F)_11 dl_i/deta] l_j
// so that the volume part of the element matrix for Omega = (mu, eta) is
//   sigma_t M - mu Gx - eta Gy   (since J Omega . F^{-T} grad_ref = (adj(F) Omega) . grad_ref),
// and at the nq Gauss points of each face the outward normal times the length element
//   n ds = adj(F)^T n_ref ds_ref.
// On a face shared by two elements the right/top element side is computed and the
// left/bottom side stored as its exact negation, so both sides take the same upwind
// decision at every point.
#include <cmath>
#include <cstring>

#include "common.h"

namespace vef {

struct MapTab {
  int m, nq;
  double lv[kMaxM + 1][kMaxNq + 2];  // mesh-order Lagrange values at GL points, then 0, then 1
  double ld[kMaxM + 1][kMaxNq + 2];
};

__device__ __forceinline__ void map_jac(const double* __restrict__ ctrl, const MapTab& mt, int kx,
                                        int ky, double F[2][2]) {
  // F = [[dx/dxi, dx/deta], [dy/dxi, dy/deta]] at reference point (pt kx, pt ky)
  F[0][0] = F[0][1] = F[1][0] = F[1][1] = 0.0;
  const int q = mt.m + 1;
  for (int b = 0; b < q; ++b) {
    for (int a = 0; a < q; ++a) {
      const double x = ctrl[2 * (a + q * b)];
      const double y = ctrl[2 * (a + q * b) + 1];
      const double dxi = mt.ld[a][kx] * mt.lv[b][ky];
      const double deta = mt.lv[a][kx] * mt.ld[b][ky];
      F[0][0] += x * dxi;
      F[0][1] += x * deta;
      F[1][0] += y * dxi;
      F[1][1] += y * deta;
    }
  }
}

// One thread per (element, volume point): w_q J and w_q adj(F).
__global__ void geom_vol_kernel(const double* __restrict__ ctrl, long long E, MapTab mt,
                                Tab1D tab, double* __restrict__ g5) {
  const int nq = tab.nq;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * nq * nq) return;
  long long e = t / (nq * nq);
  int q = (int)(t % (nq * nq));
  int k1 = q % nq, k2 = q / nq;
  double F[2][2];
  map_jac(ctrl + e * 2 * (mt.m + 1) * (mt.m + 1), mt, k1, k2, F);
  const double w = tab.glw[k1] * tab.glw[k2];
  double* o = g5 + t * 5;
  o[0] = w * (F[0][0] * F[1][1] - F[0][1] * F[1][0]);
  o[1] = w * F[1][1];   // adj00
  o[2] = -w * F[0][1];  // adj01
  o[3] = -w * F[1][0];  // adj10
  o[4] = w * F[0][0];   // adj11
}

// One thread per (element, i, j): M, Gx, Gy entries.
__global__ void geom_mat_kernel(const double* __restrict__ g5, long long E, Tab1D tab,
                                double* __restrict__ M, double* __restrict__ Gx,
                                double* __restrict__ Gy) {
  const int np1 = tab.np1, n = np1 * np1, nq = tab.nq;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * n * n) return;
  long long e = t / (n * n);
  int ij = (int)(t % (n * n));
  int i = ij / n, j = ij % n;
  int ia = i % np1, ib = i / np1, ja = j % np1, jb = j / np1;
  double m = 0.0, gx = 0.0, gy = 0.0;
  const double* g = g5 + e * nq * nq * 5;
  for (int k2 = 0; k2 < nq; ++k2) {
    for (int k1 = 0; k1 < nq; ++k1) {
      const double* o = g + (k1 + nq * k2) * 5;
      const double bi = tab.l[ia][k1] * tab.l[ib][k2];
      const double bj = tab.l[ja][k1] * tab.l[jb][k2];
      const double dxi = tab.dl[ia][k1] * tab.l[ib][k2];
      const double deta = tab.l[ia][k1] * tab.dl[ib][k2];
      m += o[0] * bi * bj;
      gx += (o[1] * dxi + o[3] * deta) * bj;
      gy += (o[2] * dxi + o[4] * deta) * bj;
    }
  }
  M[t] = m;
  Gx[t] = gx;
  Gy[t] = gy;
}

// One thread per (element, face, point): n ds = adj(F)^T n_ref ds_ref (weight not included).
__global__ void geom_face_kernel(const double* __restrict__ ctrl, long long E, MapTab mt, int nq,
                                 double* __restrict__ nds) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * 4 * nq) return;
  long long e = t / (4 * nq);
  int f = (int)((t / nq) % 4), k = (int)(t % nq);
  const int P0 = nq, P1 = nq + 1;  // table columns of reference coordinates 0 and 1
  int kx, ky;
  if (f == 0) { kx = k; ky = P0; }
  else if (f == 1) { kx = P1; ky = k; }
  else if (f == 2) { kx = k; ky = P1; }
  else { kx = P0; ky = k; }
  double F[2][2];
  map_jac(ctrl + e * 2 * (mt.m + 1) * (mt.m + 1), mt, kx, ky, F);
  // adj(F)^T = [[F11, -F10], [-F01, F00]]
  double nx, ny;
  if (f == 0) { nx = F[1][0]; ny = -F[0][0]; }        // n_ref = (0,-1)
  else if (f == 1) { nx = F[1][1]; ny = -F[0][1]; }   // (1, 0)
  else if (f == 2) { nx = -F[1][0]; ny = F[0][0]; }   // (0, 1)
  else { nx = -F[1][1]; ny = F[0][1]; }               // (-1, 0)
  nds[2 * t] = nx;
  nds[2 * t + 1] = ny;
}

// Left and bottom faces of interior elements take the negated value of the neighbour's
// right / top face.
__global__ void geom_canon_kernel(int nx, int ny, int nq, double* __restrict__ nds) {
  long long E = (long long)nx * ny;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * 2 * nq) return;
  long long e = t / (2 * nq);
  int which = (int)((t / nq) % 2), k = (int)(t % nq);
  int i = (int)(e % nx), j = (int)(e / nx);
  if (which == 0) {  // bottom face of e <- top face of (i, j-1)
    if (j == 0) return;
    long long nb = e - nx;
    nds[((e * 4 + 0) * nq + k) * 2 + 0] = -nds[((nb * 4 + 2) * nq + k) * 2 + 0];
    nds[((e * 4 + 0) * nq + k) * 2 + 1] = -nds[((nb * 4 + 2) * nq + k) * 2 + 1];
  } else {           // left face of e <- right face of (i-1, j)
    if (i == 0) return;
    long long nb = e - 1;
    nds[((e * 4 + 3) * nq + k) * 2 + 0] = -nds[((nb * 4 + 1) * nq + k) * 2 + 0];
    nds[((e * 4 + 3) * nq + k) * 2 + 1] = -nds[((nb * 4 + 1) * nq + k) * 2 + 1];
  }
}

// g[e][j] = sum_q w_q J_q chi(x_q) l_j(x_q): weights of R = int_region phi dx over the DG
// nodal values of phi, with the box indicator chi evaluated at the volume Gauss points.
__global__ void region_weights_kernel(const double* __restrict__ ctrl, long long E, MapTab mt, Tab1D tab,
                                      double x0, double y0, double x1, double y1, double* __restrict__ g) {
  const int np1 = tab.np1, n = np1 * np1, nq = tab.nq;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * n) return;
  const long long e = t / n;
  const int j = (int)(t % n), ja = j % np1, jb = j / np1;
  const double* c = ctrl + e * 2 * (mt.m + 1) * (mt.m + 1);
  const int q = mt.m + 1;
  double acc = 0.0;
  for (int k2 = 0; k2 < nq; ++k2)
    for (int k1 = 0; k1 < nq; ++k1) {
      double x = 0.0, y = 0.0;
      for (int b = 0; b < q; ++b)
        for (int a = 0; a < q; ++a) {
          const double l = mt.lv[a][k1] * mt.lv[b][k2];
          x += c[2 * (a + q * b)] * l;
          y += c[2 * (a + q * b) + 1] * l;
        }
      if (x < x0 || x > x1 || y < y0 || y > y1) continue;
      double F[2][2];
      map_jac(c, mt, k1, k2, F);
      const double J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
      acc += tab.glw[k1] * tab.glw[k2] * J * tab.l[ja][k1] * tab.l[jb][k2];
    }
  g[t] = acc;
}

template <typename T>
__global__ void to_float_kernel(const double* __restrict__ a, T* __restrict__ b, long long n) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (T)a[t];
}

static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

vef_status ensure_buffer(void** ptr, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *ptr) return VEF_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  cudaError_t err = cudaMalloc(ptr, bytes);
  if (err != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    set_last_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes failed");
    return VEF_ERR_OOM;
  }
  *cap = bytes;
  return VEF_OK;
}

vef_status mesh_float_copies(Mesh* mesh, cudaStream_t stream) {
  if (mesh->Mmat32) return VEF_OK;
  const long long nn = mesh->E * mesh->n * mesh->n;
  const long long nf = mesh->E * 4 * mesh->nq * 2;
  VEF_CUDA_TRY(cudaMalloc(&mesh->Mmat32, nn * sizeof(float)));
  VEF_CUDA_TRY(cudaMalloc(&mesh->Gx32, nn * sizeof(float)));
  VEF_CUDA_TRY(cudaMalloc(&mesh->Gy32, nn * sizeof(float)));
  VEF_CUDA_TRY(cudaMalloc(&mesh->nds32, nf * sizeof(float)));
  to_float_kernel<<<blocks_for(nn, 256), 256, 0, stream>>>(mesh->Mmat, mesh->Mmat32, nn);
  to_float_kernel<<<blocks_for(nn, 256), 256, 0, stream>>>(mesh->Gx, mesh->Gx32, nn);
  to_float_kernel<<<blocks_for(nn, 256), 256, 0, stream>>>(mesh->Gy, mesh->Gy32, nn);
  to_float_kernel<<<blocks_for(nf, 256), 256, 0, stream>>>(mesh->nds, mesh->nds32, nf);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

void destroy_events(Mesh& M);

Mesh::~Mesh() {
  destroy_events(*this);
  if (hrt_graph) cudaGraphExecDestroy(hrt_graph);
  schedules.clear();
  cudaFree(ctrl_dev);
  cudaFree(Mmat);
  cudaFree(Gx);
  cudaFree(Gy);
  cudaFree(nds);
  cudaFree(Mmat32);
  cudaFree(Gx32);
  cudaFree(Gy32);
  cudaFree(nds32);
  cudaFree(dev_status);
  cudaFree(vef_work);
  cudaFree(bvol);
  cudaFree(work);
  cudaFree(work2);
  cudaFree(ybuf);
  cudaFree(ready_flags);
}

Schedule::~Schedule() {
  cudaFree(dir_lev0);
  cudaFree(lev_begin);
  cudaFree(lev_gbegin);
  cudaFree(lev_mbegin);
  cudaFree(member_info);
  cudaFree(member_nbpos);
  cudaFree(slot_first);
  cudaFree(slot_count);
  cudaFree(member_code);
  cudaFree(member_of);
  cudaFree(faceinfo);
  cudaFree(omega_dev);
  cudaFree(weights_dev);
  cudaFree(rec64);
  cudaFree(rec32);
  cudaFree(a64);
  cudaFree(pivot_list);
  cudaFree(adj_link);
  cudaFree(tslot);
  cudaFree(slot_gid);
  cudaFree(grp_slot);
  cudaFree(grp_nt);
  cudaFree(grp_toff);
  cudaFree(grec64);
  cudaFree(grec32);
}

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_mesh_create(int nx, int ny, int mesh_order, int p, double alpha,
                                      const double* ctrl_pts, vef_mesh* out) {
  if (!out) { set_last_error("out is NULL"); return VEF_ERR_INVALID_ARG; }
  *out = nullptr;
  if (nx < 1 || ny < 1 || (long long)nx * ny > kMaxE) {
    set_last_error("nx, ny must be >= 1 with nx*ny <= 2^22");
    return VEF_ERR_INVALID_ARG;
  }
  if (mesh_order < 1 || mesh_order > kMaxM || p < 1 || p > kMaxP) {
    set_last_error("mesh_order and p must be in 1..4");
    return VEF_ERR_INVALID_ARG;
  }
  if (!std::isfinite(alpha)) { set_last_error("alpha must be finite"); return VEF_ERR_INVALID_ARG; }
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  std::unique_ptr<vef_mesh_s> h(new vef_mesh_s());
  Mesh& M = h->impl;
  M.device = dev;
  M.nx = nx; M.ny = ny; M.m = mesh_order; M.p = p;
  M.n = (p + 1) * (p + 1);
  M.nq = p + 2;
  M.E = (long long)nx * ny;
  M.nbf = 2LL * nx + 2LL * ny;
  M.tab = make_tab1d(p);
  const int q = mesh_order + 1;
  // control points (host)
  std::vector<double> ctrl((size_t)M.E * q * q * 2);
  if (ctrl_pts) {
    std::memcpy(ctrl.data(), ctrl_pts, ctrl.size() * sizeof(double));
  } else {
    double g[kMaxM + 1];
    gll_nodes(mesh_order, g);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int b = 0; b < q; ++b)
          for (int a = 0; a < q; ++a) {
            const double X = (i + g[a]) / nx, Y = (j + g[b]) / ny;
            const double d = alpha * std::sin(2.0 * M_PI * X) * std::sin(2.0 * M_PI * Y);
            size_t o = (((size_t)j * nx + i) * q * q + a + q * b) * 2;
            ctrl[o] = X + d;
            ctrl[o + 1] = Y + d;
          }
  }
  // mesh-order Lagrange tables at the GL points and at 0, 1
  MapTab mt{};
  mt.m = mesh_order;
  mt.nq = M.nq;
  {
    double g[kMaxM + 1];
    gll_nodes(mesh_order, g);
    for (int k = 0; k < M.nq + 2; ++k) {
      double x = k < M.nq ? M.tab.gl[k] : (k == M.nq ? 0.0 : 1.0);
      double v[kMaxM + 1], d[kMaxM + 1];
      lagrange_eval(q, g, x, v, d);
      for (int a = 0; a < q; ++a) { mt.lv[a][k] = v[a]; mt.ld[a][k] = d[a]; }
    }
  }
  double* dctrl = nullptr;
  double* g5 = nullptr;
  const long long nn = M.E * M.n * M.n;
  auto cleanup = [&]() { cudaFree(g5); };
  cudaError_t err = cudaSuccess;
  if ((err = cudaMalloc(&dctrl, ctrl.size() * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&g5, (size_t)M.E * M.nq * M.nq * 5 * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&M.Mmat, nn * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&M.Gx, nn * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&M.Gy, nn * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&M.nds, (size_t)M.E * 4 * M.nq * 2 * sizeof(double))) != cudaSuccess ||
      (err = cudaMalloc(&M.dev_status, 8 * sizeof(unsigned int))) != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    set_last_error("device allocation failed in vef_mesh_create");
    return VEF_ERR_OOM;
  }
  VEF_CUDA_TRY(cudaMemset(M.dev_status, 0, 8 * sizeof(unsigned int)));
  VEF_CUDA_TRY(cudaMemcpy(dctrl, ctrl.data(), ctrl.size() * sizeof(double), cudaMemcpyHostToDevice));
  const long long nv = M.E * M.nq * M.nq;
  geom_vol_kernel<<<blocks_for(nv, 128), 128>>>(dctrl, M.E, mt, M.tab, g5);
  geom_mat_kernel<<<blocks_for(nn, 128), 128>>>(g5, M.E, M.tab, M.Mmat, M.Gx, M.Gy);
  const long long nf = M.E * 4 * M.nq;
  geom_face_kernel<<<blocks_for(nf, 128), 128>>>(dctrl, M.E, mt, M.nq, M.nds);
  geom_canon_kernel<<<blocks_for(M.E * 2 * M.nq, 128), 128>>>(nx, ny, M.nq, M.nds);
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  if (err != cudaSuccess) { cleanup(); return cuda_fail(err, "geometry kernels"); }
  M.ctrl_dev = dctrl;
  M.map_tab = std::make_shared<MapTab>(mt);
  M.nds_host.resize((size_t)nf * 2);
  err = cudaMemcpy(M.nds_host.data(), M.nds, nf * 2 * sizeof(double), cudaMemcpyDeviceToHost);
  cleanup();
  if (err != cudaSuccess) return cuda_fail(err, "copy of face normals");
  *out = h.release();
  return VEF_OK;
}

extern "C" vef_status vef_mesh_destroy(vef_mesh mesh) {
  if (!mesh) return VEF_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(mesh->impl.device);
  cudaDeviceSynchronize();
  delete mesh;
  cudaSetDevice(cur);
  return VEF_OK;
}

extern "C" vef_status vef_mesh_query(vef_mesh mesh, vef_mesh_desc* out) {
  if (!mesh || !out) { set_last_error("NULL argument"); return VEF_ERR_INVALID_ARG; }
  const Mesh& M = mesh->impl;
  out->nx = M.nx; out->ny = M.ny; out->mesh_order = M.m; out->p = M.p;
  out->n = M.n; out->nq = M.nq; out->E = M.E; out->nbf = M.nbf;
  return VEF_OK;
}

extern "C" vef_status vef_region_weights(vef_mesh mesh, double x0, double y0, double x1, double y1,
                                         double* g, void* stream) {
  if (!mesh || !g) { set_last_error("mesh and g are required"); return VEF_ERR_INVALID_ARG; }
  const Mesh& M = mesh->impl;
  const MapTab& mt = *std::static_pointer_cast<MapTab>(M.map_tab);
  region_weights_kernel<<<blocks_for(M.E * M.n, 128), 128, 0, (cudaStream_t)stream>>>(
      M.ctrl_dev, M.E, mt, M.tab, x0, y0, x1, y1, g);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}
