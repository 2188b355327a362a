// Hybridized Raviart-Thomas (HRT) VEF solve: element-local elimination, the reduced
// system for the Lagrange multiplier, and the recovery of the scalar flux and current
// (paper Sec. "Hybridization": "Extension to VEF" and "Implementation Details").
//
// Per element K the local mixed system couples the broken RT_p current J and the Y_p
// scalar flux phi:
//     [ A  G ] [J  ]   [g - C2 lambda]        A  = int sigma_t v.J + int_Gb (1/E_b)(v.E n)(J.n)
//     [ D  Ma] [phi] = [f            ]        G  = -int grad v : E phi   (Piola gradient)
//                                             D  = int u div J,  Ma = int sigma_a u phi
//                                             g  = int v.Q1 + 2 int_Gb (1/E_b)(v.E n) J_in
//                                             f  = int u Q0
// with C2 lambda = int_G0 (v.{E} n) lambda (the face multipliers) and the constraint
// C1 J = int_G0 mu [[J.n]] = 0.  hrt_local_kernel assembles these blocks for one element per
// CTA in shared memory, inverts [[A, G], [D, Ma]] by Gauss-Jordan elimination with partial
// pivoting (the block is indefinite in general), and forms the element's share of the
// reduced system,
//     H_e = C1 W C2,   r_e = C1 (W g + X f),   [[W, X], [Y, Z]] = [[A, G], [D, Ma]]^{-1}.
// The multiplier system H lambda = r (H = sum_e H_e over the interior faces, not symmetric
// for a general Eddington tensor) is solved by BiCGStab with a Jacobi preconditioner,
// the matrix applied element by element (z_e = H_e lambda_e, then a per-face gather of the
// two sides, no atomics).  hrt_recover_kernel then forms J and phi element by element.
//
// Spaces (identical to the CPU reference of this discretisation): RT_p on the reference
// square with the x component in Q_{p+1} x Q_p and the y component in Q_p x Q_{p+1}, nodal
// at the p+2 Gauss-Lobatto points across (normal flux on the end nodes) and the p+1
// Gauss-Legendre points along; contravariant Piola transform v = F v_hat / J, whose
// gradient (d v / d xi) F^{-1} uses the map's second derivatives; the transport's DG basis
// for phi; degree-p Lagrange multipliers at the p+1 Gauss-Legendre points of each interior
// face; the transport's Gauss-Legendre rules, so the Eddington tensor is P / phi from the
// closure pass's nodal moments.  Interior faces: vertical first (j (nx-1) + i), then
// horizontal ((nx-1) ny + j nx + i).
#include <algorithm>
#include <cmath>
#include <vector>

#include "device.cuh"

namespace vef {
namespace {

// 1D tables of one order p and mesh order m: index k < nq is the Gauss point s_k, nq is the
// point 0 and nq + 1 the point 1.
struct HrtTab {
  int p, m, nq;
  double w[kMaxNq];                               // Gauss weights
  double cl[kMaxP + 2][kMaxNq + 2], dcl[kMaxP + 2][kMaxNq + 2];   // p+2 Gauss-Lobatto nodes
  double op[kMaxP + 1][kMaxNq + 2], dop[kMaxP + 1][kMaxNq + 2];   // p+1 Gauss-Legendre nodes
  double dg[kMaxP + 1][kMaxNq + 2];               // DG basis (p+1 Gauss-Lobatto nodes)
  double mv[kMaxM + 1][kMaxNq + 2], md[kMaxM + 1][kMaxNq + 2], mdd[kMaxM + 1][kMaxNq + 2];
};

HrtTab make_hrt_tab(int p, int m) {
  HrtTab t{};
  t.p = p;
  t.m = m;
  t.nq = p + 2;
  double s[kMaxNq], gw[kMaxNq];
  gauss_legendre(t.nq, s, gw);
  for (int k = 0; k < t.nq; ++k) t.w[k] = gw[k];
  double cl[kMaxP + 2], op[kMaxP + 1], dg[kMaxP + 1], mn[kMaxM + 1], dummy[kMaxNq];
  gll_nodes(p + 1, cl);
  gauss_legendre(p + 1, op, dummy);
  gll_nodes(p, dg);
  gll_nodes(m, mn);
  for (int k = 0; k < t.nq + 2; ++k) {
    const double x = k < t.nq ? s[k] : (k == t.nq ? 0.0 : 1.0);
    double v[kMaxP + 2], d[kMaxP + 2];
    lagrange_eval(p + 2, cl, x, v, d);
    for (int a = 0; a < p + 2; ++a) { t.cl[a][k] = v[a]; t.dcl[a][k] = d[a]; }
    lagrange_eval(p + 1, op, x, v, d);
    for (int a = 0; a < p + 1; ++a) { t.op[a][k] = v[a]; t.dop[a][k] = d[a]; }
    lagrange_eval(p + 1, dg, x, v, d);
    for (int a = 0; a < p + 1; ++a) t.dg[a][k] = v[a];
    // control-point basis: values, first and second derivatives (second by differencing the
    // exact first derivatives would lose digits; use the product-rule sum instead)
    lagrange_eval(m + 1, mn, x, v, d);
    for (int a = 0; a <= m; ++a) {
      t.mv[a][k] = v[a];
      t.md[a][k] = d[a];
      double s2 = 0.0;
      for (int i = 0; i <= m; ++i) {
        if (i == a) continue;
        for (int j = 0; j <= m; ++j) {
          if (j == a || j == i) continue;
          double term = 1.0 / ((mn[a] - mn[i]) * (mn[a] - mn[j]));
          for (int c = 0; c <= m; ++c)
            if (c != a && c != i && c != j) term *= (x - mn[c]) / (mn[a] - mn[c]);
          s2 += term;
        }
      }
      t.mdd[a][k] = s2;
    }
  }
  return t;
}

template <int P>
struct HrtShape {
  static constexpr int Q = P + 1, N = Q * Q, NQ = P + 2, NQ2 = NQ * NQ;
  static constexpr int NX = (P + 2) * (P + 1);   // dofs of one component
  static constexpr int NJ = 2 * NX;
  static constexpr int MM = NJ + N;               // local system size
  static constexpr int LD = MM + 1;
  static constexpr int NL = P + 1, NL4 = 4 * NL;
};

// reference RT basis function a at table points (kx, ky): value (2) and d/dxi, d/deta (2 each)
template <int P>
__device__ __forceinline__ void rt_ref(const HrtTab& t, int a, int kx, int ky, double v[2], double dxi[2],
                                       double deta[2]) {
  using S = HrtShape<P>;
  v[0] = v[1] = dxi[0] = dxi[1] = deta[0] = deta[1] = 0.0;
  if (a < S::NX) {
    const int ax = a % (P + 2), bx = a / (P + 2);
    v[0] = t.cl[ax][kx] * t.op[bx][ky];
    dxi[0] = t.dcl[ax][kx] * t.op[bx][ky];
    deta[0] = t.cl[ax][kx] * t.dop[bx][ky];
  } else {
    const int b = a - S::NX, ay = b % (P + 1), by = b / (P + 1);
    v[1] = t.op[ay][kx] * t.cl[by][ky];
    dxi[1] = t.dop[ay][kx] * t.cl[by][ky];
    deta[1] = t.op[ay][kx] * t.dcl[by][ky];
  }
}

// map Jacobian F (row-major [i][k] = d x_i / d xi_k) and second derivatives
// H[i][k][l] = d^2 x_i / d xi_k d xi_l at table point (kx, ky)
__device__ __forceinline__ void map_geom(const double* __restrict__ c, const HrtTab& t, int kx, int ky,
                                         double F[4], double H[8]) {
  for (int i = 0; i < 4; ++i) F[i] = 0.0;
  for (int i = 0; i < 8; ++i) H[i] = 0.0;
  const int q = t.m + 1;
  for (int b = 0; b < q; ++b)
    for (int a = 0; a < q; ++a) {
      const double cx = c[2 * (a + q * b)], cy = c[2 * (a + q * b) + 1];
      const double dx = t.md[a][kx] * t.mv[b][ky], dy = t.mv[a][kx] * t.md[b][ky];
      const double xx = t.mdd[a][kx] * t.mv[b][ky], xy = t.md[a][kx] * t.md[b][ky],
                   yy = t.mv[a][kx] * t.mdd[b][ky];
      F[0] += cx * dx; F[1] += cx * dy; F[2] += cy * dx; F[3] += cy * dy;
      H[0] += cx * xx; H[1] += cx * xy; H[2] += cx * xy; H[3] += cx * yy;   // x: [k][l]
      H[4] += cy * xx; H[5] += cy * xy; H[6] += cy * xy; H[7] += cy * yy;   // y: [k][l]
    }
}

// face-point table indices of face f, point k
__device__ __forceinline__ void face_pt(int f, int k, int nq, int& kx, int& ky) {
  kx = f == 0 ? k : (f == 1 ? nq + 1 : (f == 2 ? k : nq));
  ky = f == 0 ? nq : (f == 1 ? k : (f == 2 ? nq + 1 : k));
}

// Eddington tensor (xx, xy, yy) of element e at a point where the DG basis values are
// B[j] (from the element's nodal phi and P)
template <int N>
__device__ __forceinline__ void eddington_at(const double* __restrict__ phi, const double* __restrict__ P,
                                             long long En, long long e, const double B[N], double Eo[3]) {
  double f = 0, a = 0, b = 0, c = 0;
  for (int j = 0; j < N; ++j) {
    const size_t o = (size_t)e * N + j;
    f += B[j] * phi[o];
    a += B[j] * P[o];
    b += B[j] * P[En + o];
    c += B[j] * P[2 * En + o];
  }
  Eo[0] = a / f;
  Eo[1] = b / f;
  Eo[2] = c / f;
}

// DG basis values at table point (kx, ky)
template <int P>
__device__ __forceinline__ void dg_at(const HrtTab& t, int kx, int ky, double B[(P + 1) * (P + 1)]) {
  for (int j = 0; j < (P + 1) * (P + 1); ++j) B[j] = t.dg[j % (P + 1)][kx] * t.dg[j / (P + 1)][ky];
}

struct HrtIn {
  const double* ctrl;   // [E][(m+1)^2][2]
  const double* Mm;     // [E][n][n] mass matrices
  const double* nds;    // [E][4][nq][2]
  const double* sigma_t;
  const double* sigma_s;
  const double* phi;    // [E][n] transport scalar flux (nodal)
  const double* P;      // [3][E][n] second moment (nodal)
  const double* Eb;     // [nbf][nq]
  const double* Jin;    // [nbf][nq]
  const double* Q0;     // [E][n] nodal
  const double* Q1;     // [2][E][n] nodal or null
};

struct HrtOut {
  double* Li;   // [E][MM][MM] inverse of the local system (row-major)
  double* C2;   // [E][NJ][NL4]
  double* g;    // [E][NJ]
  double* f;    // [E][N]
  double* He;   // [E][NL4][NL4]
  double* re;   // [E][NL4]
};

template <int P>
struct HrtSmem {
  using S = HrtShape<P>;
  double L[S::MM * S::LD];
  double vq[S::NQ2][S::NJ][2];       // physical v at the volume points
  double sg[S::NJ][S::NQ2];          // -w J (grad v : E) at the volume points
  double wJ[S::NQ2];                 // w J at the volume points
  double C1[S::NL4][S::NJ];
  double C2[S::NJ][S::NL4];
  double gv[S::NJ], fv[S::N];
  double T1[S::NJ][S::NL4];          // W C2
  double u[S::NJ];                   // W g + X f
  double colk[S::MM];
  double ctrl[(kMaxM + 1) * (kMaxM + 1) * 2];
  int perm[S::MM];
  int piv;
};

template <int P>
__global__ void __launch_bounds__(256)
hrt_local_kernel(long long E, int nx, int ny, HrtTab t, HrtIn in, HrtOut out, unsigned int* status) {
  using S = HrtShape<P>;
  constexpr int N = S::N, NQ = S::NQ, NQ2 = S::NQ2, NJ = S::NJ, MM = S::MM, LD = S::LD, NL = S::NL, NL4 = S::NL4;
  extern __shared__ __align__(16) unsigned char hrt_smem[];
  HrtSmem<P>& sm = *reinterpret_cast<HrtSmem<P>*>(hrt_smem);
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long En = E * N;
  const long long nbf = 2LL * nx + 2LL * ny;
  const int qc = (t.m + 1) * (t.m + 1);
  for (long long e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    for (int i = tid; i < 2 * qc; i += nth) sm.ctrl[i] = in.ctrl[(size_t)e * 2 * qc + i];
    const double st = in.sigma_t[e], sa = in.sigma_t[e] - in.sigma_s[e];
    __syncthreads();
    // volume points: physical v and -w J (grad v : E) for every basis function
    for (int idx = tid; idx < NQ2 * NJ; idx += nth) {
      const int q = idx / NJ, a = idx % NJ, k1 = q % NQ, k2 = q / NQ;
      double F[4], H[8];
      map_geom(sm.ctrl, t, k1, k2, F, H);
      const double J = F[0] * F[3] - F[1] * F[2];
      const double adj[4] = {F[3], -F[1], -F[2], F[0]};
      double dJ[2];
      for (int l = 0; l < 2; ++l)   // Jacobi: dJ = tr(adj F dF)
        dJ[l] = adj[0] * H[0 * 4 + 0 * 2 + l] + adj[1] * H[1 * 4 + 0 * 2 + l] + adj[2] * H[0 * 4 + 1 * 2 + l] +
                adj[3] * H[1 * 4 + 1 * 2 + l];
      double vh[2], dx[2], dy[2];
      rt_ref<P>(t, a, k1, k2, vh, dx, dy);
      double v[2], dv[2][2];   // dv[i][l] = d v_i / d xi_l
      for (int i = 0; i < 2; ++i) v[i] = (F[2 * i] * vh[0] + F[2 * i + 1] * vh[1]) / J;
      for (int l = 0; l < 2; ++l) {
        const double* dvh = l == 0 ? dx : dy;
        for (int i = 0; i < 2; ++i) {
          const double dFv = H[i * 4 + 0 * 2 + l] * vh[0] + H[i * 4 + 1 * 2 + l] * vh[1];
          const double Fdv = F[2 * i] * dvh[0] + F[2 * i + 1] * dvh[1];
          dv[i][l] = (dFv + Fdv) / J - dJ[l] / J * v[i];
        }
      }
      double B[N], Eq[3];
      dg_at<P>(t, k1, k2, B);
      eddington_at<N>(in.phi, in.P, En, e, B, Eq);
      // grad v = dv F^{-1}, F^{-1} = adj / J ; grad v : E
      double gE = 0.0;
      for (int i = 0; i < 2; ++i)
        for (int mcol = 0; mcol < 2; ++mcol) {
          const double gim = (dv[i][0] * adj[0 * 2 + mcol] + dv[i][1] * adj[1 * 2 + mcol]) / J;
          const double Eim = (i == mcol) ? (i == 0 ? Eq[0] : Eq[2]) : Eq[1];
          gE += gim * Eim;
        }
      const double w = t.w[k1] * t.w[k2];
      sm.vq[q][a][0] = v[0];
      sm.vq[q][a][1] = v[1];
      sm.sg[a][q] = -w * J * gE;
      if (a == 0) sm.wJ[q] = w * J;
    }
    for (int idx = tid; idx < NL4 * NJ; idx += nth) {
      (&sm.C1[0][0])[idx] = 0.0;
      (&sm.C2[0][0])[idx] = 0.0;
    }
    __syncthreads();
    // A (volume), G, D, Ma, f, g (volume)
    for (int idx = tid; idx < MM * MM; idx += nth) {
      const int r = idx / MM, c = idx % MM;
      double val = 0.0;
      if (r < NJ && c < NJ) {
        for (int q = 0; q < NQ2; ++q)
          val += sm.wJ[q] * (sm.vq[q][r][0] * sm.vq[q][c][0] + sm.vq[q][r][1] * sm.vq[q][c][1]);
        val *= st;
      } else if (r < NJ) {
        const int cc = c - NJ;
        for (int q = 0; q < NQ2; ++q)
          val += sm.sg[r][q] * t.dg[cc % (P + 1)][q % NQ] * t.dg[cc / (P + 1)][q / NQ];
      } else if (c < NJ) {
        const int rr = r - NJ;
        for (int q = 0; q < NQ2; ++q) {
          const int k1 = q % NQ, k2 = q / NQ;
          double vh[2], dx[2], dy[2];
          rt_ref<P>(t, c, k1, k2, vh, dx, dy);
          val += t.w[k1] * t.w[k2] * t.dg[rr % (P + 1)][k1] * t.dg[rr / (P + 1)][k2] * (dx[0] + dy[1]);
        }
      } else {
        val = sa * in.Mm[((size_t)e * N + (r - NJ)) * N + (c - NJ)];
      }
      sm.L[r * LD + c] = val;
    }
    for (int c = tid; c < N; c += nth) {
      double s = 0.0;
      for (int j = 0; j < N; ++j) s += in.Mm[((size_t)e * N + c) * N + j] * in.Q0[(size_t)e * N + j];
      sm.fv[c] = s;
    }
    for (int a = tid; a < NJ; a += nth) {
      double s = 0.0;
      if (in.Q1) {
        for (int q = 0; q < NQ2; ++q) {
          double B[N];
          dg_at<P>(t, q % NQ, q / NQ, B);
          double q1x = 0.0, q1y = 0.0;
          for (int j = 0; j < N; ++j) {
            q1x += B[j] * in.Q1[(size_t)e * N + j];
            q1y += B[j] * in.Q1[En + (size_t)e * N + j];
          }
          s += sm.wJ[q] * (sm.vq[q][a][0] * q1x + sm.vq[q][a][1] * q1y);
        }
      }
      sm.gv[a] = s;
    }
    __syncthreads();
    // faces: multiplier couplings on interior faces, Miften-Larsen terms on boundary faces
    const int ie = (int)(e % nx), je = (int)(e / nx);
    for (int f = 0; f < 4; ++f) {
      const int nb = nb_elem(nx, ny, (int)e, f);
      if (nb >= 0) {
        const int fo = (f + 2) & 3;
        for (int idx = tid; idx < NJ * NL; idx += nth) {
          const int a = idx / NL, tt = idx % NL;
          double c2 = 0.0, c1 = 0.0;
          for (int k = 0; k < NQ; ++k) {
            int kx, ky;
            face_pt(f, k, NQ, kx, ky);
            double F[4], H[8];
            map_geom(sm.ctrl, t, kx, ky, F, H);
            const double J = F[0] * F[3] - F[1] * F[2];
            double vh[2], dx[2], dy[2];
            rt_ref<P>(t, a, kx, ky, vh, dx, dy);
            const double v0 = (F[0] * vh[0] + F[1] * vh[1]) / J, v1 = (F[2] * vh[0] + F[3] * vh[1]) / J;
            // the two sides' Eddington tensors at this face point (their own traces)
            double Bo[N], Bn[N], Eo[3], Enb[3];
            dg_at<P>(t, kx, ky, Bo);
            int nkx, nky;
            face_pt(fo, k, NQ, nkx, nky);
            dg_at<P>(t, nkx, nky, Bn);
            eddington_at<N>(in.phi, in.P, En, e, Bo, Eo);
            eddington_at<N>(in.phi, in.P, En, nb, Bn, Enb);
            const double a00 = 0.5 * (Eo[0] + Enb[0]), a01 = 0.5 * (Eo[1] + Enb[1]), a11 = 0.5 * (Eo[2] + Enb[2]);
            const double* nd = in.nds + (((size_t)e * 4 + f) * NQ + k) * 2;
            const double En0 = a00 * nd[0] + a01 * nd[1], En1 = a01 * nd[0] + a11 * nd[1];
            const double lam = t.op[tt][k];
            c2 += t.w[k] * lam * (v0 * En0 + v1 * En1);
            const double nref0 = f == 1 ? 1.0 : (f == 3 ? -1.0 : 0.0), nref1 = f == 2 ? 1.0 : (f == 0 ? -1.0 : 0.0);
            c1 += t.w[k] * lam * (vh[0] * nref0 + vh[1] * nref1);
          }
          sm.C2[a][f * NL + tt] = c2;
          sm.C1[f * NL + tt][a] = c1;
        }
      } else {
        const long long bf = bface(nx, ny, (int)e, f);
        for (int idx = tid; idx < NJ * NJ + NJ; idx += nth) {
          const int a = idx < NJ * NJ ? idx / NJ : idx - NJ * NJ;
          const int b = idx < NJ * NJ ? idx % NJ : -1;
          double s = 0.0;
          for (int k = 0; k < NQ; ++k) {
            int kx, ky;
            face_pt(f, k, NQ, kx, ky);
            double F[4], H[8];
            map_geom(sm.ctrl, t, kx, ky, F, H);
            const double J = F[0] * F[3] - F[1] * F[2];
            const double* nd = in.nds + (((size_t)e * 4 + f) * NQ + k) * 2;
            const double ln = sqrt(nd[0] * nd[0] + nd[1] * nd[1]);
            const double un0 = nd[0] / ln, un1 = nd[1] / ln;
            double Bo[N], Eo[3];
            dg_at<P>(t, kx, ky, Bo);
            eddington_at<N>(in.phi, in.P, En, e, Bo, Eo);
            const double En0 = Eo[0] * un0 + Eo[1] * un1, En1 = Eo[1] * un0 + Eo[2] * un1;
            double vh[2], dx[2], dy[2];
            rt_ref<P>(t, a, kx, ky, vh, dx, dy);
            const double va0 = (F[0] * vh[0] + F[1] * vh[1]) / J, va1 = (F[2] * vh[0] + F[3] * vh[1]) / J;
            const double vEn = va0 * En0 + va1 * En1;
            const double eb = in.Eb[bf * NQ + k];
            if (b >= 0) {
              rt_ref<P>(t, b, kx, ky, vh, dx, dy);
              const double vb0 = (F[0] * vh[0] + F[1] * vh[1]) / J, vb1 = (F[2] * vh[0] + F[3] * vh[1]) / J;
              s += t.w[k] * ln / eb * vEn * (vb0 * un0 + vb1 * un1);
            } else {
              s += 2.0 * t.w[k] * ln * in.Jin[bf * NQ + k] / eb * vEn;
            }
          }
          if (b >= 0) sm.L[a * LD + b] += s;
          else sm.gv[a] += s;
        }
      }
      __syncthreads();
    }
    (void)ie; (void)je;
    // in-place Gauss-Jordan inversion of L with partial pivoting
    for (int k = 0; k < MM; ++k) {
      if (tid < 32) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < MM; i += 32) {
          const double v = fabs(sm.L[i * LD + k]);
          if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, off);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
          sm.piv = bi;
          sm.perm[k] = bi;
          if (!(best > 1e-300)) atomicOr(status, kDevSingular);
        }
      }
      __syncthreads();
      const int pr = sm.piv;
      if (pr != k)
        for (int j = tid; j < MM; j += nth) {
          const double tmp = sm.L[k * LD + j];
          sm.L[k * LD + j] = sm.L[pr * LD + j];
          sm.L[pr * LD + j] = tmp;
        }
      __syncthreads();
      const double inv = 1.0 / sm.L[k * LD + k];
      for (int i = tid; i < MM; i += nth) sm.colk[i] = sm.L[i * LD + k];
      __syncthreads();
      for (int j = tid; j < MM; j += nth)
        if (j != k) sm.L[k * LD + j] *= inv;
      __syncthreads();
      for (int idx = tid; idx < MM * MM; idx += nth) {
        const int i = idx / MM, j = idx % MM;
        if (i == k) continue;
        if (j == k) sm.L[i * LD + k] = -sm.colk[i] * inv;
        else sm.L[i * LD + j] -= sm.colk[i] * sm.L[k * LD + j];
      }
      if (tid == 0) sm.L[k * LD + k] = inv;
      __syncthreads();
    }
    for (int k = MM - 1; k >= 0; --k) {   // undo the row interchanges as column interchanges
      const int pr = sm.perm[k];
      if (pr != k)
        for (int i = tid; i < MM; i += nth) {
          const double tmp = sm.L[i * LD + k];
          sm.L[i * LD + k] = sm.L[i * LD + pr];
          sm.L[i * LD + pr] = tmp;
        }
      __syncthreads();
    }
    // W C2 and W g + X f, then H_e = C1 (W C2) and r_e = C1 (W g + X f)
    for (int idx = tid; idx < NJ * NL4 + NJ; idx += nth) {
      if (idx < NJ * NL4) {
        const int a = idx / NL4, c = idx % NL4;
        double s = 0.0;
        for (int b = 0; b < NJ; ++b) s += sm.L[a * LD + b] * sm.C2[b][c];
        sm.T1[a][c] = s;
      } else {
        const int a = idx - NJ * NL4;
        double s = 0.0;
        for (int b = 0; b < NJ; ++b) s += sm.L[a * LD + b] * sm.gv[b];
        for (int c = 0; c < N; ++c) s += sm.L[a * LD + NJ + c] * sm.fv[c];
        sm.u[a] = s;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < NL4 * NL4 + NL4; idx += nth) {
      if (idx < NL4 * NL4) {
        const int r = idx / NL4, c = idx % NL4;
        double s = 0.0;
        for (int a = 0; a < NJ; ++a) s += sm.C1[r][a] * sm.T1[a][c];
        out.He[(size_t)e * NL4 * NL4 + idx] = s;
      } else {
        const int r = idx - NL4 * NL4;
        double s = 0.0;
        for (int a = 0; a < NJ; ++a) s += sm.C1[r][a] * sm.u[a];
        out.re[(size_t)e * NL4 + r] = s;
      }
    }
    for (int idx = tid; idx < MM * MM; idx += nth)
      out.Li[(size_t)e * MM * MM + idx] = sm.L[(idx / MM) * LD + idx % MM];
    for (int idx = tid; idx < NJ * NL4; idx += nth) out.C2[(size_t)e * NJ * NL4 + idx] = (&sm.C2[0][0])[idx];
    for (int a = tid; a < NJ; a += nth) out.g[(size_t)e * NJ + a] = sm.gv[a];
    for (int c = tid; c < N; c += nth) out.f[(size_t)e * N + c] = sm.fv[c];
  }
}

// global multiplier index of face f of element e, or -1 on the boundary
__device__ __forceinline__ long long face_index(int nx, int ny, int e, int f) {
  const int i = e % nx, j = e / nx;
  const long long nv = (long long)(nx - 1) * ny;
  if (f == 1) return i < nx - 1 ? (long long)j * (nx - 1) + i : -1;
  if (f == 3) return i > 0 ? (long long)j * (nx - 1) + i - 1 : -1;
  if (f == 2) return j < ny - 1 ? nv + (long long)j * nx + i : -1;
  return j > 0 ? nv + (long long)(j - 1) * nx + i : -1;
}

// z_e = H_e x_e (x gathered from the element's interior faces; boundary faces give 0)
template <int P>
__global__ void hrt_local_apply_kernel(long long E, int nx, int ny, const double* __restrict__ He,
                                       const double* __restrict__ x, double* __restrict__ z) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * NL4) return;
  const long long e = t / NL4;
  const int r = (int)(t % NL4);
  const double* h = He + (size_t)e * NL4 * NL4 + (size_t)r * NL4;
  double s = 0.0;
  for (int f = 0; f < 4; ++f) {
    const long long fi = face_index(nx, ny, (int)e, f);
    if (fi < 0) continue;
    for (int tt = 0; tt < NL; ++tt) s += h[f * NL + tt] * x[fi * NL + tt];
  }
  z[t] = s;
}

// y[face dof] = sum of the two sides' z rows (or their H_e diagonals for the preconditioner)
template <int P>
__global__ void hrt_gather_kernel(int nx, int ny, long long nfaces, const double* __restrict__ z,
                                  const double* __restrict__ He, double* __restrict__ y) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nfaces * NL) return;
  const long long fid = t / NL;
  const int tt = (int)(t % NL);
  const long long nv = (long long)(nx - 1) * ny;
  long long e1, e2;
  int f1, f2;
  if (fid < nv) {
    const long long j = fid / (nx - 1), i = fid % (nx - 1);
    e1 = j * nx + i; f1 = 1; e2 = e1 + 1; f2 = 3;
  } else {
    const long long h = fid - nv, j = h / nx, i = h % nx;
    e1 = j * nx + i; f1 = 2; e2 = e1 + nx; f2 = 0;
  }
  const int r1 = f1 * NL + tt, r2 = f2 * NL + tt;
  if (z) y[t] = z[e1 * NL4 + r1] + z[e2 * NL4 + r2];
  else y[t] = He[(size_t)e1 * NL4 * NL4 + (size_t)r1 * NL4 + r1] + He[(size_t)e2 * NL4 * NL4 + (size_t)r2 * NL4 + r2];
}

// [J; phi] = Li [g - C2 lambda_e; f]
template <int P>
__global__ void hrt_recover_kernel(long long E, int nx, int ny, const double* __restrict__ Li,
                                   const double* __restrict__ C2, const double* __restrict__ g,
                                   const double* __restrict__ f, const double* __restrict__ lam,
                                   double* __restrict__ Jout, double* __restrict__ phi_out) {
  using S = HrtShape<P>;
  constexpr int N = S::N, NJ = S::NJ, MM = S::MM, NL = S::NL, NL4 = S::NL4;
  __shared__ double rhs[MM];
  __shared__ double le[NL4];
  for (long long e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    for (int r = threadIdx.x; r < NL4; r += blockDim.x) {
      const long long fi = face_index(nx, ny, (int)e, r / NL);
      le[r] = fi < 0 ? 0.0 : lam[fi * NL + r % NL];
    }
    __syncthreads();
    for (int a = threadIdx.x; a < MM; a += blockDim.x) {
      if (a < NJ) {
        double s = g[(size_t)e * NJ + a];
        for (int c = 0; c < NL4; ++c) s -= C2[(size_t)e * NJ * NL4 + (size_t)a * NL4 + c] * le[c];
        rhs[a] = s;
      } else {
        rhs[a] = f[(size_t)e * N + a - NJ];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < MM; i += blockDim.x) {
      const double* row = Li + (size_t)e * MM * MM + (size_t)i * MM;
      double s = 0.0;
      for (int j = 0; j < MM; ++j) s += row[j] * rhs[j];
      if (i < NJ) Jout[(size_t)e * NJ + i] = s;
      else phi_out[(size_t)e * N + i - NJ] = s;
    }
  }
}

// ---- vector kernels of the Krylov solve (deterministic two-stage dot products)
constexpr int kDotBlocks = 256, kDotThreads = 256;

__global__ void dot_partial_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                                   const double* __restrict__ c, const double* __restrict__ d,
                                   double* __restrict__ part) {
  // part[blockIdx] = (a.b, c.d) over this block's grid-stride share
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double x = 0.0, y = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x += a[i] * b[i];
    if (c) y += c[i] * d[i];
  }
  s0[threadIdx.x] = x;
  s1[threadIdx.x] = y;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}

__global__ void dot_final_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  s0[threadIdx.x] = x;
  s1[threadIdx.x] = y;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

// y = a x + b y (+ c z) elementwise; mode 1: y = x / d (Jacobi)
__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y,
                             double c, const double* __restrict__ z) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = a * x[i] + b * y[i] + (z ? c * z[i] : 0.0);
}

__global__ void jacobi_kernel(long long n, const double* __restrict__ x, const double* __restrict__ d,
                              double* __restrict__ y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] / d[i];
}

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

struct HrtWork {
  double *Li, *C2, *g, *f, *He, *re, *z;
  double *r, *rh, *pv, *vv, *sv, *tv, *ph, *sh, *diag, *part, *dots;
};

template <int P>
static vef_status hrt_run(Mesh& M, const HrtIn& in, double tol, int max_iter, double* phi, double* J,
                          double* lambda, vef_hrt_info* info, cudaStream_t s) {
  using S = HrtShape<P>;
  const long long E = M.E;
  const long long nfaces = (long long)(M.nx - 1) * M.ny + (long long)M.nx * (M.ny - 1);
  const long long nl = nfaces * S::NL;
  const size_t per_e = (size_t)S::MM * S::MM + (size_t)S::NJ * S::NL4 + S::NJ + S::N + (size_t)S::NL4 * S::NL4 +
                       S::NL4 + S::NL4;
  const size_t vec = (size_t)std::max(1LL, nl);
  const size_t total = per_e * E + 11 * vec + 2 * kDotBlocks + 2;
  vef_status st = ensure_buffer((void**)&M.work, &M.work_cap, total * sizeof(double));
  if (st != VEF_OK) return st;
  double* base = M.work;
  HrtWork w{};
  w.Li = base; base += (size_t)S::MM * S::MM * E;
  w.C2 = base; base += (size_t)S::NJ * S::NL4 * E;
  w.g = base; base += (size_t)S::NJ * E;
  w.f = base; base += (size_t)S::N * E;
  w.He = base; base += (size_t)S::NL4 * S::NL4 * E;
  w.re = base; base += (size_t)S::NL4 * E;
  w.z = base; base += (size_t)S::NL4 * E;
  double* lam = lambda;
  w.r = base; base += vec;
  if (!lam) { lam = base; } base += vec;
  w.rh = base; base += vec;
  w.pv = base; base += vec;
  w.vv = base; base += vec;
  w.sv = base; base += vec;
  w.tv = base; base += vec;
  w.ph = base; base += vec;
  w.sh = base; base += vec;
  w.diag = base; base += vec;
  w.part = base; base += 2 * kDotBlocks;
  w.dots = base;
  double* diag = w.diag;
  const HrtTab tab = make_hrt_tab(P, M.m);
  HrtOut out{w.Li, w.C2, w.g, w.f, w.He, w.re};
  const size_t smem = sizeof(HrtSmem<P>);
  VEF_CUDA_TRY(cudaFuncSetAttribute(hrt_local_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  VEF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  {
    KTimer kt(&M, VEF_K_HRT, s);
    hrt_local_kernel<P><<<(unsigned)std::min<long long>(E, (long long)sms * 8), 256, smem, s>>>(
        E, M.nx, M.ny, tab, in, out, M.dev_status);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  auto matvec = [&](const double* x, double* y) -> vef_status {
    hrt_local_apply_kernel<P><<<nblk(E * S::NL4, 256), 256, 0, s>>>(E, M.nx, M.ny, w.He, x, w.z);
    hrt_gather_kernel<P><<<nblk(nl, 256), 256, 0, s>>>(M.nx, M.ny, nfaces, w.z, w.He, y);
    VEF_CUDA_TRY(cudaGetLastError());
    return VEF_OK;
  };
  auto dot2 = [&](const double* a, const double* b, const double* c, const double* d, double h[2]) -> vef_status {
    dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(nl, a, b, c, d, w.part);
    dot_final_kernel<<<1, kDotThreads, 0, s>>>(kDotBlocks, w.part, w.dots);
    VEF_CUDA_TRY(cudaMemcpyAsync(h, w.dots, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    VEF_CUDA_TRY(cudaStreamSynchronize(s));
    return VEF_OK;
  };
  const unsigned vb = nblk(nl, 256);
  int it = 0;
  double rel = 0.0;
  if (nl > 0) {
    // the reduced right-hand side r = sum_e r_e, then BiCGStab with the diagonal of H
    hrt_gather_kernel<P><<<vb, 256, 0, s>>>(M.nx, M.ny, nfaces, w.re, nullptr, w.r);   // z = r_e layout
    hrt_gather_kernel<P><<<vb, 256, 0, s>>>(M.nx, M.ny, nfaces, nullptr, w.He, diag);
    VEF_CUDA_TRY(cudaMemsetAsync(lam, 0, nl * sizeof(double), s));
    VEF_CUDA_TRY(cudaMemcpyAsync(w.rh, w.r, nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
    VEF_CUDA_TRY(cudaMemsetAsync(w.pv, 0, nl * sizeof(double), s));
    VEF_CUDA_TRY(cudaMemsetAsync(w.vv, 0, nl * sizeof(double), s));
    double h[2];
    if ((st = dot2(w.r, w.r, nullptr, nullptr, h)) != VEF_OK) return st;
    const double bnorm = std::sqrt(h[0]);
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    rel = bnorm > 0.0 ? 1.0 : 0.0;
    while (bnorm > 0.0 && it < max_iter && rel > tol) {
      if ((st = dot2(w.rh, w.r, nullptr, nullptr, h)) != VEF_OK) return st;
      const double rho_new = h[0];
      if (rho_new == 0.0) break;
      const double beta = (rho_new / rho) * (alpha / omega);
      rho = rho_new;
      // p = r + beta (p - omega v)
      axpby_kernel<<<vb, 256, 0, s>>>(nl, 1.0, w.r, beta, w.pv, -beta * omega, w.vv);
      jacobi_kernel<<<vb, 256, 0, s>>>(nl, w.pv, diag, w.ph);
      if ((st = matvec(w.ph, w.vv)) != VEF_OK) return st;
      if ((st = dot2(w.rh, w.vv, nullptr, nullptr, h)) != VEF_OK) return st;
      alpha = rho / h[0];
      // s = r - alpha v
      VEF_CUDA_TRY(cudaMemcpyAsync(w.sv, w.r, nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
      axpby_kernel<<<vb, 256, 0, s>>>(nl, -alpha, w.vv, 1.0, w.sv, 0.0, nullptr);
      jacobi_kernel<<<vb, 256, 0, s>>>(nl, w.sv, diag, w.sh);
      if ((st = matvec(w.sh, w.tv)) != VEF_OK) return st;
      if ((st = dot2(w.tv, w.sv, w.tv, w.tv, h)) != VEF_OK) return st;
      omega = h[1] > 0.0 ? h[0] / h[1] : 0.0;
      // lambda += alpha p_hat + omega s_hat ; r = s - omega t
      axpby_kernel<<<vb, 256, 0, s>>>(nl, alpha, w.ph, 1.0, lam, omega, w.sh);
      VEF_CUDA_TRY(cudaMemcpyAsync(w.r, w.sv, nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
      axpby_kernel<<<vb, 256, 0, s>>>(nl, -omega, w.tv, 1.0, w.r, 0.0, nullptr);
      ++it;
      if ((st = dot2(w.r, w.r, nullptr, nullptr, h)) != VEF_OK) return st;
      rel = std::sqrt(h[0]) / bnorm;
      if (omega == 0.0) break;
    }
  }
  {
    KTimer kt(&M, VEF_K_HRT, s);
    hrt_recover_kernel<P><<<(unsigned)std::min<long long>(E, (long long)sms * 8), 128, 0, s>>>(
        E, M.nx, M.ny, w.Li, w.C2, w.g, w.f, lam, J, phi);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  if (info) {
    info->iterations = it;
    info->rel_residual = rel;
    info->multipliers = nl;
  }
  if (nl > 0 && rel > tol) {
    set_last_error("HRT multiplier solve did not reach its tolerance");
    return VEF_ERR_NOT_CONVERGED;
  }
  return VEF_OK;
}

}  // namespace
}  // namespace vef

using namespace vef;

extern "C" vef_status vef_hrt_solve(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                    const double* phi_tr, const double* P_tr, const double* Eb,
                                    const double* Jin, const double* Q0, const double* Q1, double tol,
                                    int max_iter, double* phi, double* J, double* lambda,
                                    vef_hrt_info* info, void* stream) {
  if (!mesh || !sigma_t || !sigma_s || !phi_tr || !P_tr || !Eb || !Jin || !Q0 || !phi || !J) {
    set_last_error("mesh, sigma_t, sigma_s, phi_tr, P_tr, Eb, Jin, Q0, phi and J are required");
    return VEF_ERR_INVALID_ARG;
  }
  if (!(tol > 0.0) || max_iter < 1) {
    set_last_error("tol must be positive and max_iter >= 1");
    return VEF_ERR_INVALID_ARG;
  }
  Mesh& M = mesh->impl;
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != M.device) { set_last_error("mesh belongs to another device"); return VEF_ERR_INVALID_ARG; }
  HrtIn in{M.ctrl_dev, M.Mmat, M.nds, sigma_t, sigma_s, phi_tr, P_tr, Eb, Jin, Q0, Q1};
  cudaStream_t s = (cudaStream_t)stream;
  vef_status st;
  switch (M.p) {
    case 1: st = hrt_run<1>(M, in, tol, max_iter, phi, J, lambda, info, s); break;
    case 2: st = hrt_run<2>(M, in, tol, max_iter, phi, J, lambda, info, s); break;
    case 3: st = hrt_run<3>(M, in, tol, max_iter, phi, J, lambda, info, s); break;
    default: st = hrt_run<4>(M, in, tol, max_iter, phi, J, lambda, info, s); break;
  }
  if (st != VEF_OK) return st;
  return collect_status(M, s, nullptr);
}
