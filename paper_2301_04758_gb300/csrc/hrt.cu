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
// CTA in shared memory (the map's derivatives and the Eddington tensor evaluated once per
// Gauss point; D and C1 are the same on every element and come from host tables);
// hrt_invert_kernel, at a higher occupancy, inverts [[A, G], [D, Ma]] by Gauss-Jordan
// elimination with partial pivoting (the block is indefinite in general), and forms the
// element's share of the reduced system,
//     H_e = C1 W C2,   r_e = C1 (W g + X f),   [[W, X], [Y, Z]] = [[A, G], [D, Ma]]^{-1}.
// The multiplier system H lambda = r (H = sum_e H_e over the interior faces, not symmetric
// for a general Eddington tensor) is solved by BiCGStab with a two-level additive Schwarz
// preconditioner (element patches plus a coarse bilinear space), the matrix applied face by
// face from the two sides' rows of H_e (no atomics) and the Krylov scalars kept on the
// device.  hrt_recover_kernel then forms J and phi element by element.
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
__host__ __device__ __forceinline__ void rt_ref(const HrtTab& t, int a, int kx, int ky, double v[2], double dxi[2],
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
__host__ __device__ __forceinline__ void face_pt(int f, int k, int nq, int& kx, int& ky) {
  kx = f == 0 ? k : (f == 1 ? nq + 1 : (f == 2 ? k : nq));
  ky = f == 0 ? nq : (f == 1 ? k : (f == 2 ? nq + 1 : k));
}

// Eddington tensor (xx, xy, yy) of element e at table point (kx, ky), from the element's
// nodal phi and P (the DG basis evaluated term by term)
template <int P>
__device__ __forceinline__ void eddington_pt(const HrtTab& t, const double* __restrict__ phi,
                                             const double* __restrict__ Pm, long long En, long long e, int kx,
                                             int ky, double Eo[3]) {
  constexpr int Q = P + 1, N = Q * Q;
  double f = 0, a = 0, b = 0, c = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const double Bj = t.dg[j % Q][kx] * t.dg[j / Q][ky];
    const size_t o = (size_t)e * N + j;
    f += Bj * phi[o];
    a += Bj * Pm[o];
    b += Bj * Pm[En + o];
    c += Bj * Pm[2 * En + o];
  }
  const double rf = 1.0 / f;
  Eo[0] = a * rf;
  Eo[1] = b * rf;
  Eo[2] = c * rf;
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

// Geometry-independent blocks of the local system, formed once on the host from the same
// 1D tables: D_ref [n][NJ] = int u div_hat v_hat (the Piola transform makes int u div J dx
// the reference integral) and C1_ref [4 (p+1)][NJ] = int_f mu (v_hat . n_hat) (the reference
// normal flux against the multiplier basis; rows of boundary faces are dropped per element).
struct HrtRef {
  const double* D;    // [n][NJ]
  const double* C1;   // [4 (p+1)][NJ]
};

template <int P>
static void make_hrt_ref(const HrtTab& t, std::vector<double>& out) {
  using S = HrtShape<P>;
  constexpr int Q = P + 1, N = S::N, NQ = S::NQ, NJ = S::NJ, NL = S::NL;
  out.assign((size_t)N * NJ + (size_t)4 * NL * NJ, 0.0);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < NJ; ++c) {
      double s = 0.0;
      for (int k2 = 0; k2 < NQ; ++k2)
        for (int k1 = 0; k1 < NQ; ++k1) {
          double vh[2], dx[2], dy[2];
          rt_ref<P>(t, c, k1, k2, vh, dx, dy);
          s += t.w[k1] * t.w[k2] * t.dg[r % Q][k1] * t.dg[r / Q][k2] * (dx[0] + dy[1]);
        }
      out[(size_t)r * NJ + c] = s;
    }
  double* C1 = out.data() + (size_t)N * NJ;
  for (int f = 0; f < 4; ++f) {
    const double n0 = f == 1 ? 1.0 : (f == 3 ? -1.0 : 0.0), n1 = f == 2 ? 1.0 : (f == 0 ? -1.0 : 0.0);
    for (int tt = 0; tt < NL; ++tt)
      for (int a = 0; a < NJ; ++a) {
        double s = 0.0;
        for (int k = 0; k < NQ; ++k) {
          int kx, ky;
          face_pt(f, k, NQ, kx, ky);
          double vh[2], dx[2], dy[2];
          rt_ref<P>(t, a, kx, ky, vh, dx, dy);
          s += t.w[k] * t.op[tt][k] * (vh[0] * n0 + vh[1] * n1);
        }
        C1[(size_t)(f * NL + tt) * NJ + a] = s;
      }
  }
}

template <int P>
struct HrtSmem {
  using S = HrtShape<P>;
  static constexpr int NF = 4 * S::NQ;   // face points
  double L[S::MM * S::LD];
  double vq[S::NQ2][S::NJ][2];       // physical v at the volume points
  double sg[S::NJ][S::NQ2];          // -w J (grad v : E) at the volume points
  double wJ[S::NQ2];                 // w J at the volume points
  double C2[S::NJ][S::NL4];
  double gv[S::NJ], fv[S::N];
  double ctrl[(kMaxM + 1) * (kMaxM + 1) * 2];
  // per volume point: F (4, row-major), J, dJ/dxi (2), second derivatives (8), E (3), Q1 (2),
  // 1 / J
  double pv[S::NQ2][21];
  // per face point: interior faces w (F^T {E} n ds) / J (2); boundary faces (F^T E n^) / J (2),
  // (F^T n^) / J (2), w |n ds| / E_b and 2 w |n ds| J_in / E_b
  double pf[NF][6];
  double pa[S::NQ][S::NJ], pb[S::NQ][S::NJ];   // boundary face: v_hat . the two vectors above
};

template <int P>
__global__ void __launch_bounds__(256, 2)
hrt_local_kernel(long long E, int nx, int ny, HrtTab tab, HrtRef ref, HrtIn in, HrtOut out, unsigned int* status) {
  using S = HrtShape<P>;
  constexpr int N = S::N, NQ = S::NQ, NQ2 = S::NQ2, NJ = S::NJ, MM = S::MM, LD = S::LD, NL = S::NL, NL4 = S::NL4;
  constexpr int NF = HrtSmem<P>::NF;
  extern __shared__ __align__(16) unsigned char hrt_smem[];
  HrtSmem<P>& sm = *reinterpret_cast<HrtSmem<P>*>(hrt_smem);
  const int tid = threadIdx.x, nth = blockDim.x;
  // the 1D tables in shared memory: every loop below indexes them per thread, which the
  // constant bank of a kernel parameter would serve one distinct address at a time
  __shared__ HrtTab t;
  static_assert(sizeof(HrtTab) % sizeof(double) == 0, "HrtTab is copied in 8-byte words");
  for (int i = tid; i < (int)(sizeof(HrtTab) / sizeof(double)); i += nth)
    reinterpret_cast<double*>(&t)[i] = reinterpret_cast<const double*>(&tab)[i];
  __syncthreads();
  const long long En = E * N;
  const int qc = (t.m + 1) * (t.m + 1);
  for (long long e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    for (int i = tid; i < 2 * qc; i += nth) sm.ctrl[i] = in.ctrl[(size_t)e * 2 * qc + i];
    const double st = in.sigma_t[e], sa = in.sigma_t[e] - in.sigma_s[e];
    __syncthreads();
    // (1) once per point: the map's derivatives and the Eddington tensor (both sides of an
    // interior face, averaged), at the volume and face Gauss points
    for (int pt = tid; pt < NQ2 + NF; pt += nth) {
      const bool vol = pt < NQ2;
      const int f = vol ? -1 : (pt - NQ2) / NQ, k = vol ? 0 : (pt - NQ2) % NQ;
      int kx, ky;
      if (vol) { kx = pt % NQ; ky = pt / NQ; }
      else face_pt(f, k, NQ, kx, ky);
      double F[4], H[8];
      map_geom(sm.ctrl, t, kx, ky, F, H);
      const double J = F[0] * F[3] - F[1] * F[2];
      double Eo[3];
      eddington_pt<P>(t, in.phi, in.P, En, e, kx, ky, Eo);
      if (vol) {
        double* g = sm.pv[pt];
        const double adj[4] = {F[3], -F[1], -F[2], F[0]};
        for (int i = 0; i < 4; ++i) g[i] = F[i];
        g[4] = J;
        for (int l = 0; l < 2; ++l)   // Jacobi's formula: dJ = tr(adj F dF)
          g[5 + l] = adj[0] * H[0 * 4 + 0 * 2 + l] + adj[1] * H[1 * 4 + 0 * 2 + l] +
                     adj[2] * H[0 * 4 + 1 * 2 + l] + adj[3] * H[1 * 4 + 1 * 2 + l];
        for (int i = 0; i < 8; ++i) g[7 + i] = H[i];
        for (int i = 0; i < 3; ++i) g[15 + i] = Eo[i];
        double q1x = 0.0, q1y = 0.0;
        if (in.Q1)
          for (int j = 0; j < N; ++j) {
            const double Bj = t.dg[j % (P + 1)][kx] * t.dg[j / (P + 1)][ky];
            q1x += Bj * in.Q1[(size_t)e * N + j];
            q1y += Bj * in.Q1[En + (size_t)e * N + j];
          }
        g[18] = q1x;
        g[19] = q1y;
        g[20] = 1.0 / J;
      } else {
        double* o = sm.pf[pt - NQ2];
        const double* nd = in.nds + (((size_t)e * 4 + f) * NQ + k) * 2;
        const int nb = nb_elem(nx, ny, (int)e, f);
        if (nb >= 0) {
          int nkx, nky;
          face_pt((f + 2) & 3, k, NQ, nkx, nky);
          double Enb[3];
          eddington_pt<P>(t, in.phi, in.P, En, nb, nkx, nky, Enb);
          const double a00 = 0.5 * (Eo[0] + Enb[0]), a01 = 0.5 * (Eo[1] + Enb[1]), a11 = 0.5 * (Eo[2] + Enb[2]);
          const double En0 = a00 * nd[0] + a01 * nd[1], En1 = a01 * nd[0] + a11 * nd[1];
          // v_a . {E} n ds = v_hat_a . F^T ({E} n ds) / J
          o[0] = t.w[k] * (F[0] * En0 + F[2] * En1) / J;
          o[1] = t.w[k] * (F[1] * En0 + F[3] * En1) / J;
        } else {
          const long long bf = bface(nx, ny, (int)e, f);
          const double ln = sqrt(nd[0] * nd[0] + nd[1] * nd[1]);
          const double un0 = nd[0] / ln, un1 = nd[1] / ln;
          const double En0 = Eo[0] * un0 + Eo[1] * un1, En1 = Eo[1] * un0 + Eo[2] * un1;
          const double eb = in.Eb[bf * NQ + k];
          o[0] = (F[0] * En0 + F[2] * En1) / J;
          o[1] = (F[1] * En0 + F[3] * En1) / J;
          o[2] = (F[0] * un0 + F[2] * un1) / J;
          o[3] = (F[1] * un0 + F[3] * un1) / J;
          o[4] = t.w[k] * ln / eb;
          o[5] = 2.0 * t.w[k] * ln * in.Jin[bf * NQ + k] / eb;
        }
      }
    }
    __syncthreads();
    // (2) per (volume point, basis function): the physical v and -w J (grad v : E)
    for (int idx = tid; idx < NQ2 * NJ; idx += nth) {
      const int q = idx / NJ, a = idx % NJ, k1 = q % NQ, k2 = q / NQ;
      const double* g = sm.pv[q];
      const double F[4] = {g[0], g[1], g[2], g[3]};
      const double J = g[4], rJ = g[20];
      const double adj[4] = {F[3], -F[1], -F[2], F[0]};
      double vh[2], dx[2], dy[2];
      rt_ref<P>(t, a, k1, k2, vh, dx, dy);
      double v[2], dv[2][2];   // dv[i][l] = d v_i / d xi_l
      for (int i = 0; i < 2; ++i) v[i] = (F[2 * i] * vh[0] + F[2 * i + 1] * vh[1]) * rJ;
      for (int l = 0; l < 2; ++l) {
        const double* dvh = l == 0 ? dx : dy;
        for (int i = 0; i < 2; ++i) {
          const double dFv = g[7 + i * 4 + 0 * 2 + l] * vh[0] + g[7 + i * 4 + 1 * 2 + l] * vh[1];
          const double Fdv = F[2 * i] * dvh[0] + F[2 * i + 1] * dvh[1];
          dv[i][l] = (dFv + Fdv - g[5 + l] * v[i]) * rJ;
        }
      }
      // grad v = dv F^{-1}, F^{-1} = adj / J; grad v : E
      double gE = 0.0;
      for (int i = 0; i < 2; ++i)
        for (int mcol = 0; mcol < 2; ++mcol) {
          const double gim = (dv[i][0] * adj[0 * 2 + mcol] + dv[i][1] * adj[1 * 2 + mcol]) * rJ;
          const double Eim = (i == mcol) ? (i == 0 ? g[15] : g[17]) : g[16];
          gE += gim * Eim;
        }
      const double w = t.w[k1] * t.w[k2];
      sm.vq[q][a][0] = v[0];
      sm.vq[q][a][1] = v[1];
      sm.sg[a][q] = -w * J * gE;
      if (a == 0) sm.wJ[q] = w * J;
    }
    for (int idx = tid; idx < NL4 * NJ; idx += nth) (&sm.C2[0][0])[idx] = 0.0;
    __syncthreads();
    // (3) A (symmetric: one triangle computed), G, D (reference), sigma_a M, f, g
    for (int idx = tid; idx < MM * MM; idx += nth) {
      const int r = idx / MM, c = idx % MM;
      if (r < NJ && c < NJ) {
        if (c < r) continue;
        double val = 0.0;
        for (int q = 0; q < NQ2; ++q)
          val += sm.wJ[q] * (sm.vq[q][r][0] * sm.vq[q][c][0] + sm.vq[q][r][1] * sm.vq[q][c][1]);
        val *= st;
        sm.L[r * LD + c] = val;
        sm.L[c * LD + r] = val;
        continue;
      }
      double val;
      if (r < NJ) {
        const int cc = c - NJ;
        val = 0.0;
        for (int q = 0; q < NQ2; ++q)
          val += sm.sg[r][q] * t.dg[cc % (P + 1)][q % NQ] * t.dg[cc / (P + 1)][q / NQ];
      } else if (c < NJ) {
        val = ref.D[(r - NJ) * NJ + c];
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
      if (in.Q1)
        for (int q = 0; q < NQ2; ++q)
          s += sm.wJ[q] * (sm.vq[q][a][0] * sm.pv[q][18] + sm.vq[q][a][1] * sm.pv[q][19]);
      sm.gv[a] = s;
    }
    __syncthreads();
    // (4) faces: multiplier couplings on interior faces, Miften-Larsen terms on boundary faces
    for (int f = 0; f < 4; ++f) {
      const double* o0 = sm.pf[f * NQ];
      if (nb_elem(nx, ny, (int)e, f) >= 0) {
        for (int idx = tid; idx < NJ * NL; idx += nth) {
          const int a = idx / NL, tt = idx % NL;
          double c2 = 0.0;
          for (int k = 0; k < NQ; ++k) {
            int kx, ky;
            face_pt(f, k, NQ, kx, ky);
            double vh[2], dx[2], dy[2];
            rt_ref<P>(t, a, kx, ky, vh, dx, dy);
            c2 += t.op[tt][k] * (vh[0] * o0[6 * k] + vh[1] * o0[6 * k + 1]);
          }
          sm.C2[a][f * NL + tt] = c2;
        }
      } else {
        for (int idx = tid; idx < NQ * NJ; idx += nth) {
          const int k = idx / NJ, a = idx % NJ;
          int kx, ky;
          face_pt(f, k, NQ, kx, ky);
          double vh[2], dx[2], dy[2];
          rt_ref<P>(t, a, kx, ky, vh, dx, dy);
          const double* o = o0 + 6 * k;
          sm.pa[k][a] = vh[0] * o[0] + vh[1] * o[1];
          sm.pb[k][a] = vh[0] * o[2] + vh[1] * o[3];
        }
        __syncthreads();
        for (int idx = tid; idx < NJ * NJ + NJ; idx += nth) {
          const int a = idx < NJ * NJ ? idx / NJ : idx - NJ * NJ;
          const int b = idx < NJ * NJ ? idx % NJ : -1;
          double s = 0.0;
          if (b >= 0) {
            for (int k = 0; k < NQ; ++k) s += o0[6 * k + 4] * sm.pa[k][a] * sm.pb[k][b];
            sm.L[a * LD + b] += s;
          } else {
            for (int k = 0; k < NQ; ++k) s += o0[6 * k + 5] * sm.pa[k][a];
            sm.gv[a] += s;
          }
        }
      }
      __syncthreads();
    }
    // the assembled local system (inverted by hrt_invert_kernel) and the couplings
    for (int idx = tid; idx < MM * MM; idx += nth)
      out.Li[(size_t)e * MM * MM + idx] = sm.L[(idx / MM) * LD + idx % MM];
    for (int idx = tid; idx < NJ * NL4; idx += nth) out.C2[(size_t)e * NJ * NL4 + idx] = (&sm.C2[0][0])[idx];
    for (int a = tid; a < NJ; a += nth) out.g[(size_t)e * NJ + a] = sm.gv[a];
    for (int c = tid; c < N; c += nth) out.f[(size_t)e * N + c] = sm.fv[c];
  }
}

// Inversion of the assembled local systems and the element's share of the reduced system,
// apart from the assembly so that it runs many CTAs per SM: its Gauss-Jordan steps are
// short and separated by barriers, and only the number of CTAs in flight hides them.
template <int P>
struct HrtInvSmem {
  using S = HrtShape<P>;
  double L[S::MM * S::LD];
  double C1[S::NL4][S::NJ];
  double C2[S::NJ][S::NL4];
  double gv[S::NJ], fv[S::N];
  double T1[S::NJ][S::NL4];          // W C2
  double u[S::NJ];                   // W g + X f
  double colk[S::MM];
  double inv;                        // reciprocal of the current pivot
  int perm[S::MM];
  int piv;
};

template <int P>
__global__ void __launch_bounds__(128)
hrt_invert_kernel(long long E, int nx, int ny, HrtRef ref, HrtOut out, unsigned int* status) {
  using S = HrtShape<P>;
  constexpr int N = S::N, NJ = S::NJ, MM = S::MM, LD = S::LD, NL = S::NL, NL4 = S::NL4;
  extern __shared__ __align__(16) unsigned char hrt_inv_smem[];
  HrtInvSmem<P>& sm = *reinterpret_cast<HrtInvSmem<P>*>(hrt_inv_smem);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (long long e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    for (int idx = tid; idx < MM * MM; idx += nth)
      sm.L[(idx / MM) * LD + idx % MM] = out.Li[(size_t)e * MM * MM + idx];
    for (int idx = tid; idx < NL4 * NJ; idx += nth) {
      const int r = idx / NJ;
      (&sm.C1[0][0])[idx] = nb_elem(nx, ny, (int)e, r / NL) >= 0 ? ref.C1[idx] : 0.0;
      (&sm.C2[0][0])[idx] = out.C2[(size_t)e * NJ * NL4 + idx];
    }
    for (int a = tid; a < NJ; a += nth) sm.gv[a] = out.g[(size_t)e * NJ + a];
    for (int c = tid; c < N; c += nth) sm.fv[c] = out.f[(size_t)e * N + c];
    __syncthreads();
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
          sm.inv = 1.0 / sm.L[bi * LD + k];   // one FP64 division per step, not one per thread
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
      const double inv = sm.inv;
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

// the two elements and local faces on either side of interior face fid
__device__ __forceinline__ void face_sides(int nx, int ny, long long fid, long long& e1, int& f1, long long& e2,
                                           int& f2) {
  const long long nv = (long long)(nx - 1) * ny;
  if (fid < nv) {
    const long long j = fid / (nx - 1), i = fid % (nx - 1);
    e1 = j * nx + i; f1 = 1; e2 = e1 + 1; f2 = 3;
  } else {
    const long long h = fid - nv, j = h / nx, i = h % nx;
    e1 = j * nx + i; f1 = 2; e2 = e1 + nx; f2 = 0;
  }
}

// r[face dof] = the two sides' rows of r_e (the reduced right-hand side)
template <int P>
__global__ void hrt_gather_kernel(int nx, int ny, long long nfaces, const double* __restrict__ z,
                                  double* __restrict__ y) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nfaces * NL) return;
  long long e1, e2;
  int f1, f2;
  face_sides(nx, ny, t / NL, e1, f1, e2, f2);
  const int tt = (int)(t % NL);
  y[t] = z[e1 * NL4 + f1 * NL + tt] + z[e2 * NL4 + f2 * NL + tt];
}

// row (f NL + tt) of H_e applied to the element's multipliers (boundary faces carry none)
template <int P>
__device__ __forceinline__ double he_row(int nx, int ny, const double* __restrict__ He,
                                         const double* __restrict__ x, long long e, int f, int tt) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  const double* row = He + (size_t)e * NL4 * NL4 + (size_t)(f * NL + tt) * NL4;
  double s = 0.0;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const long long fi = face_index(nx, ny, (int)e, g);
    if (fi < 0) continue;
#pragma unroll
    for (int u = 0; u < NL; ++u) s = fma(row[g * NL + u], x[fi * NL + u], s);
  }
  return s;
}

// Element-patch additive Schwarz preconditioner: for each element the restriction of H to
// the multipliers of its interior faces, H_e plus, on each such face, the neighbour's
// diagonal block of that face (its only contribution there), inverted; the preconditioner
// applies every element's inverse to its faces' values and sums the two elements' results on
// each face.  One warp per element with the matrix in shared memory, Gauss-Jordan with
// partial pivoting; the rows and columns of boundary faces are the identity, so they stay
// decoupled and carry zeros.
template <int P>
__global__ void __launch_bounds__(128)
hrt_asm_setup_kernel(long long E, int nx, int ny, const double* __restrict__ He, double* __restrict__ Pinv,
                     unsigned int* status) {
  constexpr int NL = P + 1, NL4 = 4 * NL, LDP = NL4 + 1;
  __shared__ double sm[4][NL4 * LDP];
  __shared__ double scol[4][NL4];     // column k before the step
  __shared__ int sperm[4][NL4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long e = blockIdx.x * 4LL + w;
  if (e >= E) return;   // whole warps leave together; the kernel has no block barrier
  double* A = sm[w];
  int nbe[4], nbf[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    nbe[f] = nb_elem(nx, ny, (int)e, f);
    nbf[f] = (f + 2) & 3;
  }
  for (int idx = lane; idx < NL4 * NL4; idx += 32) {
    const int r = idx / NL4, c = idx % NL4, fr = r / NL, fc = c / NL;
    double v;
    if (nbe[fr] < 0 || nbe[fc] < 0) {
      v = r == c ? 1.0 : 0.0;
    } else {
      v = He[(size_t)e * NL4 * NL4 + idx];
      if (fr == fc) {
        const int on = nbf[fr] * NL;
        v += He[(size_t)nbe[fr] * NL4 * NL4 + (size_t)(on + r % NL) * NL4 + on + c % NL];
      }
    }
    A[r * LDP + c] = v;
  }
  __syncwarp();
  bool singular = false;
  for (int k = 0; k < NL4; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + lane; i < NL4; i += 32) {
      const double v = fabs(A[i * LDP + k]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    singular = singular || !(best > 1e-300);
    if (lane == 0) sperm[w][k] = bi;
    if (bi != k)
      for (int j = lane; j < NL4; j += 32) {
        const double t = A[k * LDP + j];
        A[k * LDP + j] = A[bi * LDP + j];
        A[bi * LDP + j] = t;
      }
    __syncwarp();
    const double inv = 1.0 / A[k * LDP + k];
    for (int i = lane; i < NL4; i += 32) scol[w][i] = A[i * LDP + k];
    __syncwarp();
    for (int j = lane; j < NL4; j += 32)
      if (j != k) A[k * LDP + j] *= inv;
    __syncwarp();
    for (int idx = lane; idx < NL4 * NL4; idx += 32) {
      const int i = idx / NL4, j = idx % NL4;
      if (i == k) continue;
      const double cik = scol[w][i];
      if (j == k) A[i * LDP + k] = -cik * inv;
      else A[i * LDP + j] -= cik * A[k * LDP + j];
    }
    __syncwarp();
    if (lane == 0) A[k * LDP + k] = inv;
    __syncwarp();
  }
  for (int k = NL4 - 1; k >= 0; --k) {   // undo the row interchanges as column interchanges
    const int pr = sperm[w][k];
    if (pr != k)
      for (int i = lane; i < NL4; i += 32) {
        const double t = A[i * LDP + k];
        A[i * LDP + k] = A[i * LDP + pr];
        A[i * LDP + pr] = t;
      }
    __syncwarp();
  }
  for (int idx = lane; idx < NL4 * NL4; idx += 32) Pinv[(size_t)e * NL4 * NL4 + idx] = A[(idx / NL4) * LDP + idx % NL4];
  if (lane == 0 && singular) atomicOr(status, kDevSingular);
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

// ---- the multiplier system's Krylov solve: BiCGStab (van der Vorst) with the two-level
// Schwarz preconditioner (the element patches above and the coarse space below).  Its
// scalars stay on the device: every dot product is reduced in two fixed stages (per-block
// partial sums, then each reader sums the kKB partials in the same order), so the iteration
// is deterministic and no kernel waits on the host; the host reads the convergence state
// once every kCheck iterations.  One iteration is 11 launches: p; p_hat = M^{-1} p (element
// patches with the coarse restriction, coarse solve, per-multiplier gather); v = H p_hat
// with r_hat.v; s; s_hat (the same three); t = H s_hat with t.s and t.t; lambda and r with
// r_hat.r and r.r.  The
// kernels take their iteration as an offset from a base index held on the device, so one
// CUDA graph of kCheck iterations (and the base's advance) is replayed block after block.
constexpr int kKB = 256, kKT = 256, kCheck = 16;
enum { kDotRV = 0, kDotTS = 1, kDotTT = 2, kDotRR_hat = 3, kDotRR = 4, kNumDots = 5 };

struct KScal { double rho, alpha, omega; };
struct KState {
  int done;      // 1: converged, 2: breakdown
  int iters;     // iterations completed when done was set
  int base;      // iterations launched before the current block
  int pad;
  double bb;     // ||r0||^2
  double rr;     // ||r||^2 at the last check
  double tol2;   // squared relative tolerance
};
static_assert(sizeof(KState) % sizeof(double) == 0, "KState is carved from a double buffer");

struct Kry {
  int nx, ny;
  long long nfaces, nl;
  long long E;
  const double* He;
  const double* Pinv;   // [E][4 (p+1)][4 (p+1)] element-patch inverses of the preconditioner
  double* z;            // [E][4 (p+1)] the preconditioner's element results
  // coarse space of the preconditioner: bilinear functions on a grid of (ncx+1) x (ncy+1)
  // vertices whose cells hold cx x cy elements (the last ones fewer)
  int ncx, ncy, cx, cy, nc;
  double gl[kMaxP + 1];   // the multiplier nodes on [0, 1]
  int* cv;                // [nl] lower-left coarse vertex of each multiplier's coarse cell
  double2* cw;            // [nl] its local coordinates (xi, eta) in that cell
  double* A0;             // [nc][nc] the coarse operator R0 H R0^T, then its inverse
  double* pc;             // [ncx ncy][4] per cell: its multipliers' restriction to its vertices
  double* zc;             // [nc] coarse correction
  double *x, *r, *rh, *p, *v, *s, *t, *ph, *sh;
  double* part;   // [kNumDots][kKB]
  KScal* sc;      // [iterations + 1]: sc[i] holds iteration i's rho, alpha, omega (sc[0] = 1)
  KState* st;
};

// whether an earlier launch ended the iteration (read once per block, so the whole block
// leaves together)
__device__ __forceinline__ bool kry_stopped(const Kry& k) {
  __shared__ int done;
  if (threadIdx.x == 0) done = *(volatile const int*)&k.st->done;
  __syncthreads();
  return done != 0;
}

// sum of the kKB partials of dot q, in a fixed order, broadcast to the block
__device__ double kry_sum(const double* __restrict__ part, int q, double* red) {
  if (threadIdx.x < 32) {
    double a = 0.0;
#pragma unroll
    for (int i = 0; i < kKB / 32; ++i) a += part[q * kKB + threadIdx.x + 32 * i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (threadIdx.x == 0) *red = a;
  }
  __syncthreads();
  const double v = *red;
  __syncthreads();
  return v;
}

// block sums of a and b into part[qa][blockIdx], part[qb][blockIdx] (qb < 0: a only)
__device__ void kry_partial(double a, double b, double* part, int qa, int qb) {
  __shared__ double ra[kKT / 32], rb[kKT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ra[w] = a; rb[w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { sa += ra[i]; sb += rb[i]; }
    part[qa * kKB + blockIdx.x] = sa;
    if (qb >= 0) part[qb * kKB + blockIdx.x] = sb;
  }
}

// The preconditioner's element half: z_e = Pinv_e x|e for every element and row (the face
// half, each face's two sides summed, is kry_precond_gather_kernel), on blocks b of nb
template <int P>
__device__ __forceinline__ void asm_apply_blocks(const Kry& k, const double* __restrict__ x, unsigned b,
                                                 unsigned nb) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  for (long long t = b * (long long)blockDim.x + threadIdx.x; t < k.E * NL4; t += (long long)nb * blockDim.x) {
    const long long e = t / NL4;
    const double* row = k.Pinv + (size_t)t * NL4;
    double s = 0.0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const long long fi = face_index(k.nx, k.ny, (int)e, g);
      if (fi < 0) continue;
#pragma unroll
      for (int u = 0; u < NL; ++u) s = fma(row[g * NL + u], x[fi * NL + u], s);
    }
    k.z[t] = s;
  }
}

// ---- coarse space of the preconditioner (two-level additive Schwarz): the coarse
// functions are bilinear on a grid of at most 12 x 12 vertices laid over the elements, taken
// at the multiplier nodes of every interior face; the coarse operator A0 = R0 H R0^T is
// assembled from the elements' H_e and inverted once per solve, and each application adds
// R0^T A0^{-1} R0 x to the element-patch part.
// (144 vertices: the coarse operator, 162 KB in FP64, is inverted in one CTA's shared memory)
constexpr int kCoarseMaxCells = 11, kCoarseMax = (kCoarseMaxCells + 1) * (kCoarseMaxCells + 1);

// the coarse cell holding multiplier node tt of interior face fid (its lower-left vertex v0)
// and the node's local coordinates in it.  A node on a cell's left or lower line belongs to
// that cell, one on the domain's right or upper coarse line to the last cell: so vertical
// faces on lines x = i0 .. i1 - 1 and horizontal faces on lines y = j0 .. j1 - 1 of the
// cell's element range [i0, i1) x [j0, j1) are its own.
__device__ __forceinline__ void coarse_coords(const Kry& k, long long fid, int tt, int& v0, double& xi,
                                              double& eta) {
  const long long nv = (long long)(k.nx - 1) * k.ny;
  double X, Y;   // in element widths from the lower-left corner
  if (fid < nv) {
    const long long j = fid / (k.nx - 1), i = fid % (k.nx - 1);
    X = (double)(i + 1);
    Y = (double)j + k.gl[tt];
  } else {
    const long long h = fid - nv, j = h / k.nx, i = h % k.nx;
    X = (double)i + k.gl[tt];
    Y = (double)(j + 1);
  }
  const int kx = min((int)(X / k.cx), k.ncx - 1), ky = min((int)(Y / k.cy), k.ncy - 1);
  const double x0 = (double)(kx * k.cx), x1 = (double)min((kx + 1) * k.cx, k.nx);
  const double y0 = (double)(ky * k.cy), y1 = (double)min((ky + 1) * k.cy, k.ny);
  xi = (X - x0) / (x1 - x0);
  eta = (Y - y0) / (y1 - y0);
  v0 = ky * (k.ncx + 1) + kx;
}

// the four bilinear weights, vertices in the order v0, v0 + 1, v0 + W, v0 + W + 1
__device__ __forceinline__ void bilinear(double xi, double eta, double w[4]) {
  w[0] = (1.0 - xi) * (1.0 - eta);
  w[1] = xi * (1.0 - eta);
  w[2] = (1.0 - xi) * eta;
  w[3] = xi * eta;
}

// coarse vertices and bilinear weights of multiplier node tt of interior face fid
__device__ __forceinline__ void coarse_weights(const Kry& k, long long fid, int tt, int v[4], double w[4]) {
  double xi, eta;
  coarse_coords(k, fid, tt, v[0], xi, eta);
  const int W = k.ncx + 1;
  v[1] = v[0] + 1;
  v[2] = v[0] + W;
  v[3] = v[2] + 1;
  bilinear(xi, eta, w);
}

// the node table of the coarse space, once per solve
template <int P>
__global__ void hrt_coarse_nodes_kernel(Kry k) {
  constexpr int NL = P + 1;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= k.nl) return;
  int v0;
  double xi, eta;
  coarse_coords(k, t / NL, (int)(t % NL), v0, xi, eta);
  k.cv[t] = v0;
  k.cw[t] = make_double2(xi, eta);
}

// per coarse cell (one CTA): the sum over its elements of P_e^T H_e P_e, P_e the element's
// multipliers' weights on the cell's four vertices (every face of an element inside the
// cell lies in the cell's closure); threads take elements in a fixed stride and the block
// sums in a fixed order
template <int P>
__global__ void __launch_bounds__(128) hrt_coarse_cell_kernel(Kry k, double* __restrict__ Acell) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  const int cell = blockIdx.x, kx = cell % k.ncx, ky = cell / k.ncx;
  const int i0 = kx * k.cx, i1 = min(i0 + k.cx, k.nx), j0 = ky * k.cy, j1 = min(j0 + k.cy, k.ny);
  const int ni = i1 - i0, nel = ni * (j1 - j0);
  const int W = k.ncx + 1;
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  for (int t = threadIdx.x; t < nel; t += blockDim.x) {
    const long long e = (long long)(j0 + t / ni) * k.nx + i0 + t % ni;
    double Pw[NL4][4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const long long fi = face_index(k.nx, k.ny, (int)e, g);
#pragma unroll
      for (int tt = 0; tt < NL; ++tt) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Pw[g * NL + tt][c] = 0.0;
        if (fi < 0) continue;
        int v[4];
        double w[4];
        coarse_weights(k, fi, tt, v, w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          // a face on the cell's upper or right line may be assigned to the next cell, whose
          // far vertices then carry weight zero: keep the cell's own four
          const int lx = v[c] % W - kx, ly = v[c] / W - ky;
          if (lx < 0 || lx > 1 || ly < 0 || ly > 1) continue;
          Pw[g * NL + tt][ly * 2 + lx] += w[c];
        }
      }
    }
    const double* He = k.He + (size_t)e * NL4 * NL4;
    for (int i = 0; i < NL4; ++i) {
      double T[4] = {0.0, 0.0, 0.0, 0.0};   // (H_e P_e)[i][:]
      for (int j = 0; j < NL4; ++j) {
        const double h = He[i * NL4 + j];
#pragma unroll
        for (int b = 0; b < 4; ++b) T[b] = fma(h, Pw[j][b], T[b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a * 4 + b] = fma(Pw[i][a], T[b], acc[a * 4 + b]);
    }
  }
  __shared__ double red[4][16];   // blockDim 128: four warps
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    double x = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < 16)
    Acell[(size_t)cell * 16 + threadIdx.x] =
        ((red[0][threadIdx.x] + red[1][threadIdx.x]) + red[2][threadIdx.x]) + red[3][threadIdx.x];
}

// the dense coarse operator, one row per thread from the cells around its vertex
__global__ void hrt_coarse_assemble_kernel(Kry k, const double* __restrict__ Acell) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= k.nc) return;
  const int W = k.ncx + 1, ax = a % W, ay = a / W;
  double* row = k.A0 + (size_t)a * k.nc;
  for (int b = 0; b < k.nc; ++b) row[b] = 0.0;
  for (int cy = ay - 1; cy <= ay; ++cy)
    for (int cx = ax - 1; cx <= ax; ++cx) {
      if (cx < 0 || cy < 0 || cx >= k.ncx || cy >= k.ncy) continue;
      const int cell = cy * k.ncx + cx, la = (ay - cy) * 2 + (ax - cx);
      for (int lb = 0; lb < 4; ++lb) {
        const int b = (cy + lb / 2) * W + cx + lb % 2;
        row[b] += Acell[(size_t)cell * 16 + la * 4 + lb];
      }
    }
  // a coarse function that vanishes on every interior face (a domain corner's when its cell
  // is one element wide) has an empty row and column: put 1 on the diagonal, its restriction
  // being zero, so it contributes nothing and A0 stays invertible
  double mx = 0.0;
  for (int b = 0; b < k.nc; ++b) mx = fmax(mx, fabs(row[b]));
  if (mx == 0.0) row[a] = 1.0;
}

// Gauss-Jordan inverse of the coarse operator with partial pivoting, in FP32 in one CTA's
// shared memory, of A0 scaled by its largest entry; written back in FP64 over A0.  The
// coarse solve is part of the preconditioner only: its accuracy changes the iteration
// count, not the FP64 Krylov iteration's answer.  (FP64 here is held to one SM's two FP64
// FMA per clock: n^3 = 3 M FMA is 0.75 ms, FP32 runs at 64 times that rate.)
// Per pivot step two barriers: every warp finds the pivot row itself (same order, same
// result), the pivot row, the row it changes places with and the pivot column go to
// buffers, and each thread then updates only its own entries, reading the row that moves
// to row pr from the buffer.  A pivot below 1e-30 of the largest entry (A0 singular in
// FP32) drops the coarse part: the inverse is written as zero and the preconditioner is the
// element patches alone.
constexpr int kCoarseInvThreads = 512, kCoarsePerLane = (kCoarseMax + 31) / 32;
__global__ void __launch_bounds__(kCoarseInvThreads) hrt_coarse_invert_kernel(Kry k) {
  const int n = k.nc, ld = n | 1, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarp = kCoarseInvThreads / 32;
  extern __shared__ float A[];   // [n][ld]
  __shared__ float R[kCoarseMax], krow[kCoarseMax], colk[kCoarseMax];
  __shared__ int perm[kCoarseMax], src[kCoarseMax];
  __shared__ double wmax[nwarp];
  __shared__ int singular;
  if (tid == 0) singular = 0;
  double m = 0.0;
  for (int idx = tid; idx < n * n; idx += kCoarseInvThreads) m = fmax(m, fabs(k.A0[idx]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[warp] = m;
  __syncthreads();
  m = 0.0;
  for (int w = 0; w < nwarp; ++w) m = fmax(m, wmax[w]);
  const double rs = m > 0.0 ? 1.0 / m : 1.0;
  for (int idx = tid; idx < n * n; idx += kCoarseInvThreads) A[(idx / n) * ld + idx % n] = (float)(k.A0[idx] * rs);
  __syncthreads();
  for (int kk = 0; kk < n; ++kk) {
    float best = -1.0f;
    int pr = kk;
#pragma unroll
    for (int q = 0; q < kCoarsePerLane; ++q) {
      const int i = kk + lane + 32 * q;
      const float v = i < n ? fabsf(A[i * ld + kk]) : -1.0f;
      if (v > best) { best = v; pr = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, pr, o);
      if (ob > best || (ob == best && oi < pr)) { best = ob; pr = oi; }
    }
    if (tid == 0) {
      perm[kk] = pr;
      if (!(best > 1e-30f)) singular = 1;
    }
    const float iv = 1.0f / A[pr * ld + kk];
    for (int j = tid; j < n; j += kCoarseInvThreads) {
      R[j] = j == kk ? iv : A[pr * ld + j] * iv;
      krow[j] = A[kk * ld + j];
      colk[j] = j == kk ? A[pr * ld + kk] : (j == pr ? A[kk * ld + kk] : A[j * ld + kk]);
    }
    __syncthreads();
    float r[kCoarsePerLane];   // this lane's columns of the new pivot row
#pragma unroll
    for (int q = 0; q < kCoarsePerLane; ++q) r[q] = lane + 32 * q < n ? R[lane + 32 * q] : 0.0f;
    for (int i = warp; i < n; i += nwarp) {
      float* Ai = A + i * ld;
      const float c = colk[i];
      const bool moved = i == pr;   // row pr now holds the old row kk
      float a[kCoarsePerLane];      // all loads of the row before its stores
#pragma unroll
      for (int q = 0; q < kCoarsePerLane; ++q) {
        const int j = lane + 32 * q;
        a[q] = j < n ? (moved ? krow[j] : Ai[j]) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < kCoarsePerLane; ++q) {
        const int j = lane + 32 * q;
        if (j < n) Ai[j] = i == kk ? r[q] : (j == kk ? -c * iv : fmaf(-c, r[q], a[q]));
      }
    }
    __syncthreads();
  }
  // the row interchanges, undone as column interchanges in reverse order, as one gather
  if (tid == 0) {
    for (int j = 0; j < n; ++j) src[j] = j;
    for (int kk = n - 1; kk >= 0; --kk) {
      const int t = src[kk];
      src[kk] = src[perm[kk]];
      src[perm[kk]] = t;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += kCoarseInvThreads) {
    const int i = idx / n, j = idx % n;
    k.A0[idx] = singular ? 0.0 : (double)A[i * ld + src[j]] * rs;
  }
}

// per coarse cell (one CTA): the restriction of x to its four vertices from the multiplier
// nodes the cell owns (coarse_coords), threads in a fixed stride and a fixed-order block sum
template <int P>
__device__ __forceinline__ void coarse_restrict_cell(const Kry& k, const double* __restrict__ x, int cell) {
  constexpr int NL = P + 1;
  const int kx = cell % k.ncx, ky = cell / k.ncx;
  const int i0 = kx * k.cx, i1 = min(i0 + k.cx, k.nx), j0 = ky * k.cy, j1 = min(j0 + k.cy, k.ny);
  const long long nv = (long long)(k.nx - 1) * k.ny;
  const int xa = max(i0, 1), ya = max(j0, 1);
  const int nvf = max(0, i1 - xa) * (j1 - j0), nhf = max(0, j1 - ya) * (i1 - i0);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < (nvf + nhf) * NL; t += blockDim.x) {
    const int fl = t / NL, tt = t - fl * NL;
    long long fid;
    if (fl < nvf) {
      const int xv = xa + fl / (j1 - j0), j = j0 + fl % (j1 - j0);
      fid = (long long)j * (k.nx - 1) + (xv - 1);
    } else {
      const int g = fl - nvf, yh = ya + g / (i1 - i0), i = i0 + g % (i1 - i0);
      fid = nv + (long long)(yh - 1) * k.nx + i;
    }
    const long long q = fid * NL + tt;
    const double2 c = k.cw[q];
    double w[4];
    bilinear(c.x, c.y, w);
    const double xq = x[q];
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[b] = fma(w[b], xq, acc[b]);
  }
  __shared__ double red[8][4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    double v = acc[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][b] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double sum = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += red[i][threadIdx.x];
    k.pc[(size_t)cell * 4 + threadIdx.x] = sum;
  }
}

// the two parts of an application that read only x, in one launch: blocks [0, napply) the
// element patches, the rest one coarse cell each
template <int P>
__global__ void __launch_bounds__(256) kry_precond_local_kernel(Kry k, const double* __restrict__ x,
                                                                unsigned napply) {
  if (kry_stopped(k)) return;
  if (blockIdx.x < napply) asm_apply_blocks<P>(k, x, blockIdx.x, napply);
  else coarse_restrict_cell<P>(k, x, (int)(blockIdx.x - napply));
}

// zc = A0^{-1} vc, vc summed per vertex from the cells around it (fixed order) into shared
// memory by every block, then one warp per row
__global__ void __launch_bounds__(256) kry_coarse_solve_kernel(Kry k) {
  if (kry_stopped(k)) return;
  __shared__ double vc[kCoarseMax];
  const int W = k.ncx + 1;
  for (int a = threadIdx.x; a < k.nc; a += blockDim.x) {
    const int ax = a % W, ay = a / W;
    double v = 0.0;
    for (int cy = ay - 1; cy <= ay; ++cy)
      for (int cx = ax - 1; cx <= ax; ++cx) {
        if (cx < 0 || cy < 0 || cx >= k.ncx || cy >= k.ncy) continue;
        v += k.pc[(size_t)(cy * k.ncx + cx) * 4 + (ay - cy) * 2 + (ax - cx)];
      }
    vc[a] = v;
  }
  __syncthreads();
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= k.nc) return;
  const double* Ar = k.A0 + (size_t)row * k.nc;
  double s = 0.0;
  for (int b = lane; b < k.nc; b += 32) s = fma(Ar[b], vc[b], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) k.zc[row] = s;
}

// y = M^{-1} x assembled per multiplier: the two sides' element-patch results plus the
// coarse correction R0^T zc
template <int P>
__global__ void kry_precond_gather_kernel(Kry k, double* __restrict__ y) {
  constexpr int NL = P + 1, NL4 = 4 * NL;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= k.nl) return;
  long long e1, e2;
  int f1, f2;
  face_sides(k.nx, k.ny, t / NL, e1, f1, e2, f2);
  const int tt = (int)(t % NL);
  const int v0 = k.cv[t], W = k.ncx + 1;
  const double2 c = k.cw[t];
  double w[4];
  bilinear(c.x, c.y, w);
  const double cor = fma(w[3], k.zc[v0 + W + 1], fma(w[2], k.zc[v0 + W], fma(w[1], k.zc[v0 + 1], w[0] * k.zc[v0])));
  y[t] = (k.z[e1 * NL4 + f1 * NL + tt] + k.z[e2 * NL4 + f2 * NL + tt]) + cor;
}

// r_hat = r, x = p = v = 0, partials of r_hat.r and r.r, sc[0] = 1, state cleared
__global__ void kry_init_kernel(Kry k, double tol2) {
  double a = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k.nl; i += (long long)gridDim.x * blockDim.x) {
    const double ri = k.r[i];
    k.rh[i] = ri;
    k.x[i] = 0.0; k.p[i] = 0.0; k.v[i] = 0.0;
    a = fma(ri, ri, a);
  }
  kry_partial(a, a, k.part, kDotRR_hat, kDotRR);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    k.sc[0] = KScal{1.0, 1.0, 1.0};
    *k.st = KState{0, 0, 0, 0, 0.0, 0.0, tol2};
  }
}

// iteration base + j, step 1: convergence test on the previous residual, rho, p.
// With update == false it only records the state (the final check after the last
// iteration).
template <int P>
__global__ void kry_p_kernel(Kry k, int j, bool update) {
  __shared__ double red;
  if (kry_stopped(k)) return;
  const int it = k.st->base + j;
  const double rr = kry_sum(k.part, kDotRR, &red);
  const double rho = kry_sum(k.part, kDotRR_hat, &red);
  const double bb = it == 0 ? rr : k.st->bb;
  const bool conv = rr <= k.st->tol2 * bb;
  const KScal pv = k.sc[it];
  const bool brk = !conv && update && (rho == 0.0 || !isfinite(rho) || pv.omega == 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (it == 0) k.st->bb = rr;
    k.st->rr = rr;
    if (conv || brk) { k.st->done = conv ? 1 : 2; k.st->iters = it; }
    k.sc[it + 1].rho = rho;
  }
  if (conv || brk || !update) return;
  const double beta = (rho / pv.rho) * (pv.alpha / pv.omega);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k.nl; i += (long long)gridDim.x * blockDim.x)
    k.p[i] = k.r[i] + beta * (k.p[i] - pv.omega * k.v[i]);
}

// y = H x with the partial dots w.y (into qa) and, when qb >= 0, y.y (into qb)
template <int P>
__global__ void kry_matvec_kernel(Kry k, const double* __restrict__ x, double* __restrict__ y,
                                  const double* __restrict__ w, int qa, int qb) {
  constexpr int NL = P + 1;
  if (kry_stopped(k)) return;
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k.nl; i += (long long)gridDim.x * blockDim.x) {
    long long e1, e2;
    int f1, f2;
    face_sides(k.nx, k.ny, i / NL, e1, f1, e2, f2);
    const int tt = (int)(i % NL);
    const double yi = he_row<P>(k.nx, k.ny, k.He, x, e1, f1, tt) + he_row<P>(k.nx, k.ny, k.He, x, e2, f2, tt);
    y[i] = yi;
    a = fma(w[i], yi, a);
    b = fma(yi, yi, b);
  }
  kry_partial(a, b, k.part, qa, qb);
}

// step 3: alpha, s = r - alpha v
template <int P>
__global__ void kry_s_kernel(Kry k, int j) {
  __shared__ double red;
  if (kry_stopped(k)) return;
  const int it = k.st->base + j;
  const double rv = kry_sum(k.part, kDotRV, &red);
  const double alpha = k.sc[it + 1].rho / rv;
  if (!isfinite(alpha)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) { k.st->done = 2; k.st->iters = it; }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) k.sc[it + 1].alpha = alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k.nl; i += (long long)gridDim.x * blockDim.x)
    k.s[i] = k.r[i] - alpha * k.v[i];
}

// step 5: omega, lambda += alpha p_hat + omega s_hat, r = s - omega t, and the partials of
// r_hat.r and r.r for the next iteration's test
__global__ void kry_x_kernel(Kry k, int j) {
  __shared__ double red;
  if (kry_stopped(k)) return;
  const int it = k.st->base + j;
  const double ts = kry_sum(k.part, kDotTS, &red);
  const double tt = kry_sum(k.part, kDotTT, &red);
  const double alpha = k.sc[it + 1].alpha;
  const double omega = tt > 0.0 ? ts / tt : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) k.sc[it + 1].omega = omega;
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k.nl; i += (long long)gridDim.x * blockDim.x) {
    k.x[i] += alpha * k.ph[i] + omega * k.sh[i];
    const double ri = k.s[i] - omega * k.t[i];
    k.r[i] = ri;
    a = fma(k.rh[i], ri, a);
    b = fma(ri, ri, b);
  }
  kry_partial(a, b, k.part, kDotRR_hat, kDotRR);
}

// the base index advances past a block of n iterations
__global__ void kry_bump_kernel(KState* st, int n) { st->base += n; }

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// n iterations starting at offset 0 from the device's base, then the base's advance
template <int P>
static void kry_block(const Kry& k, int n, cudaStream_t s) {
  constexpr int NL4 = 4 * (P + 1);
  const unsigned eb = nblk(k.E * NL4, 256), fb = nblk(k.nl, 256);
  // element patches, coarse restriction and solve, then per multiplier the sum
  auto precond = [&](const double* x, double* y) {
    kry_precond_local_kernel<P><<<eb + (unsigned)(k.ncx * k.ncy), 256, 0, s>>>(k, x, eb);
    kry_coarse_solve_kernel<<<(unsigned)((k.nc + 7) / 8), 256, 0, s>>>(k);
    kry_precond_gather_kernel<P><<<fb, 256, 0, s>>>(k, y);
  };
  for (int j = 0; j < n; ++j) {
    kry_p_kernel<P><<<kKB, kKT, 0, s>>>(k, j, true);
    precond(k.p, k.ph);                                                        // p_hat = M^{-1} p
    kry_matvec_kernel<P><<<kKB, kKT, 0, s>>>(k, k.ph, k.v, k.rh, kDotRV, -1);
    kry_s_kernel<P><<<kKB, kKT, 0, s>>>(k, j);
    precond(k.s, k.sh);                                                        // s_hat = M^{-1} s
    kry_matvec_kernel<P><<<kKB, kKT, 0, s>>>(k, k.sh, k.t, k.s, kDotTS, kDotTT);
    kry_x_kernel<<<kKB, kKT, 0, s>>>(k, j);
  }
  kry_bump_kernel<<<1, 1, 0, s>>>(k.st, n);
}

// The graph of one block of kCheck iterations for the mesh's current scratch layout,
// captured once and kept on the handle while the layout stays.
template <int P>
static vef_status kry_graph(Mesh& M, const Kry& k, cudaGraphExec_t* out) {
  if (M.hrt_graph && M.hrt_graph_work == (const void*)M.work && M.hrt_graph_nl == k.nl && M.hrt_graph_p == P) {
    *out = M.hrt_graph;
    return VEF_OK;
  }
  if (M.hrt_graph) {
    cudaGraphExecDestroy(M.hrt_graph);
    M.hrt_graph = nullptr;
  }
  cudaStream_t cs;
  VEF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    kry_block<P>(k, kCheck, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&M.hrt_graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    M.hrt_graph = nullptr;
    set_last_error(std::string("CUDA error capturing the multiplier iteration: ") + cudaGetErrorString(e));
    return VEF_ERR_CUDA;
  }
  M.hrt_graph_work = M.work;
  M.hrt_graph_nl = k.nl;
  M.hrt_graph_p = P;
  *out = M.hrt_graph;
  return VEF_OK;
}

template <int P>
static vef_status hrt_run(Mesh& M, const HrtIn& in, double tol, int max_iter, double* phi, double* J,
                          double* lambda, vef_hrt_info* info, cudaStream_t s) {
  using S = HrtShape<P>;
  const long long E = M.E;
  const long long nfaces = (long long)(M.nx - 1) * M.ny + (long long)M.nx * (M.ny - 1);
  const long long nl = nfaces * S::NL;
  const size_t per_e = (size_t)S::MM * S::MM + (size_t)S::NJ * S::NL4 + S::NJ + S::N + (size_t)S::NL4 * S::NL4 +
                       S::NL4;
  const size_t vec = (size_t)std::max(1LL, nl);
  const size_t nsc = (size_t)max_iter + 2;
  const HrtTab tab = make_hrt_tab(P, M.m);
  std::vector<double> refh;
  make_hrt_ref<P>(tab, refh);
  // the coarse grid: at most kCoarseMaxCells cells per direction
  Kry k{};
  k.cx = (M.nx + kCoarseMaxCells - 1) / kCoarseMaxCells;
  k.cy = (M.ny + kCoarseMaxCells - 1) / kCoarseMaxCells;
  k.ncx = (M.nx + k.cx - 1) / k.cx;
  k.ncy = (M.ny + k.cy - 1) / k.cy;
  const int nc = (k.ncx + 1) * (k.ncy + 1);
  k.nc = nc;
  {
    double gw[kMaxP + 1];
    gauss_legendre(P + 1, k.gl, gw);
  }
  const size_t total = per_e * E + 10 * vec + (size_t)(S::NL4 * S::NL4 + S::NL4) * E +
                       (size_t)nc * nc + (size_t)nc + 20 * (size_t)k.ncx * k.ncy + 2 * vec + (vec + 1) / 2 +
                       (size_t)kNumDots * kKB + 3 * nsc + sizeof(KState) / sizeof(double) + refh.size() +
                       32;   // each of the takes below rounded up to two doubles
  vef_status st = ensure_buffer((void**)&M.work, &M.work_cap, total * sizeof(double));
  if (st != VEF_OK) return st;
  double* base = M.work;
  // 16-byte aligned pieces (cw is read as double2)
  auto take = [&](size_t n) { double* q = base; base += (n + 1) & ~(size_t)1; return q; };
  double* Li = take((size_t)S::MM * S::MM * E);
  double* C2 = take((size_t)S::NJ * S::NL4 * E);
  double* g = take((size_t)S::NJ * E);
  double* f = take((size_t)S::N * E);
  double* He = take((size_t)S::NL4 * S::NL4 * E);
  double* re = take((size_t)S::NL4 * E);
  k.nx = M.nx; k.ny = M.ny; k.nfaces = nfaces; k.nl = nl; k.He = He;
  k.x = take(vec);   // copied to lambda at the end (the graph keeps one layout)
  k.r = take(vec); k.rh = take(vec); k.p = take(vec); k.v = take(vec); k.s = take(vec);
  k.t = take(vec); k.ph = take(vec); k.sh = take(vec);
  double* Pinv = take((size_t)S::NL4 * S::NL4 * E);
  k.Pinv = Pinv;
  k.z = take((size_t)S::NL4 * E);
  k.E = E;
  k.A0 = take((size_t)nc * nc);
  k.pc = take((size_t)4 * k.ncx * k.ncy);
  k.zc = take((size_t)nc);
  double* Acell = take((size_t)16 * k.ncx * k.ncy);
  k.cw = reinterpret_cast<double2*>(take(2 * vec));
  k.cv = reinterpret_cast<int*>(take((vec + 1) / 2));
  k.part = take((size_t)kNumDots * kKB);
  k.st = reinterpret_cast<KState*>(take(sizeof(KState) / sizeof(double)));
  k.sc = reinterpret_cast<KScal*>(take(3 * nsc));   // last: its length follows max_iter
  double* refd = take(refh.size());
  // pageable source: the copy has taken the data when the call returns
  VEF_CUDA_TRY(cudaMemcpyAsync(refd, refh.data(), refh.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  const HrtRef ref{refd, refd + (size_t)S::N * S::NJ};
  HrtOut out{Li, C2, g, f, He, re};
  const size_t smem = sizeof(HrtSmem<P>), ismem = sizeof(HrtInvSmem<P>);
  VEF_CUDA_TRY(cudaFuncSetAttribute(hrt_local_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  VEF_CUDA_TRY(cudaFuncSetAttribute(hrt_invert_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
  const size_t csmem = (size_t)nc * (nc | 1) * sizeof(float);
  VEF_CUDA_TRY(cudaFuncSetAttribute(hrt_coarse_invert_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem));
  int dev = 0, sms = 0, inv_per_sm = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  VEF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VEF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&inv_per_sm, hrt_invert_kernel<P>, 128, ismem));
  {
    KTimer kt(&M, VEF_K_HRT, s);
    hrt_local_kernel<P><<<(unsigned)std::min<long long>(E, (long long)sms * 8), 256, smem, s>>>(
        E, M.nx, M.ny, tab, ref, in, out, M.dev_status);
    hrt_invert_kernel<P><<<(unsigned)std::min<long long>(E, (long long)sms * std::max(1, inv_per_sm)), 128, ismem,
                           s>>>(E, M.nx, M.ny, ref, out, M.dev_status);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  int it = 0;
  KState hs{};
  if (nl > 0) {
    hrt_gather_kernel<P><<<nblk(nl, 256), 256, 0, s>>>(M.nx, M.ny, nfaces, re, k.r);
    hrt_asm_setup_kernel<P><<<(unsigned)((E + 3) / 4), 128, 0, s>>>(E, M.nx, M.ny, He, Pinv, M.dev_status);
    hrt_coarse_nodes_kernel<P><<<nblk(nl, 256), 256, 0, s>>>(k);
    hrt_coarse_cell_kernel<P><<<(unsigned)(k.ncx * k.ncy), 128, 0, s>>>(k, Acell);
    hrt_coarse_assemble_kernel<<<nblk(nc, 128), 128, 0, s>>>(k, Acell);
    hrt_coarse_invert_kernel<<<1, kCoarseInvThreads, csmem, s>>>(k);
    kry_init_kernel<<<kKB, kKT, 0, s>>>(k, tol * tol);
    VEF_CUDA_TRY(cudaGetLastError());
    cudaGraphExec_t graph = nullptr;
    if (max_iter >= kCheck && (st = kry_graph<P>(M, k, &graph)) != VEF_OK) return st;
    while (it < max_iter) {
      const int n = std::min(kCheck, max_iter - it);
      if (n == kCheck) VEF_CUDA_TRY(cudaGraphLaunch(graph, s));
      else kry_block<P>(k, n, s);
      it += n;
      VEF_CUDA_TRY(cudaGetLastError());
      VEF_CUDA_TRY(cudaMemcpyAsync(&hs, k.st, sizeof(KState), cudaMemcpyDeviceToHost, s));
      VEF_CUDA_TRY(cudaStreamSynchronize(s));
      if (hs.done) break;
    }
    if (!hs.done) {   // the test after the last iteration
      kry_p_kernel<P><<<kKB, kKT, 0, s>>>(k, 0, false);
      VEF_CUDA_TRY(cudaMemcpyAsync(&hs, k.st, sizeof(KState), cudaMemcpyDeviceToHost, s));
      VEF_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (hs.done) it = hs.iters;
    if (lambda) VEF_CUDA_TRY(cudaMemcpyAsync(lambda, k.x, nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  {
    KTimer kt(&M, VEF_K_HRT, s);
    hrt_recover_kernel<P><<<(unsigned)std::min<long long>(E, (long long)sms * 8), 128, 0, s>>>(
        E, M.nx, M.ny, Li, C2, g, f, k.x, J, phi);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  const bool conv = nl == 0 || hs.done == 1;
  const double rel = nl == 0 || hs.bb <= 0.0 ? 0.0 : std::sqrt(hs.rr / hs.bb);
  if (info) {
    info->iterations = it;
    info->rel_residual = rel;
    info->multipliers = nl;
  }
  if (!conv) {
    set_last_error(hs.done == 2 ? "HRT multiplier solve broke down (BiCGStab)"
                                : "HRT multiplier solve did not reach its tolerance");
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
