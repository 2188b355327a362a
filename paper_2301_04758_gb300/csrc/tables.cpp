// Host-side 1D rules on [0,1]: Gauss-Lobatto and Gauss-Legendre points by Newton's
// method on the Legendre three-term recurrence, and Lagrange basis values/derivatives
// by the product formula.
#include <cmath>

#include "common.h"

namespace vef {

// P_n(x) and P_n'(x) by the recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // (1 - x^2) P_n' = n (P_{n-1} - x P_n)
  *dP = n * (p0 - x * p1) / (1.0 - x * x);
}

void gll_nodes(int m, double* out) {
  // endpoints plus the roots of P_m'; Newton on P_m' with
  // (1 - x^2) P_m'' = 2 x P_m' - m (m+1) P_m, started at Chebyshev-Lobatto points.
  out[0] = 0.0;
  out[m] = 1.0;
  for (int j = 1; j < m; ++j) {
    double x = -std::cos(M_PI * j / m);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(m, x, &P, &dP);
      double d2P = (2.0 * x * dP - m * (m + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    out[j] = 0.5 * (x + 1.0);
  }
}

void gauss_legendre(int n, double* x01, double* w01) {
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double P = 0, dP = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(n, x, &P, &dP);
      double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    legendre(n, x, &P, &dP);
    x01[i] = 0.5 * (x + 1.0);
    w01[i] = 1.0 / ((1.0 - x * x) * dP * dP);  // 2/((1-x^2)P'^2) on [-1,1], halved
  }
}

void lagrange_eval(int nn, const double* nodes, double x, double* val, double* der) {
  for (int a = 0; a < nn; ++a) {
    double v = 1.0;
    for (int c = 0; c < nn; ++c)
      if (c != a) v *= (x - nodes[c]) / (nodes[a] - nodes[c]);
    val[a] = v;
    double d = 0.0;
    for (int k = 0; k < nn; ++k) {
      if (k == a) continue;
      double t = 1.0 / (nodes[a] - nodes[k]);
      for (int c = 0; c < nn; ++c)
        if (c != a && c != k) t *= (x - nodes[c]) / (nodes[a] - nodes[c]);
      d += t;
    }
    der[a] = d;
  }
}

Tab1D make_tab1d(int p) {
  Tab1D t{};
  t.p = p;
  t.np1 = p + 1;
  t.nq = p + 2;
  gll_nodes(p, t.gll);
  gauss_legendre(t.nq, t.gl, t.glw);
  for (int k = 0; k < t.nq; ++k) {
    double v[kMaxP + 1], d[kMaxP + 1];
    lagrange_eval(p + 1, t.gll, t.gl[k], v, d);
    for (int a = 0; a <= p; ++a) {
      t.l[a][k] = v[a];
      t.dl[a][k] = d[a];
    }
  }
  return t;
}

}  // namespace vef
