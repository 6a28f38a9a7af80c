// Host construction of the 1D tables of the bases (reading of Section 3.2; the
// paper fixes neither nodes nor quadrature): Lagrange basis of order p on the
// Gauss-Lobatto-Legendre points (H1), Lagrange basis of order p-1 on the p
// Gauss-Legendre points (L2), and the q1-point Gauss-Legendre rule, all on the
// reference interval [0, 1].
#include <cmath>
#include <stdexcept>
#include <vector>

#include "lh_internal.h"

namespace lh {

// GLL points on [0,1] in closed form for p <= 4.
void gll_nodes(int p, double *z) {
  switch (p) {
    case 1: z[0] = 0.0; z[1] = 1.0; break;
    case 2: z[0] = 0.0; z[1] = 0.5; z[2] = 1.0; break;
    case 3: {
      const double a = 1.0 / std::sqrt(5.0);
      z[0] = 0.0; z[1] = 0.5 * (1.0 - a); z[2] = 0.5 * (1.0 + a); z[3] = 1.0;
      break;
    }
    case 4: {
      const double a = std::sqrt(3.0 / 7.0);
      z[0] = 0.0; z[1] = 0.5 * (1.0 - a); z[2] = 0.5; z[3] = 0.5 * (1.0 + a); z[4] = 1.0;
      break;
    }
    default: throw std::invalid_argument("order must be in 1..4");
  }
}

// n-point Gauss-Legendre rule on [0,1]: roots of P_n by Newton's method from the
// Chebyshev-like initial guesses cos(pi (k + 3/4) / (n + 1/2)), weights 2/((1-t^2) P_n'(t)^2).
static void gauss_legendre(int n, double *x, double *w) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double t = std::cos(pi * (k + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;                 // Legendre recurrence
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? t : p1;
      const double pm = n == 1 ? 1.0 : p0;
      dp = n * (t * pn - pm) / (t * t - 1.0);
      const double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = t;
    for (int j = 2; j <= n; ++j) {
      const double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    const double pn = n == 1 ? t : p1, pm = n == 1 ? 1.0 : p0;
    dp = n * (t * pn - pm) / (t * t - 1.0);
    // ascending order on [0,1]
    x[n - 1 - k] = 0.5 * (t + 1.0);
    w[n - 1 - k] = 1.0 / ((1.0 - t * t) * dp * dp);   // (2/((1-t^2)P'^2)) / 2
  }
}

static double lagrange(const double *z, int n, int i, double x) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != i) v *= (x - z[m]) / (z[i] - z[m]);
  return v;
}

static double lagrange_d(const double *z, int n, int i, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double t = 1.0 / (z[i] - z[m]);
    for (int k = 0; k < n; ++k)
      if (k != i && k != m) t *= (x - z[k]) / (z[i] - z[k]);
    s += t;
  }
  return s;
}

void h1_basis_at(int p, double x, double *vals, double *ders) {
  double z[5];
  gll_nodes(p, z);
  for (int i = 0; i <= p; ++i) {
    vals[i] = lagrange(z, p + 1, i, x);
    ders[i] = lagrange_d(z, p + 1, i, x);
  }
}

int table_length(int p, int q1) {
  const int D = p + 1, Q = q1, L = p;
  return 5 * Q * D + 2 * Q * L + 2 * Q + D;
}

void build_tables(int p, int q1, double *tab, int tab_len) {
  const int D = p + 1, Q = q1, L = p;
  if (tab_len < table_length(p, q1)) throw std::invalid_argument("table buffer too small");
  std::vector<double> xq(Q), wq(Q), z(D), zl(L > 0 ? L : 1), wl(L > 0 ? L : 1);
  gauss_legendre(Q, xq.data(), wq.data());
  gll_nodes(p, z.data());
  gauss_legendre(L, zl.data(), wl.data());
  const int oB = 0, oG = Q * D, oBt = 2 * Q * D, oGt = 3 * Q * D, oBl = 4 * Q * D, oBlt = oBl + Q * L,
            oB2t = oBlt + Q * L, oW = oB2t + Q * D, oIW = oW + Q, oZ = oIW + Q;
  for (int q = 0; q < Q; ++q) {
    for (int i = 0; i < D; ++i) {
      const double b = lagrange(z.data(), D, i, xq[q]);
      const double g = lagrange_d(z.data(), D, i, xq[q]);
      tab[oB + q * D + i] = b;
      tab[oG + q * D + i] = g;
      tab[oBt + i * Q + q] = b;
      tab[oGt + i * Q + q] = g;
      tab[oB2t + i * Q + q] = b * b;
    }
    for (int j = 0; j < L; ++j) {
      const double b = lagrange(zl.data(), L, j, xq[q]);
      tab[oBl + q * L + j] = b;
      tab[oBlt + j * Q + q] = b;
    }
    tab[oW + q] = wq[q];
    tab[oIW + q] = 1.0 / wq[q];
  }
  for (int i = 0; i < D; ++i) tab[oZ + i] = z[i];
}

}  // namespace lh
