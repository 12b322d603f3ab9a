// Host construction of the 1D tables of Sec. 3 (solution points, Lagrange
// basis, Radau g_DG correction derivatives) for the CUDA path.
#include <cmath>

#include "internal.cuh"

namespace frk {
namespace {

// Legendre P_n and P_n' at x from the Bonnet recurrence.
void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, dp0 = 0.0, dp1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    const double dp2 = dp0 + (2.0 * k - 1.0) * p1;  // P_k' = P_{k-2}' + (2k-1) P_{k-1}
    p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2;
  }
  *P = p1; *dP = dp1;
}

}  // namespace

void build_tables(int p, Tables* t) {
  const int n = p + 1;
  *t = Tables{};
  // Gauss-Legendre points: Newton on P_n from Chebyshev-like guesses.
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, x, &P, &dP);
      const double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double P, dP;
    legendre(n, x, &P, &dP);
    t->xi[i] = x;
    t->w[i] = 2.0 / ((1.0 - x * x) * dP * dP);
  }
  // barycentric weights of the Lagrange basis
  double bw[kMaxN];
  for (int k = 0; k < n; ++k) {
    double prod = 1.0;
    for (int j = 0; j < n; ++j)
      if (j != k) prod *= (t->xi[k] - t->xi[j]);
    bw[k] = 1.0 / prod;
  }
  // l_k(-1), l_k(+1)
  for (int k = 0; k < n; ++k) {
    double am = 1.0, ap = 1.0;
    for (int j = 0; j < n; ++j) {
      if (j == k) continue;
      am *= (-1.0 - t->xi[j]) / (t->xi[k] - t->xi[j]);
      ap *= (1.0 - t->xi[j]) / (t->xi[k] - t->xi[j]);
    }
    t->lm[k] = am;
    t->lp[k] = ap;
  }
  // derivative matrix D_ik = l_k'(xi_i): barycentric form, diagonal by row sums
  double D[kMaxN][kMaxN];
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      D[i][k] = (bw[k] / bw[i]) / (t->xi[i] - t->xi[k]);
      diag -= D[i][k];
    }
    D[i][i] = diag;
  }
  // Radau corrections: g_L = (-1)^n/2 (P_n - P_{n-1}), g_R = (P_n + P_{n-1})/2
  const double sgn = (n % 2 == 0) ? 1.0 : -1.0;
  for (int i = 0; i < n; ++i) {
    double Pa, dPa, Pb, dPb;
    legendre(n, t->xi[i], &Pa, &dPa);
    legendre(n - 1, t->xi[i], &Pb, &dPb);
    t->dgL[i] = 0.5 * sgn * (dPa - dPb);
    t->dgR[i] = 0.5 * (dPa + dPb);
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      t->D[i][k] = D[i][k];
      t->Dt[i][k] = D[i][k] - t->dgL[i] * t->lm[k] - t->dgR[i] * t->lp[k];
    }
}

}  // namespace frk
