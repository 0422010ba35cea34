// Lowest eigenpair of the Lanczos tridiagonal matrix H_eff (App. B), fp64.
//
// Eigenvalue: bisection on the Sturm sequence count (the number of negative
// pivots of the LDL^T factorisation of T - x I equals the number of
// eigenvalues below x).  Eigenvector: inverse iteration with T - lambda I
// factorised by Gaussian elimination with partial pivoting.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mcd_internal.h"

namespace mcd {
namespace {

int count_below(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    const double bb = (i == 0) ? 0.0 : b[i] * b[i];
    q = (a[i] - x) - (i == 0 ? 0.0 : bb / q);
    if (q == 0.0) q = -1e-300;   // x is an eigenvalue: count it as below
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Solve (T - s I) x = r in place (x on entry = r), m >= 1, partial pivoting.
void solve_shifted(const double* a, const double* b, int m, double s, std::vector<double>& x) {
  // rows hold (d, du, du2) after elimination; dl eliminated.
  std::vector<double> d(m), du(m, 0.0), du2(m, 0.0), dl(m, 0.0);
  for (int i = 0; i < m; ++i) d[i] = a[i] - s;
  for (int i = 0; i + 1 < m; ++i) {
    du[i] = b[i + 1];
    dl[i] = b[i + 1];
  }
  std::vector<int> swapped(m, 0);
  std::vector<double> mult(m, 0.0);
  for (int i = 0; i + 1 < m; ++i) {
    if (std::fabs(d[i]) >= std::fabs(dl[i])) {
      double piv = d[i] != 0.0 ? d[i] : 1e-300;
      d[i] = piv;
      mult[i] = dl[i] / piv;
      d[i + 1] -= mult[i] * du[i];
      // du2[i] stays 0
    } else {
      // swap rows i and i+1
      swapped[i] = 1;
      const double f = d[i] / dl[i];
      mult[i] = f;
      d[i] = dl[i];
      const double tmp = d[i + 1];
      d[i + 1] = du[i] - f * tmp;
      du[i] = tmp;
      if (i + 2 < m) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du2[i];
      }
    }
  }
  if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
  // forward: apply L^{-1}
  for (int i = 0; i + 1 < m; ++i) {
    if (swapped[i]) {
      const double tmp = x[i];
      x[i] = x[i + 1];
      x[i + 1] = tmp - mult[i] * x[i];
    } else {
      x[i + 1] -= mult[i] * x[i];
    }
  }
  // back substitution with U (d, du, du2)
  x[m - 1] /= d[m - 1];
  if (m > 1) x[m - 2] = (x[m - 2] - du[m - 2] * x[m - 1]) / d[m - 2];
  for (int i = m - 3; i >= 0; --i) x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / d[i];
}

}  // namespace

double tridiag_lowest(const double* a, const double* b, int m, double* vec) {
  if (m <= 0) return 0.0;
  if (m == 1) {
    if (vec) vec[0] = 1.0;
    return a[0];
  }
  // Gershgorin bounds
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < m ? std::fabs(b[i + 1]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const double scale = std::max(std::fabs(lo), std::fabs(hi));
  for (int it = 0; it < 200 && (hi - lo) > 4e-16 * std::max(scale, 1e-300); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(a, b, m, mid) >= 1)
      hi = mid;
    else
      lo = mid;
  }
  const double lam = 0.5 * (lo + hi);
  if (vec) {
    std::vector<double> x(m, 1.0);
    for (int i = 0; i < m; ++i) x[i] = 1.0 + 0.01 * ((i * 7919) % 13);
    const double s = lam - 1e-13 * std::max(scale, 1.0);
    for (int rep = 0; rep < 3; ++rep) {
      solve_shifted(a, b, m, s, x);
      double nrm = 0.0;
      for (double v : x) nrm += v * v;
      nrm = std::sqrt(nrm);
      for (double& v : x) v /= nrm;
    }
    // fix sign: first nonzero component positive
    double sgn = 1.0;
    for (int i = 0; i < m; ++i)
      if (std::fabs(x[i]) > 1e-300) { sgn = x[i] > 0 ? 1.0 : -1.0; break; }
    for (int i = 0; i < m; ++i) vec[i] = sgn * x[i];
  }
  return lam;
}

}  // namespace mcd
