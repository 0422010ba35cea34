// Dense symmetric eigenproblem of the band-Lanczos effective matrix H_eff
// (App. C: "we diagonalize these effective matrices"), fp64, host.
//
// Method (Golub & Van Loan, Matrix Computations, Sec. 8.3): Householder
// reduction to tridiagonal form A = Q T Q^T, then implicit symmetric QR steps
// with the Wilkinson shift on T, the Givens rotations applied to the rows of
// Q that are asked for.  Only the leading `rows` rows of the eigenvector
// matrix are formed: the Green function needs the eigenvectors' components on
// the first Krylov block only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mcd_internal.h"

namespace mcd {

int symeig_leading(int n, double* A, double* w, int rows, double* X) {
  if (n <= 0) return 0;
  rows = std::min(rows, n);
  // E = leading rows of Q, built as I[0:rows, :] * H_0 * H_1 * ...
  std::vector<double> E(size_t(rows) * n, 0.0);
  for (int i = 0; i < rows; ++i) E[size_t(i) * n + i] = 1.0;
  std::vector<double> v(n), p(n), q(n);
  auto a = [&](int i, int j) -> double& { return A[size_t(i) * n + j]; };
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;   // length of x = A[k+1.., k]
    double nx = 0.0;
    for (int i = 0; i < m; ++i) nx += a(k + 1 + i, k) * a(k + 1 + i, k);
    nx = std::sqrt(nx);
    if (nx == 0.0) continue;
    const double x0 = a(k + 1, k);
    const double alpha = x0 >= 0 ? -nx : nx;
    for (int i = 0; i < m; ++i) v[i] = a(k + 1 + i, k);
    v[0] -= alpha;
    double vv = 0.0;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // p = beta * B v, B = A[k+1.., k+1..]
    for (int i = 0; i < m; ++i) {
      const double* row = &a(k + 1 + i, k + 1);
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += row[j] * v[j];
      p[i] = beta * s;
    }
    double pv = 0.0;
    for (int i = 0; i < m; ++i) pv += p[i] * v[i];
    const double h = 0.5 * beta * pv;
    for (int i = 0; i < m; ++i) q[i] = p[i] - h * v[i];
    // B <- B - v q^T - q v^T  (= H B H with H = I - beta v v^T)
    for (int i = 0; i < m; ++i) {
      double* row = &a(k + 1 + i, k + 1);
      const double vi = v[i], qi = q[i];
      for (int j = 0; j < m; ++j) row[j] -= vi * q[j] + qi * v[j];
    }
    a(k + 1, k) = a(k, k + 1) = alpha;
    for (int i = 1; i < m; ++i) a(k + 1 + i, k) = a(k, k + 1 + i) = 0.0;
    // E <- E H
    for (int r = 0; r < rows; ++r) {
      double* er = &E[size_t(r) * n + k + 1];
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += er[i] * v[i];
      s *= beta;
      for (int i = 0; i < m; ++i) er[i] -= s * v[i];
    }
  }
  std::vector<double> d(n), e(std::max(n - 1, 1), 0.0);
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
  // implicit QR on (d, e); rotations applied to the columns of E
  const double eps = 2.220446049250313e-16;
  int hi = n - 1;
  long iter = 0;
  const long max_iter = 60L * n + 100;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    if (++iter > max_iter) return -1;
    // Wilkinson shift from the trailing 2x2 block
    const double dd = 0.5 * (d[hi - 1] - d[hi]);
    const double bb = e[hi - 1];
    const double den = dd + std::copysign(std::hypot(dd, bb), dd == 0.0 ? 1.0 : dd);
    const double mu = d[hi] - bb * bb / den;
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      double r = std::hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = z / r;
      }
      if (k > lo) e[k - 1] = r;
      const double ak = d[k], ak1 = d[k + 1], bk = e[k];
      d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      d[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      if (k + 1 < hi) {
        z = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      for (int rr = 0; rr < rows; ++rr) {
        double* er = &E[size_t(rr) * n];
        const double u0 = er[k], u1 = er[k + 1];
        er[k] = c * u0 + s * u1;
        er[k + 1] = -s * u0 + c * u1;
      }
    }
  }
  // ascending order
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int i, int j) { return d[i] < d[j]; });
  for (int i = 0; i < n; ++i) w[i] = d[ord[i]];
  if (X)
    for (int r = 0; r < rows; ++r)
      for (int i = 0; i < n; ++i) X[size_t(r) * n + i] = E[size_t(r) * n + ord[i]];
  return 0;
}

}  // namespace mcd
