// Host FP64 quadrature and Hermite tables for liblesbgk (see tables.h).
#include "tables.h"

#include <algorithm>
#include <cmath>

namespace lesbgk_tables {

void hermite_values(int mmax, double x, double *out) {
  out[0] = 1.0;
  if (mmax >= 1) out[1] = x;
  for (int m = 1; m < mmax; ++m) out[m + 1] = x * out[m] - m * out[m - 1];
}

// Cyclic Jacobi eigen-solver for a small dense symmetric matrix A (n x n,
// row-major, destroyed).  Eigenvalues land on the diagonal, eigenvectors in
// the columns of V.
static void jacobi_eigen(int n, double *A, double *V) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-60) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = cs * akp - sn * akq;
          A[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = cs * apk - sn * aqk;
          A[q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = cs * vkp - sn * vkq;
          V[k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
}

int gauss_hermite(int n, double *c, double *w) {
  if (n < 1 || n > kMaxRoots) return -1;
  double A[kMaxRoots * kMaxRoots] = {0}, V[kMaxRoots * kMaxRoots];
  // monic recurrence He_{k+1} = x He_k - k He_{k-1}: Jacobi off-diagonal sqrt(k)
  for (int k = 1; k < n; ++k) A[(k - 1) * n + k] = A[k * n + (k - 1)] = std::sqrt((double)k);
  jacobi_eigen(n, A, V);
  struct Node { double x, w; } nodes[kMaxRoots];
  for (int i = 0; i < n; ++i) nodes[i] = {A[i * n + i], V[0 * n + i] * V[0 * n + i]};
  std::sort(nodes, nodes + n, [](const Node &a, const Node &b) { return a.x < b.x; });
  double h[kMaxRoots + 2];
  for (int i = 0; i < n; ++i) {
    double x = nodes[i].x;
    for (int it = 0; it < 3; ++it) {  // Newton on He_n, He_n' = n He_{n-1}
      hermite_values(n, x, h);
      double d = n * h[n - 1];
      if (d != 0.0) x -= h[n] / d;
    }
    nodes[i].x = x;
  }
  for (int i = 0; i < n; ++i) {
    int j = n - 1 - i;
    c[i] = 0.5 * (nodes[i].x - nodes[j].x);
    w[i] = 0.5 * (nodes[i].w + nodes[j].w);
  }
  if (n % 2) c[n / 2] = 0.0;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += w[i];
  for (int i = 0; i < n; ++i) w[i] /= s;
  return 0;
}

void gaussian_hermite_moments(int order, double rho, double ux, double uy, double lxx, double lxy,
                              double lyy, double e[kMaxOrder + 1][kMaxOrder + 1]) {
  for (int m = 0; m <= kMaxOrder; ++m)
    for (int k = 0; k <= kMaxOrder; ++k) e[m][k] = 0.0;
  e[0][0] = rho;
  for (int n = 1; n <= order; ++n) {
    for (int m = 0; m <= n; ++m) {
      int k = n - m;
      if (m >= 1) {  // raise m from (m-1, k)
        double v = ux * e[m - 1][k];
        if (m >= 2) v += (m - 1) * lxx * e[m - 2][k];
        if (k >= 1) v += k * lxy * e[m - 1][k - 1];
        e[m][k] = v;
      } else {  // m = 0: raise k from (0, k-1)
        double v = uy * e[0][k - 1];
        if (k >= 2) v += (k - 1) * lyy * e[0][k - 2];
        e[0][k] = v;
      }
    }
  }
}

}  // namespace lesbgk_tables
