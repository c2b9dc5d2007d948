// Host-side FP64 set-up of the lattice tables (quadrature, Hermite values,
// Gaussian Hermite moments).  Used once per solver at creation.
#pragma once

namespace lesbgk_tables {

constexpr int kMaxRoots = 8;
constexpr int kMaxOrder = 4;

// n-point Gauss-Hermite rule for the unit Gaussian weight (Sec. 2.2): the
// abscissae are the roots of He_n, ascending; the weights sum to 1.
// Computed as the eigen-decomposition of the Jacobi matrix of the monic
// Hermite recurrence (Golub-Welsch), roots polished by Newton on He_n, and the
// pair symmetry c[n-1-i] = -c[i] imposed.  Returns 0, or -1 for n out of range.
int gauss_hermite(int n, double *c, double *w);

// He_m(x) for m = 0..mmax into out[0..mmax].
void hermite_values(int mmax, double x, double *out);

// Bivariate Hermite moments e[m][k] = rho E[He_m(X) He_k(Y)] of the Gaussian
// (X, Y) ~ N(u, I + Lam) for m + k <= order (Lam = lambda - I, symmetric,
// lam_xy = Lam[1]).  Generating function rho exp(u.t + t.Lam.t/2), i.e.
//   e[m+1][k] = u_x e[m][k] + m Lam_xx e[m-1][k] + k Lam_xy e[m][k-1]
//   e[m][k+1] = u_y e[m][k] + m Lam_xy e[m-1][k] + k Lam_yy e[m][k-1].
void gaussian_hermite_moments(int order, double rho, double ux, double uy, double lxx, double lxy,
                              double lyy, double e[kMaxOrder + 1][kMaxOrder + 1]);

}  // namespace lesbgk_tables
