/*
 * lesbgk_oracle.c -- plain FP64 CPU oracle for the lattice ES-BGK time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline in bench.py load this file's library.  The product (the CUDA
 * library under paper_1209_6548_gb300/csrc) never links, calls or includes it,
 * and this file includes nothing from the product.
 *
 * What it computes, each function citing the passage it follows (Meng, Zhang,
 * Hadjiconstantinou, Radtke & Shan, "Lattice ellipsoidal statistical BGK model
 * for thermal non-equilibrium flows", arXiv 1209.6548):
 *
 *   - 1D Gauss-Hermite abscissae = roots of He_n, weights by Eq. (weight)
 *     w = n!/[n He_{n-1}(c)]^2, and the D-dimensional tensor-product set
 *     (Sec. 2.2), D = 2 or 3.
 *   - Tensor Hermite polynomials chi^(n)_{i1..in}, n <= 4, in full index form
 *     (the basis of Eq. approxf; Grad's definitions), indices 0..D-1.
 *   - Moments rho, u, P_ij, T, sigma_ij, q_i of Eq. (mac) in D dimensions.
 *   - tau = (Kn/Pr) mu/p, mu = T^varpi, p = rho T, Pr = 1/(1-b) (Sec. 2.1-2.2).
 *   - lambda_ij = T delta_ij + b sigma_ij / rho (Eq. cfeq).
 *   - a_ES^(0..4) as printed in Sec. 2.2 and f_ES,a = w_a sum_n a:chi/n!.
 *   - Body force F = omega sum_{n=1}^{N} g a^(n-1):chi^(n)/(n-1)! (Sec. 2.2),
 *     with a^(k) the distribution's own Hermite moments.
 *   - Forward Euler + second-order TVD/minmod fluxes (Sec. 3.1), as printed
 *     (both flux differences from f^n), or dimensionally split (y-sweep then
 *     x-sweep) for flows that vary in both x and y.
 *   - Truncated Maxwellian S(T,u), Eq. (feq0), and the diffuse wall of
 *     Sec. 3.2 (outgoing half = rho_W S, ghosts = wall node).
 *
 * Walls in x (a cavity; not in the paper, whose flows are all uniform in x):
 * fully diffuse walls at rest on columns i = 0 and nx-1, treated like the
 * y-walls; a node on both a y-wall and an x-wall (a corner) follows the
 * corner rule of wall_corner().
 *
 * Readings where the paper is silent (each restated where it is used):
 *   D is the dimension of the velocity set, used in T, Eq. (feq0) and the chi
 *   traces (the paper's runs take D = 3 without naming their set; the 2D sets
 *   give D = 2); the grid is two-dimensional whatever D is: populations are
 *   advected along x and y only (nothing varies in z);
 *   for c < 0 the flux is the mirror image of the printed c > 0 formula;
 *   Psi(Theta)*(f_{i+1}-f_i) is 0 when f_{i+1} = f_i (Psi is bounded);
 *   walls sit on nodes j = 0 and j = ny-1; the wall node is first updated like
 *   any node, then rho_W is formed from its updated incoming half and its
 *   outgoing half is replaced; S carries the same order N as f_ES.
 *
 * Everything is double precision and written for a reader to check against
 * the paper by eye: no blocking, no fusion, no product-basis factorisation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 3       /* largest velocity-set dimension */
#define ORC_MAXR 64      /* largest 1D rule the root finder is asked for */
#define ORC_MAXQ 216     /* largest velocity set the step handles (6^3) */
#define ORC_MAXN 4       /* highest Hermite order */
#define ORC_MAXT 81      /* components of a rank-4 tensor in D = 3 */

typedef struct orc_params {
  int32_t nroots;   /* roots of He_nroots per axis: Q = nroots^2 */
  int32_t order;    /* Hermite truncation order N (0..4) */
  int32_t nx, ny;   /* nodes in x (periodic) and y */
  int32_t bc_y;     /* 0 = periodic in y, 1 = diffuse walls on j=0, j=ny-1 */
  int32_t scheme;   /* 0 = the update of Sec. 3.1 as printed (both flux
                       differences from f^n); 1 = split: a y-sweep, then an
                       x-sweep of the y-swept values (reading for 2D flows) */
  int32_t dim;      /* velocity-set dimension D: 2 (Q = nroots^2) or 3
                       (Q = nroots^3); 0 means 2 */
  int32_t bc_x;     /* 0 = periodic in x, 1 = diffuse walls at rest on i=0, i=nx-1 */
  double kn;        /* Kn of Sec. 2.2 */
  double b;         /* ES parameter, Pr = 1/(1-b) */
  double visc_exp;  /* varpi in mu = T^varpi */
  double dt, dx, dy;
  double wall_T[2];   /* [0] bottom (j=0), [1] top (j=ny-1) */
  double wall_ux[2];
  double g[2];        /* body force (g_x, g_y); g_z = 0 */
  double wall_specular; /* 1 - gamma of the Maxwell wall model (Sec. 3.2); 0 = fully diffuse */
  double wall_T_amp;    /* wall temperature T_w(t) = wall_T + amp sin(freq t) (Sec. 4.2) */
  double wall_T_freq;
  double time;          /* time of the state handed to orc_init / orc_step / orc_run */
  double wall_Tx[2];    /* x-wall temperatures, [0] left (i=0), [1] right (i=nx-1) */
} orc_params;

static int orc_threads = 1;
void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return orc_threads; }

/* ------------------------------------------------------------------ */
/* 1D probabilists' Hermite polynomial He_n(x) by the three-term       */
/* recurrence He_{k+1} = x He_k - k He_{k-1}.                          */
/* ------------------------------------------------------------------ */
double orc_hermite_he(int n, double x) {
  if (n == 0) return 1.0;
  double hm1 = 1.0, h = x;
  for (int k = 1; k < n; ++k) {
    double hp1 = x * h - (double)k * hm1;
    hm1 = h;
    h = hp1;
  }
  return h;
}

/* Roots of He_n by sign-change scan + bisection; weights by Eq. (weight):
 * w = n! / [n He_{n-1}(c)]^2.  Abscissae ascending.  Returns 0 or -1. */
int orc_gauss_hermite_1d(int n, double *c, double *w) {
  if (n < 1 || n > ORC_MAXR) return -1;
  double lim = 2.0 * sqrt((double)n) + 2.0;
  int found = 0;
  double step = 1e-3;
  double x0 = -lim, f0 = orc_hermite_he(n, x0);
  while (x0 < lim && found < n) {
    double x1 = x0 + step, f1 = orc_hermite_he(n, x1);
    if (f1 == 0.0) {
      c[found++] = x1;
      x0 = x1 + step * 0.5;
      f0 = orc_hermite_he(n, x0);
      continue;
    }
    if ((f0 < 0.0) != (f1 < 0.0)) {
      double lo = x0, hi = x1, flo = f0;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double fm = orc_hermite_he(n, mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      c[found++] = 0.5 * (lo + hi);
    }
    x0 = x1;
    f0 = f1;
  }
  if (found != n) return -1;
  double nfact = 1.0;
  for (int k = 2; k <= n; ++k) nfact *= (double)k;
  for (int a = 0; a < n; ++a) {
    double h = (double)n * orc_hermite_he(n - 1, c[a]);
    w[a] = nfact / (h * h);
  }
  return 0;
}

/* D-dimensional tensor-product ("production") set, Sec. 2.2:
 *   D = 2: alpha = ix*nroots + iy,            c = (c_ix, c_iy)
 *   D = 3: alpha = (ix*nroots + iy)*nroots + iz, c = (c_ix, c_iy, c_iz)
 * w_alpha = product of the 1D weights.  cz may be NULL for D = 2. */
int orc_velocity_set_d(int nroots, int D, double *cx, double *cy, double *cz, double *w) {
  double c1[ORC_MAXR], w1[ORC_MAXR];
  if ((D != 2 && D != 3) || orc_gauss_hermite_1d(nroots, c1, w1)) return -1;
  int nz = D == 3 ? nroots : 1;
  for (int ix = 0; ix < nroots; ++ix)
    for (int iy = 0; iy < nroots; ++iy)
      for (int iz = 0; iz < nz; ++iz) {
        int a = (ix * nroots + iy) * nz + iz;
        cx[a] = c1[ix];
        cy[a] = c1[iy];
        if (cz) cz[a] = D == 3 ? c1[iz] : 0.0;
        w[a] = w1[ix] * w1[iy] * (D == 3 ? w1[iz] : 1.0);
      }
  return 0;
}

int orc_velocity_set(int nroots, double *cx, double *cy, double *w) {
  return orc_velocity_set_d(nroots, 2, cx, cy, NULL, w);
}

/* ------------------------------------------------------------------ */
/* Tensor Hermite polynomials in D dimensions, full index form.        */
/* A rank-n tensor is stored flat with index sum_k i_k D^(n-1-k).       */
/*   chi0 = 1                                                           */
/*   chi1_i = c_i                                                       */
/*   chi2_ij = c_i c_j - d_ij                                           */
/*   chi3_ijk = c_i c_j c_k - (c_i d_jk + c_j d_ik + c_k d_ij)          */
/*   chi4_ijkl = c_i c_j c_k c_l - (six c c d terms) + (three d d terms) */
/* ------------------------------------------------------------------ */
static double dl(int i, int j) { return i == j ? 1.0 : 0.0; }

static int rank_size(int D, int n) {
  int r = 1;
  for (int k = 0; k < n; ++k) r *= D;
  return r;
}

static void idx_of(int D, int n, int flat, int *ix) {
  for (int k = n - 1; k >= 0; --k) {
    ix[k] = flat % D;
    flat /= D;
  }
}

void orc_chi_d(int n, int D, const double *c, double *out) {
  int sz = rank_size(D, n);
  for (int f = 0; f < sz; ++f) {
    int I[4];
    idx_of(D, n, f, I);
    double v = 0.0;
    if (n == 0) {
      v = 1.0;
    } else if (n == 1) {
      v = c[I[0]];
    } else if (n == 2) {
      v = c[I[0]] * c[I[1]] - dl(I[0], I[1]);
    } else if (n == 3) {
      int i = I[0], j = I[1], k = I[2];
      v = c[i] * c[j] * c[k] - (c[i] * dl(j, k) + c[j] * dl(i, k) + c[k] * dl(i, j));
    } else if (n == 4) {
      int i = I[0], j = I[1], k = I[2], l = I[3];
      v = c[i] * c[j] * c[k] * c[l]
          - (c[i] * c[j] * dl(k, l) + c[i] * c[k] * dl(j, l) + c[i] * c[l] * dl(j, k)
             + c[j] * c[k] * dl(i, l) + c[j] * c[l] * dl(i, k) + c[k] * c[l] * dl(i, j))
          + (dl(i, j) * dl(k, l) + dl(i, k) * dl(j, l) + dl(i, l) * dl(j, k));
    }
    out[f] = v;
  }
}

void orc_chi(int n, const double *c, double *out) { orc_chi_d(n, 2, c, out); }

/* ------------------------------------------------------------------ */
/* a_ES^(n), Sec. 2.2, exactly as printed (index loops over 0..D-1).   */
/* lam is the D x D ES tensor, row-major.                              */
/* ------------------------------------------------------------------ */
void orc_a_es_d(int n, int D, double rho, const double *u, const double *lam, double *out) {
  int sz = rank_size(D, n);
#define L(p, q) (lam[(p) * D + (q)])
#define LM(p, q) (L(p, q) - dl(p, q))
  for (int f = 0; f < sz; ++f) {
    int I[4];
    idx_of(D, n, f, I);
    double v = 0.0;
    if (n == 0) {
      v = rho;
    } else if (n == 1) {
      v = rho * u[I[0]];
    } else if (n == 2) {
      int i = I[0], j = I[1];
      v = rho * (u[i] * u[j] + L(i, j) - dl(i, j));
    } else if (n == 3) {
      int i = I[0], j = I[1], k = I[2];
      v = rho * (u[i] * u[j] * u[k] + L(i, j) * u[k] + L(i, k) * u[j] + L(j, k) * u[i]
                 - dl(i, j) * u[k] - dl(i, k) * u[j] - dl(j, k) * u[i]);
    } else if (n == 4) {
      int i = I[0], j = I[1], k = I[2], l = I[3];
      v = rho * (u[i] * u[j] * u[l] * u[k]
                 + LM(i, l) * u[j] * u[k] + LM(i, j) * u[l] * u[k] + LM(i, k) * u[j] * u[l]
                 + LM(j, l) * u[i] * u[k] + LM(j, k) * u[i] * u[l] + LM(k, l) * u[i] * u[j]
                 + LM(i, j) * LM(k, l) + LM(i, k) * LM(j, l) + LM(i, l) * LM(k, j));
    }
    out[f] = v;
  }
#undef L
#undef LM
}

void orc_a_es(int n, double rho, const double *u, const double *lam, double *out) {
  orc_a_es_d(n, 2, rho, u, lam, out);
}

static double factorial(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= (double)k;
  return r;
}

/* Full contraction a:chi of two rank-n tensors. */
static double contract(int D, int n, const double *a, const double *chi) {
  double s = 0.0;
  for (int f = 0; f < rank_size(D, n); ++f) s += a[f] * chi[f];
  return s;
}

/* Velocity-set tables shared by one call: c, w and chi^(n)(c_alpha). */
typedef struct orc_lattice {
  int Q, nroots, D;
  double c[ORC_MAXQ][ORC_MAXD];  /* c[alpha][i], i < D; components i >= D are 0 */
  double w[ORC_MAXQ];
  double chi[ORC_MAXN + 1][ORC_MAXQ][ORC_MAXT];
} orc_lattice;

static int dim_of(const orc_params *p) { return p->dim == 0 ? 2 : p->dim; }

/* Heap-allocated (the chi tables take 0.7 MB for D3Q216); free() it. */
static orc_lattice *lattice_new(int nroots, int D) {
  if (nroots < 1 || (D != 2 && D != 3)) return NULL;
  int Q = D == 3 ? nroots * nroots * nroots : nroots * nroots;
  if (Q > ORC_MAXQ) return NULL;
  orc_lattice *L = (orc_lattice *)calloc(1, sizeof(orc_lattice));
  if (!L) return NULL;
  L->nroots = nroots;
  L->D = D;
  L->Q = Q;
  double cx[ORC_MAXQ], cy[ORC_MAXQ], cz[ORC_MAXQ];
  if (orc_velocity_set_d(nroots, D, cx, cy, cz, L->w)) {
    free(L);
    return NULL;
  }
  for (int a = 0; a < Q; ++a) {
    L->c[a][0] = cx[a];
    L->c[a][1] = cy[a];
    L->c[a][2] = cz[a];
    for (int n = 0; n <= ORC_MAXN; ++n) orc_chi_d(n, D, L->c[a], L->chi[n][a]);
  }
  return L;
}

/* alpha with c_y -> -c_y (the specular image across a wall normal to y) */
static int mirror_y(const orc_lattice *L, int a) {
  int nr = L->nroots, nz = L->D == 3 ? nr : 1;
  int iz = a % nz, iy = (a / nz) % nr, ix = a / (nz * nr);
  return (ix * nr + (nr - 1 - iy)) * nz + iz;
}

/* ------------------------------------------------------------------ */
/* Moments of Eq. (mac) in D dimensions.                               */
/* out: rho, ux, uy, T, sxx, sxy, syy, qx, qy                           */
/* P_ij = sum f C_i C_j;  T = P_ii/(D rho);  sigma = P - delta P_ii/D;  */
/* q_i = 1/2 sum f C_i C^2 (C^2 over all D components).  For D = 3 the  */
/* z components (u_z, sigma_iz, q_z) are left out of out; Pout gets     */
/* the whole D x D tensor and uout (if set) the D velocity components.  */
/* ------------------------------------------------------------------ */
static void cell_moments(const orc_lattice *L, const double *f, double *out, double *Pout, double *uout) {
  const int D = L->D;
  double rho = 0.0, m[ORC_MAXD] = {0.0, 0.0, 0.0};
  for (int a = 0; a < L->Q; ++a) {
    rho += f[a];
    for (int i = 0; i < D; ++i) m[i] += f[a] * L->c[a][i];
  }
  double u[ORC_MAXD] = {0.0, 0.0, 0.0};
  for (int i = 0; i < D; ++i) u[i] = m[i] / rho;
  double P[ORC_MAXD * ORC_MAXD] = {0.0}, q[ORC_MAXD] = {0.0, 0.0, 0.0};
  for (int a = 0; a < L->Q; ++a) {
    double C[ORC_MAXD], C2 = 0.0;
    for (int i = 0; i < D; ++i) {
      C[i] = L->c[a][i] - u[i];
      C2 += C[i] * C[i];
    }
    for (int i = 0; i < D; ++i) {
      for (int j = 0; j < D; ++j) P[i * D + j] += f[a] * C[i] * C[j];
      q[i] += 0.5 * f[a] * C[i] * C2;
    }
  }
  double trP = 0.0;
  for (int i = 0; i < D; ++i) trP += P[i * D + i];
  double T = trP / (D * rho);
  double tr = trP / D;
  out[0] = rho; out[1] = u[0]; out[2] = u[1]; out[3] = T;
  out[4] = P[0] - tr; out[5] = P[1]; out[6] = P[D + 1] - tr;
  out[7] = q[0]; out[8] = q[1];
  if (Pout)
    for (int k = 0; k < D * D; ++k) Pout[k] = P[k];
  if (uout)
    for (int i = 0; i < D; ++i) uout[i] = u[i];
}

/* ------------------------------------------------------------------ */
/* Per-cell collision ingredients:                                     */
/*   f_ES,a = w_a sum_{n<=N} a_ES^(n):chi^(n)(c_a)/n!                   */
/*   g_a    = w_a sum_{n=1..N} g a^(n-1):chi^(n)(c_a)/(n-1)!            */
/*   tau    = (Kn/Pr) mu/p                                              */
/* ------------------------------------------------------------------ */
static void cell_collision(const orc_lattice *L, const orc_params *p, const double *f,
                           double *fes, double *gf, double *tau_out) {
  const int D = L->D;
  double m[9], P[ORC_MAXD * ORC_MAXD], u[ORC_MAXD];
  cell_moments(L, f, m, P, u);
  double rho = m[0], T = m[3];
  /* lambda = T delta + b sigma / rho, sigma = P - delta tr(P)/D (Eq. cfeq, Eq. mac) */
  double trP = 0.0;
  for (int i = 0; i < D; ++i) trP += P[i * D + i];
  double lam[ORC_MAXD * ORC_MAXD];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double sig = P[i * D + j] - dl(i, j) * trP / D;
      lam[i * D + j] = T * dl(i, j) + p->b * sig / rho;
    }
  int N = p->order;
  double aes[ORC_MAXN + 1][ORC_MAXT];
  for (int n = 0; n <= N; ++n) orc_a_es_d(n, D, rho, u, lam, aes[n]);
  /* the distribution's own Hermite moments a^(k) = sum_b f_b chi^(k)(c_b) */
  double af[ORC_MAXN + 1][ORC_MAXT];
  for (int n = 0; n < N; ++n) {
    for (int k = 0; k < rank_size(D, n); ++k) {
      double s = 0.0;
      for (int b = 0; b < L->Q; ++b) s += f[b] * L->chi[n][b][k];
      af[n][k] = s;
    }
  }
  double g[ORC_MAXD] = {p->g[0], p->g[1], 0.0};
  for (int a = 0; a < L->Q; ++a) {
    double s = 0.0;
    for (int n = 0; n <= N; ++n) s += contract(D, n, aes[n], L->chi[n][a]) / factorial(n);
    fes[a] = L->w[a] * s;
    double gs = 0.0;
    for (int n = 1; n <= N; ++n) {
      /* g_{i1} a^(n-1)_{i2..in} chi^(n)_{i1 i2..in} */
      double t = 0.0;
      int szm = rank_size(D, n - 1);
      for (int i1 = 0; i1 < D; ++i1)
        for (int r = 0; r < szm; ++r) t += g[i1] * af[n - 1][r] * L->chi[n][a][i1 * szm + r];
      gs += t / factorial(n - 1);
    }
    gf[a] = L->w[a] * gs;
  }
  double Pr = 1.0 / (1.0 - p->b);
  double mu = pow(T, p->visc_exp);
  double pr = rho * T;
  *tau_out = (p->kn / Pr) * mu / pr;
}

/* Exported for the tests: f_ES, g_a and tau of one cell. */
int orc_cell_terms(const orc_params *p, const double *f, double *fes, double *gf, double *tau) {
  orc_lattice *L = lattice_new(p->nroots, dim_of(p));
  if (!L) return -1;
  cell_collision(L, p, f, fes, gf, tau);
  free(L);
  return 0;
}

/* Exported for the tests: the moments of one cell in D dimensions:
 * out9 as in orc_moments, P (D x D), u (D). */
int orc_cell_moments(int nroots, int D, const double *f, double *out9, double *P, double *u) {
  orc_lattice *L = lattice_new(nroots, D);
  if (!L) return -1;
  cell_moments(L, f, out9, P, u);
  free(L);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Truncated Maxwellian S(T,u), Eq. (feq0), carried to order N <= 4,   */
/* in D dimensions (c.u, u.u and c.c over all D components).           */
/* Lines of Eq. (feq0): orders 0,1,2 | order 3 | order 4 (three lines). */
/* ------------------------------------------------------------------ */
static double feq0_S(int N, int D, double T, const double *u, const double *c, double w) {
  double cu = 0.0, uu = 0.0, cc = 0.0;
  for (int i = 0; i < D; ++i) {
    cu += c[i] * u[i];
    uu += u[i] * u[i];
    cc += c[i] * c[i];
  }
  double th = T - 1.0;
  double s = 1.0;
  if (N >= 1) s += cu;
  if (N >= 2) s += 0.5 * (cu * cu - uu + th * (cc - D));
  if (N >= 3) s += cu / 6.0 * (cu * cu - 3.0 * uu + 3.0 * th * (cc - D - 2.0));
  if (N >= 4) {
    s += (cu * cu * cu * cu - 6.0 * cu * cu * uu + 3.0 * uu * uu) / 24.0;
    s += th / 4.0 * ((cc - D - 2.0) * (cu * cu - uu) - 2.0 * cu * cu);
    s += th * th / 8.0 * (cc * cc - 2.0 * (D + 2.0) * cc + D * (D + 2.0));
  }
  return w * s;
}

int orc_feq0_d(int nroots, int D, int N, double T, double ux, double uy, double *out) {
  orc_lattice *L = lattice_new(nroots, D);
  if (!L) return -1;
  double u[ORC_MAXD] = {ux, uy, 0.0};
  for (int a = 0; a < L->Q; ++a) out[a] = feq0_S(N, D, T, u, L->c[a], L->w[a]);
  free(L);
  return 0;
}

int orc_feq0(int nroots, int N, double T, double ux, double uy, double *out) {
  return orc_feq0_d(nroots, 2, N, T, ux, uy, out);
}

/* ------------------------------------------------------------------ */
/* TVD interface flux of Sec. 3.1 for one velocity along one axis.     */
/* fm2..fp2 = f at i-2..i+2; nu = |c| dt / delta.                       */
/* Returns F_{i+1/2} - F_{i-1/2}.                                       */
/* ------------------------------------------------------------------ */
static double limited(double num, double den) {
  /* [f_{i+1}-f_i] Psi(Theta), Theta = num/den, Psi = max(0, min(1, Theta)).
   * Reading: when den = 0 the product is 0 (Psi is bounded). */
  if (den == 0.0) return 0.0;
  double th = num / den;
  double psi = fmax(0.0, fmin(1.0, th));
  return den * psi;
}

static double flux_difference(double c, double nu, double fm2, double fm1, double f0, double fp1,
                              double fp2) {
  double k = 0.5 * (1.0 - nu);
  double Fp, Fm;
  if (c > 0.0) {
    /* F_{i+1/2} = f_i + k [f_{i+1}-f_i] Psi((f_i - f_{i-1})/(f_{i+1}-f_i)) */
    Fp = f0 + k * limited(f0 - fm1, fp1 - f0);
    /* F_{i-1/2} = F_{(i-1)+1/2} */
    Fm = fm1 + k * limited(fm1 - fm2, f0 - fm1);
  } else {
    /* mirror image (reading): upwind node is i+1 */
    Fp = fp1 + k * limited(fp1 - fp2, f0 - fp1);
    Fm = f0 + k * limited(f0 - fp1, fm1 - f0);
  }
  return Fp - Fm;
}

/* Exported for the tests: one velocity, periodic 1D line. */
int orc_advect_1d(int n, double c, double nu, const double *f, double *diff) {
  for (int i = 0; i < n; ++i) {
#define AT(k) f[(((i) + (k)) % n + n) % n]
    diff[i] = flux_difference(c, nu, AT(-2), AT(-1), AT(0), AT(1), AT(2));
#undef AT
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Grid helpers.  Layout: f[alpha][j][i] (alpha-major, then row j,      */
/* then column i).                                                      */
/* ------------------------------------------------------------------ */
static size_t fidx(const orc_params *p, int a, int j, int i) {
  return ((size_t)a * p->ny + (size_t)j) * p->nx + (size_t)i;
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Column index of neighbour i+di: periodic wrap, or ghosts = wall node. */
static int col_of(const orc_params *p, int i) {
  if (p->bc_x == 0) return wrap(i, p->nx);
  if (i < 0) return 0;
  if (i >= p->nx) return p->nx - 1;
  return i;
}

/* Row index of neighbour j+dj: periodic wrap, or ghosts = wall node. */
static int row_of(const orc_params *p, int j) {
  if (p->bc_y == 0) return wrap(j, p->ny);
  if (j < 0) return 0;
  if (j >= p->ny) return p->ny - 1;
  return j;
}

/* Wall of Sec. 3.2 at wall node (i, j) at time t: the Maxwell model with
 * accommodation gamma = 1 - wall_specular.  The diffusely re-emitted part is
 * rho_W S(T_w(t), u_w) with rho_W = sum_{c.n<0} |c.n| f / sum_{c.n>0} |c.n| S
 * (zero net normal mass flux); the specular part is the incoming population
 * with the mirrored normal velocity.  T_w(t) = wall_T + amp sin(freq t), the
 * heating of Sec. 4.2.  With wall_specular = 0 and amp = 0 this is the fully
 * diffuse wall the paper implements. */
static void wall_node(const orc_lattice *L, const orc_params *p, double *f, int i, int j, int side,
                      double t) {
  double n_y = side == 0 ? 1.0 : -1.0;
  double u[ORC_MAXD] = {p->wall_ux[side], 0.0, 0.0};
  double Tw = p->wall_T[side] + p->wall_T_amp * sin(p->wall_T_freq * t);
  double S[ORC_MAXQ];
  for (int a = 0; a < L->Q; ++a) S[a] = feq0_S(p->order, L->D, Tw, u, L->c[a], L->w[a]);
  double num = 0.0, den = 0.0;
  for (int a = 0; a < L->Q; ++a) {
    double cn = L->c[a][1] * n_y;
    if (cn < 0.0) num += fabs(cn) * f[fidx(p, a, j, i)];
    if (cn > 0.0) den += fabs(cn) * S[a];
  }
  double rw = num / den;
  double spec = p->wall_specular;
  for (int a = 0; a < L->Q; ++a) {
    if (L->c[a][1] * n_y > 0.0) {
      int mirror = mirror_y(L, a); /* c_y -> -c_y */
      f[fidx(p, a, j, i)] = (1.0 - spec) * rw * S[a] + spec * f[fidx(p, mirror, j, i)];
    }
  }
}

/* Diffuse wall at rest normal to x at node (i, j): side 0 = left wall
 * (i = 0, normal +x), side 1 = right wall (i = nx-1, normal -x); the rule of
 * wall_node with c_x in place of c_y and S(T_wx, u = 0). */
static void wall_node_x(const orc_lattice *L, const orc_params *p, double *f, int i, int j, int side) {
  double n_x = side == 0 ? 1.0 : -1.0;
  double u[ORC_MAXD] = {0.0, 0.0, 0.0};
  double S[ORC_MAXQ];
  for (int a = 0; a < L->Q; ++a) S[a] = feq0_S(p->order, L->D, p->wall_Tx[side], u, L->c[a], L->w[a]);
  double num = 0.0, den = 0.0;
  for (int a = 0; a < L->Q; ++a) {
    double cn = L->c[a][0] * n_x;
    if (cn < 0.0) num += fabs(cn) * f[fidx(p, a, j, i)];
    if (cn > 0.0) den += fabs(cn) * S[a];
  }
  double rw = num / den;
  for (int a = 0; a < L->Q; ++a)
    if (L->c[a][0] * n_x > 0.0) f[fidx(p, a, j, i)] = rw * S[a];
}

/* Corner node (i, j) on the x-wall `xside` and the y-wall `yside` (a reading;
 * the paper has no corners).  The node belongs to both walls: populations
 * moving away from either wall (c.n_x > 0 or c.n_y > 0, n_x and n_y the
 * inward normals) are re-emitted as rho_W S(T_wx, u = 0) -- the side wall's,
 * so a moving lid stops short of the corners -- and the others, arriving
 * from the interior towards both walls, are kept.  rho_W makes the net mass
 * flux along n = n_x + n_y zero; with the wall at rest sum_a (c.n) S_a = 0,
 * so rho_W = sum_in |c.n| f / sum_in |c.n| S over the kept populations. */
static void wall_corner(const orc_lattice *L, const orc_params *p, double *f, int i, int j, int xside,
                        int yside) {
  double n_x = xside == 0 ? 1.0 : -1.0, n_y = yside == 0 ? 1.0 : -1.0;
  double u[ORC_MAXD] = {0.0, 0.0, 0.0};
  double S[ORC_MAXQ];
  for (int a = 0; a < L->Q; ++a) S[a] = feq0_S(p->order, L->D, p->wall_Tx[xside], u, L->c[a], L->w[a]);
  double num = 0.0, den = 0.0;
  for (int a = 0; a < L->Q; ++a) {
    int kept = L->c[a][0] * n_x < 0.0 && L->c[a][1] * n_y < 0.0;
    double cn = fabs(L->c[a][0] * n_x + L->c[a][1] * n_y);
    if (kept) {
      num += cn * f[fidx(p, a, j, i)];
      den += cn * S[a];
    }
  }
  double rw = num / den;
  for (int a = 0; a < L->Q; ++a) {
    int kept = L->c[a][0] * n_x < 0.0 && L->c[a][1] * n_y < 0.0;
    if (!kept) f[fidx(p, a, j, i)] = rw * S[a];
  }
}

static void apply_walls(const orc_lattice *L, const orc_params *p, double *f, double t) {
  int xw = p->bc_x == 1, yw = p->bc_y == 1;
  if (yw)
    for (int i = xw ? 1 : 0; i < p->nx - (xw ? 1 : 0); ++i) {
      wall_node(L, p, f, i, 0, 0, t);
      wall_node(L, p, f, i, p->ny - 1, 1, t);
    }
  if (xw)
    for (int j = yw ? 1 : 0; j < p->ny - (yw ? 1 : 0); ++j) {
      wall_node_x(L, p, f, 0, j, 0);
      wall_node_x(L, p, f, p->nx - 1, j, 1);
    }
  if (xw && yw) {
    wall_corner(L, p, f, 0, 0, 0, 0);
    wall_corner(L, p, f, p->nx - 1, 0, 1, 0);
    wall_corner(L, p, f, 0, p->ny - 1, 0, 1);
    wall_corner(L, p, f, p->nx - 1, p->ny - 1, 1, 1);
  }
}

static int check_params(const orc_params *p) {
  int D = dim_of(p);
  if (D != 2 && D != 3) return -1;
  if (p->nroots < 2 || (D == 3 ? p->nroots * p->nroots * p->nroots : p->nroots * p->nroots) > ORC_MAXQ) return -1;
  if (p->order < 0 || p->order > ORC_MAXN) return -1;
  if (p->nx < 1 || p->ny < 1) return -1;
  if (p->bc_y == 1 && p->ny < 2) return -1;
  if (p->bc_x != 0 && p->bc_x != 1) return -1;
  if (p->bc_x == 1 && p->nx < 2) return -1;
  if (p->scheme != 0 && p->scheme != 1) return -1;
  if (!(p->wall_specular >= 0.0 && p->wall_specular <= 1.0)) return -1;
  return 0;
}

/* Initial state: f = rho S(T,u) from fields[4][ny][nx] = rho, ux, uy, T;
 * then the wall rule once so the state satisfies the boundary condition. */
int orc_init(const orc_params *p, const double *fields, double *f) {
  if (check_params(p)) return -1;
  orc_lattice *L = lattice_new(p->nroots, dim_of(p));
  if (!L) return -1;
  size_t cells = (size_t)p->nx * p->ny;
  for (int j = 0; j < p->ny; ++j)
    for (int i = 0; i < p->nx; ++i) {
      size_t c = (size_t)j * p->nx + i;
      double rho = fields ? fields[c] : 1.0;
      double u[ORC_MAXD] = {fields ? fields[cells + c] : 0.0, fields ? fields[2 * cells + c] : 0.0, 0.0};
      double T = fields ? fields[3 * cells + c] : 1.0;
      for (int a = 0; a < L->Q; ++a)
        f[fidx(p, a, j, i)] = rho * feq0_S(p->order, L->D, T, u, L->c[a], L->w[a]);
    }
  apply_walls(L, p, f, p->time);
  free(L);
  return 0;
}

/* One time step n -> n+1 of the scheme in Sec. 3.1 followed by the walls of
 * Sec. 3.2.  f_in and f_out must not alias.
 *
 * scheme 0 is the printed update: both flux differences are taken from f^n.
 * scheme 1 (a reading, for flows that vary in x and y, where the printed
 * unsplit sum of two one-dimensional second-order fluxes has an amplification
 * factor above 1): first the y-sweep f* = f^n - (c_y dt/dy) dF_y(f^n), then
 * the x-sweep of f*; collision and force are evaluated from f^n as printed.
 * For fields that do not vary in x both schemes give the same update. */
int orc_step(const orc_params *p, const double *fin, double *fout) {
  if (check_params(p)) return -1;
  orc_lattice *Lp = lattice_new(p->nroots, dim_of(p));
  if (!Lp) return -1;
  const orc_lattice *L = Lp;
  const int Q = L->Q;
  const size_t n = (size_t)Q * p->nx * p->ny;
  double *fstar = NULL;
  if (p->scheme == 1) {
    fstar = (double *)malloc(n * sizeof(double));
    if (!fstar) {
      free(Lp);
      return -1;
    }
#pragma omp parallel for schedule(static) num_threads(orc_threads)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i)
        for (int a = 0; a < Q; ++a) {
          double cy = L->c[a][1], fy[5];
          for (int k = -2; k <= 2; ++k) fy[k + 2] = fin[fidx(p, a, row_of(p, j + k), i)];
          double nuy = fabs(cy) * p->dt / p->dy;
          double dFy = flux_difference(cy, nuy, fy[0], fy[1], fy[2], fy[3], fy[4]);
          fstar[fidx(p, a, j, i)] = fin[fidx(p, a, j, i)] - cy * p->dt / p->dy * dFy;
        }
  }
#pragma omp parallel for schedule(static) num_threads(orc_threads)
  for (int j = 0; j < p->ny; ++j) {
    double f[ORC_MAXQ], fes[ORC_MAXQ], gf[ORC_MAXQ], tau;
    for (int i = 0; i < p->nx; ++i) {
      for (int a = 0; a < Q; ++a) f[a] = fin[fidx(p, a, j, i)];
      cell_collision(L, p, f, fes, gf, &tau);
      for (int a = 0; a < Q; ++a) {
        double cx = L->c[a][0], cy = L->c[a][1]; /* c_z is not advected: the grid is 2D */
        double nux = fabs(cx) * p->dt / p->dx, nuy = fabs(cy) * p->dt / p->dy;
        double fx[5], fy[5];
        double coll = p->dt / tau * (fes[a] - f[a]) + gf[a] * p->dt;
        if (p->scheme == 1) {
          for (int k = -2; k <= 2; ++k) fx[k + 2] = fstar[fidx(p, a, j, col_of(p, i + k))];
          double dFx = flux_difference(cx, nux, fx[0], fx[1], fx[2], fx[3], fx[4]);
          fout[fidx(p, a, j, i)] = fx[2] - cx * p->dt / p->dx * dFx + coll;
        } else {
          for (int k = -2; k <= 2; ++k) {
            fx[k + 2] = fin[fidx(p, a, j, col_of(p, i + k))];
            fy[k + 2] = fin[fidx(p, a, row_of(p, j + k), i)];
          }
          double dFx = flux_difference(cx, nux, fx[0], fx[1], fx[2], fx[3], fx[4]);
          double dFy = flux_difference(cy, nuy, fy[0], fy[1], fy[2], fy[3], fy[4]);
          fout[fidx(p, a, j, i)] = f[a] - cx * p->dt / p->dx * dFx - cy * p->dt / p->dy * dFy + coll;
        }
      }
    }
  }
  free(fstar);
  apply_walls(L, p, fout, p->time + p->dt); /* the wall state at the new time */
  free(Lp);
  return 0;
}

/* nsteps steps from time p->time; f is updated in place (work is a scratch
 * array of the same size). */
int orc_run(const orc_params *p, double *f, double *work, int64_t nsteps) {
  size_t nq = (size_t)p->nroots * p->nroots * (dim_of(p) == 3 ? p->nroots : 1);
  size_t n = nq * p->nx * p->ny;
  orc_params q = *p;
  for (int64_t s = 0; s < nsteps; ++s) {
    q.time = p->time + (double)s * p->dt;
    if (orc_step(&q, f, work)) return -1;
    memcpy(f, work, n * sizeof(double));
  }
  return 0;
}

/* Moments of every node: out[9][ny][nx]; sums = {mass, x-mom, y-mom, energy}
 * with energy = sum_cells 1/2 sum_a f_a c_a^2 (c^2 over all D components). */
int orc_moments(const orc_params *p, const double *f, double *out, double *sums) {
  if (check_params(p)) return -1;
  orc_lattice *L = lattice_new(p->nroots, dim_of(p));
  if (!L) return -1;
  size_t cells = (size_t)p->nx * p->ny;
  double s[4] = {0, 0, 0, 0};
  for (int j = 0; j < p->ny; ++j)
    for (int i = 0; i < p->nx; ++i) {
      double fc[ORC_MAXQ], m[9];
      for (int a = 0; a < L->Q; ++a) fc[a] = f[fidx(p, a, j, i)];
      cell_moments(L, fc, m, NULL, NULL);
      size_t c = (size_t)j * p->nx + i;
      if (out)
        for (int k = 0; k < 9; ++k) out[k * cells + c] = m[k];
      for (int a = 0; a < L->Q; ++a) {
        double c2 = 0.0;
        for (int d = 0; d < L->D; ++d) c2 += L->c[a][d] * L->c[a][d];
        s[0] += fc[a];
        s[1] += fc[a] * L->c[a][0];
        s[2] += fc[a] * L->c[a][1];
        s[3] += 0.5 * fc[a] * c2;
      }
    }
  free(L);
  if (sums)
    for (int k = 0; k < 4; ++k) sums[k] = s[k];
  return 0;
}
