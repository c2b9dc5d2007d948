// Host-side set-up shared by the solvers (see setup.h).
#include "setup.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "tables.h"

namespace lesbgk_setup {

namespace {
thread_local char g_err[512] = "";
}  // namespace

const char *last_error_buffer() { return g_err; }

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char *where) {
  return fail(LESBGK_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

void clear_error() { g_err[0] = 0; }

int default_order(int nroots) { return nroots == 4 ? 3 : 4; }

int check_params(const lesbgk_params *p) {
  if (!p) return fail(LESBGK_EINVAL, "params is NULL");
  if (p->struct_size != sizeof(lesbgk_params))
    return fail(LESBGK_EINVAL, "struct_size %u != %zu", p->struct_size, sizeof(lesbgk_params));
  if (p->nroots != 4 && p->nroots != 6) return fail(LESBGK_EINVAL, "nroots must be 4 or 6");
  const int order = p->order ? p->order : default_order(p->nroots);
  if (order != 3 && order != 4) return fail(LESBGK_EINVAL, "order must be 3 or 4");
  if (p->nx < 1 || p->ny < 1) return fail(LESBGK_EINVAL, "nx, ny must be >= 1");
  // node indices stay below 2^31 (each thread's warp index and the row/column
  // products in the kernels are 64-bit or bounded by it)
  if ((long long)p->nx * p->ny > (1LL << 31) - 1) return fail(LESBGK_EINVAL, "grid too large (nx ny >= 2^31)");
  if (p->dim != 0 && p->dim != 2 && p->dim != 3) return fail(LESBGK_EINVAL, "dim must be 2 or 3");
  if (p->dim == 3 && !((p->nroots == 4 && order == 3) || (p->nroots == 6 && order == 4)))
    return fail(LESBGK_EINVAL, "D = 3 is built as D3Q64 (nroots 4, order 3) and D3Q216 (nroots 6, order 4)");
  if (p->bc_y != LESBGK_PERIODIC && p->bc_y != LESBGK_DIFFUSE) return fail(LESBGK_EINVAL, "bad bc_y");
  if (p->bc_x != LESBGK_PERIODIC && p->bc_x != LESBGK_DIFFUSE) return fail(LESBGK_EINVAL, "bad bc_x");
  if (p->bc_x == LESBGK_DIFFUSE) {
    if (p->nx < 2) return fail(LESBGK_EINVAL, "walls in x need nx >= 2");
    if (p->storage == LESBGK_F32C) return fail(LESBGK_EINVAL, "walls in x take FP32, FP16 or BF16 storage");
    if (p->wall_specular != 0.0) return fail(LESBGK_EINVAL, "walls in x are built with fully diffuse y-walls");
    for (int s = 0; s < 2; ++s)
      if (!(p->wall_Tx[s] > 0.0) || !std::isfinite(p->wall_Tx[s])) return fail(LESBGK_EINVAL, "wall_Tx must be > 0");
  }
  if (p->bc_y == LESBGK_DIFFUSE && p->ny < 2) return fail(LESBGK_EINVAL, "walls need ny >= 2");
  if (!(p->dx >= 0.0 && p->dy >= 0.0) || !std::isfinite(p->dx) || !std::isfinite(p->dy) ||
      ((p->dx > 0.0) != (p->dy > 0.0)))
    return fail(LESBGK_EINVAL, "dx and dy must both be 0 (derived) or both > 0");
  if (p->row_period < 0) return fail(LESBGK_EINVAL, "row_period must be >= 0");
  if (p->storage != LESBGK_F32 && p->storage != LESBGK_F16 && p->storage != LESBGK_BF16 &&
      p->storage != LESBGK_F32C)
    return fail(LESBGK_EINVAL, "storage must be LESBGK_F32, LESBGK_F16, LESBGK_BF16 or LESBGK_F32C");
  if (p->storage == LESBGK_F32C &&
      (p->nroots != 4 || order != 3 || p->bc_x != LESBGK_PERIODIC || p->wall_specular != 0.0))
    return fail(LESBGK_EINVAL, "compensated storage is built for D2Q16 and D3Q64 (order 3), periodic in x, "
                "without a specular share");
  if (p->storage != LESBGK_F32 && order != default_order(p->nroots))
    return fail(LESBGK_EINVAL, "16-bit storage is built for the default order only");
  if (p->scheme != LESBGK_UNSPLIT && p->scheme != LESBGK_SPLIT)
    return fail(LESBGK_EINVAL, "scheme must be LESBGK_UNSPLIT or LESBGK_SPLIT");
  if (!(p->kn > 0.0) || !std::isfinite(p->kn)) return fail(LESBGK_EINVAL, "Kn must be > 0");
  if (!(p->b >= -0.5 && p->b < 1.0)) return fail(LESBGK_EINVAL, "b must satisfy -1/2 <= b < 1");
  if (!(p->visc_exp >= 0.0 && p->visc_exp <= 1.0)) return fail(LESBGK_EINVAL, "visc_exp must be in [0,1]");
  if (!(p->dt >= 0.0) || !std::isfinite(p->dt)) return fail(LESBGK_EINVAL, "dt must be >= 0");
  if (p->dt == 0.0 && !(p->cfl > 0.0 && p->cfl <= 1.0)) return fail(LESBGK_EINVAL, "cfl must be in (0,1]");
  if (!(p->wall_specular >= 0.0 && p->wall_specular <= 1.0))
    return fail(LESBGK_EINVAL, "wall_specular must be in [0, 1]");
  if (!std::isfinite(p->wall_T_amp) || !std::isfinite(p->wall_T_freq))
    return fail(LESBGK_EINVAL, "non-finite wall heating parameters");
  if (!(std::fabs(p->wall_T_amp) < std::fmin(p->wall_T[0], p->wall_T[1])))
    return fail(LESBGK_EINVAL, "|wall_T_amp| must stay below the wall temperatures");
  if (p->wall_specular != 0.0 && p->storage != LESBGK_F32)
    return fail(LESBGK_EINVAL, "Maxwell walls (wall_specular > 0) are built for FP32 storage");
  for (int s = 0; s < 2; ++s) {
    if (!(p->wall_T[s] > 0.0) || !std::isfinite(p->wall_T[s])) return fail(LESBGK_EINVAL, "wall_T must be > 0");
    if (!std::isfinite(p->wall_ux[s]) || !std::isfinite(p->g[s])) return fail(LESBGK_EINVAL, "non-finite wall_ux/g");
  }
  return 0;
}

FieldStats field_stats_host(const double *h_init, size_t cells) {
  FieldStats st{h_init[0], 0.0, -1};
  for (size_t k = 0; k < cells; ++k) {
    const double r = h_init[k], T = h_init[3 * cells + k];
    if (!(r > 0.0) || !(T > 0.0) || !std::isfinite(r) || !std::isfinite(T) || !std::isfinite(h_init[cells + k]) ||
        !std::isfinite(h_init[2 * cells + k])) {
      st.bad_node = (long long)k;
      return st;
    }
    st.rho_max = std::fmax(st.rho_max, r);
    st.T_max = std::fmax(st.T_max, T);
  }
  return st;
}

int build_setup(const lesbgk_params &p, int order, const FieldStats *stats, Setup *out) {
  using namespace lesbgk_tables;
  Setup *h = out;
  const int nr = p.nroots, N = order;
  double c[kMaxRoots], w[kMaxRoots];
  if (gauss_hermite(nr, c, w)) return fail(LESBGK_EINVAL, "quadrature failed");
  KArgs &A = h->args;
  std::memset(&A, 0, sizeof A);
  h->cmax = std::fabs(c[0]);
  // spacing: a walled axis spans [0, 1] with walls on its end nodes; a
  // periodic axis of n nodes has 1/n, or the walled axis's spacing when only
  // one axis has walls (square cells)
  const bool xw = p.bc_x == LESBGK_DIFFUSE, yw = p.bc_y == LESBGK_DIFFUSE;
  if (!xw && !yw) {
    h->dx = 1.0 / p.nx;
    h->dy = 1.0 / p.ny;
  } else if (!xw) {
    h->dy = 1.0 / (p.ny - 1);
    h->dx = h->dy;
  } else if (!yw) {
    h->dx = 1.0 / (p.nx - 1);
    h->dy = h->dx;
  } else {
    h->dx = 1.0 / (p.nx - 1);
    h->dy = 1.0 / (p.ny - 1);
  }
  if (p.dx > 0.0) {  // explicit spacing (a y-slab keeps the whole domain's)
    h->dx = p.dx;
    h->dy = p.dy;
  }
  // reference state for tau_ref
  double tmax = 1.0, rmax = 1.0;
  if (p.bc_y == LESBGK_DIFFUSE)
    tmax = std::fmax(tmax, std::fmax(p.wall_T[0], p.wall_T[1]) + std::fabs(p.wall_T_amp));
  if (p.bc_x == LESBGK_DIFFUSE) tmax = std::fmax(tmax, std::fmax(p.wall_Tx[0], p.wall_Tx[1]));
  if (stats) {
    if (stats->bad_node >= 0)
      return fail(LESBGK_EINVAL, "initial field at node %lld not admissible (rho, T > 0, finite)", stats->bad_node);
    rmax = stats->rho_max;
    tmax = std::fmax(tmax, stats->T_max);
  }
  const double pr = 1.0 / (1.0 - p.b);
  h->tau_ref = (p.kn / pr) * std::pow(tmax, p.visc_exp - 1.0) / rmax;
  const double hmin = std::fmin(h->dx, h->dy);
  if (p.dt > 0.0) {
    h->dt = p.dt;
    if (h->cmax * h->dt / hmin > 1.0) return fail(LESBGK_EUNSTABLE, "CFL %.3f > 1", h->cmax * h->dt / hmin);
    if (h->dt / h->tau_ref >= 2.0) return fail(LESBGK_EUNSTABLE, "dt/tau_ref = %.3f >= 2", h->dt / h->tau_ref);
  } else {
    h->dt = std::fmin(p.cfl * hmin / h->cmax, h->tau_ref);
  }
  const double dt = h->dt;
  double fact[kMaxOrder + 1] = {1, 1, 2, 6, 24};
  for (int i = 0; i < nr; ++i) {
    double hv[kMaxOrder + 1];
    hermite_values(kMaxOrder, c[i], hv);
    A.c[i] = (float)c[i];
    for (int m = 0; m <= kMaxOrder; ++m) {
      A.he[i][m] = (float)hv[m];
      A.hw[i][m] = (float)(w[i] * hv[m] / fact[m]);
    }
    A.ax[i] = (float)(c[i] * dt / h->dx);
    A.kx[i] = (float)(0.5 * (1.0 - std::fabs(c[i]) * dt / h->dx));
    A.ay[i] = (float)(c[i] * dt / h->dy);
    A.ky[i] = (float)(0.5 * (1.0 - std::fabs(c[i]) * dt / h->dy));
    A.nay[i] = -A.ay[i];
    A.kx2[i][0] = A.kx2[i][1] = A.kx[i];
    A.nax2[i][0] = A.nax2[i][1] = -A.ax[i];
  }
  // FP16 holds 2^10 (f_a - w_a)/w_a: relative deviations down to 6e-8 stay in
  // its normal range (where stochastic rounding is unbiased) and up to 64 fit;
  // the compensated storage's FP16 remainder holds lo 2^24 / w_a (|lo| is at
  // most half an FP32 ulp of the deviation: 2^-24 of it)
  const double store_scale = p.storage == LESBGK_F16 ? 1024.0 : (p.storage == LESBGK_F32C ? 16777216.0 : 1.0);
  const int nzw = p.dim == 3 ? nr / 2 : 1;  // stored z-levels
  for (int iz = 0; iz < nzw; ++iz)
    for (int ix = 0; ix < nr; ++ix)
      for (int iy = 0; iy < nr; ++iy) {
        const double wa = w[ix] * w[iy] * (p.dim == 3 ? w[nr / 2 + iz] : 1.0);
        A.wq[(iz * nr + ix) * nr + iy] = (float)(wa / store_scale);
        A.iwq[(iz * nr + ix) * nr + iy] = (float)(store_scale / wa);
      }
  A.c_omega = (float)(dt / (p.kn * (1.0 - p.b)));
  A.visc_pow = (float)(1.0 - p.visc_exp);
  A.vmode = p.visc_exp == 0.5 ? 1 : (p.visc_exp == 1.0 ? 2 : 0);
  const int D = p.dim == 3 ? 3 : 2;
  A.b = (float)p.b;
  A.beta = (float)((1.0 - p.b) / D);  // rho (lambda - I) = (1-b) tr M / D + b M
  A.dtgx = (float)(dt * p.g[0]);
  A.dtgy = (float)(dt * p.g[1]);
  A.has_force = (p.g[0] != 0.0 || p.g[1] != 0.0) ? 1 : 0;
  A.nx = p.nx;
  A.ny = p.ny;
  A.walls = p.bc_y == LESBGK_DIFFUSE ? 1 : 0;
  A.wspec = (float)p.wall_specular;
  A.plane = (long long)p.nx * p.ny;
  A.row_key = p.row_offset;
  A.row_period = p.row_period;
  h->nroots = nr;
  h->order = N;
  h->dim = D;
  for (int i = 0; i < nr; ++i) {
    h->c[i] = c[i];
    h->w[i] = w[i];
  }
  for (int s = 0; s < 2; ++s) {
    h->wall_T[s] = p.wall_T[s];
    h->wall_ux[s] = p.wall_ux[s];
  }
  h->wall_T_amp = p.wall_T_amp;
  h->wall_T_freq = p.wall_T_freq;
  h->wall_Tx[0] = p.wall_Tx[0];
  h->wall_Tx[1] = p.wall_Tx[1];
  if (p.wall_T_amp != 0.0) heat_poly(h);
  set_wall_time(*h, 0.0, &h->args);
  A.xwalls = xw ? 1 : 0;
  if (xw) x_wall_tables(*h, &h->args);
  return 0;
}

// Walls at rest normal to x and the cavity corners: S(T_wx, u = 0) per stored
// population in FP64, the x-wall constants (|c_x| over the outgoing half) and
// the corner constants (|c.n_x + c.n_y| over the kept populations).
void x_wall_tables(const Setup &h, KArgs *out) {
  using namespace lesbgk_tables;
  KArgs &A = *out;
  const int nr = h.nroots, N = h.order, H = nr / 2;
  const double *c = h.c, *w = h.w;
  const double fact[kMaxOrder + 1] = {1, 1, 2, 6, 24};
  const int nz = h.dim == 3 ? H : 1;
  for (int s = 0; s < 2; ++s) {
    double e[kMaxOrder + 1][kMaxOrder + 1];
    const double th = h.wall_Tx[s] - 1.0;
    gaussian_hermite_moments(N, 1.0, 0.0, 0.0, th, 0.0, th, e);
    const double zf[kMaxOrder + 1] = {1.0, 0.0, th, 0.0, 3.0 * th * th};
    double S[kMaxWQ];
    double A_out = 0.0, Z_out = 0.0;
    for (int iz = 0; iz < nz; ++iz)
      for (int ix = 0; ix < nr; ++ix)
        for (int iy = 0; iy < nr; ++iy) {
          double hx[kMaxOrder + 1], hy[kMaxOrder + 1], hz[kMaxOrder + 1];
          hermite_values(kMaxOrder, c[ix], hx);
          hermite_values(kMaxOrder, c[iy], hy);
          hermite_values(kMaxOrder, h.dim == 3 ? c[H + iz] : 0.0, hz);
          double sum = 0.0;
          for (int m = 0; m <= N; ++m)
            for (int k = 0; m + k <= N; ++k)
              for (int l = 0; m + k + l <= N && (l == 0 || h.dim == 3); l += 2)
                sum += e[m][k] * zf[l] * hx[m] * hy[k] * hz[l] / (fact[m] * fact[k] * fact[l]);
          const double wa = w[ix] * w[iy] * (h.dim == 3 ? w[H + iz] : 1.0);
          const int a = (iz * nr + ix) * nr + iy;
          S[a] = wa * sum;
          A.wSx[s][a] = (float)S[a];
          A.wSxdev[s][a] = (float)(S[a] - wa);
          const bool outgoing = s == 0 ? (c[ix] > 0.0) : (c[ix] < 0.0);
          if (outgoing) {
            A_out += std::fabs(c[ix]) * (S[a] - wa);
            Z_out += std::fabs(c[ix]) * S[a];
          }
        }
    A.wAx[s] = (float)A_out;
    A.wBx[s] = (float)(1.0 / Z_out);
    for (int ys = 0; ys < 2; ++ys) {  // the two corners on this x-wall
      const double nx = s == 0 ? 1.0 : -1.0, ny = ys == 0 ? 1.0 : -1.0;
      double Ac = 0.0, Zc = 0.0;
      for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nr; ++ix)
          for (int iy = 0; iy < nr; ++iy) {
            if (!(c[ix] * nx < 0.0 && c[iy] * ny < 0.0)) continue;
            const int a = (iz * nr + ix) * nr + iy;
            const double wa = w[ix] * w[iy] * (h.dim == 3 ? w[H + iz] : 1.0);
            const double cn = std::fabs(c[ix] * nx + c[iy] * ny);
            Ac += cn * (S[a] - wa);
            Zc += cn * S[a];
          }
      A.wAc[ys * 2 + s] = (float)Ac;
      A.wBc[ys * 2 + s] = (float)(1.0 / Zc);
    }
  }
}

namespace {

// Wall equilibria S_a(T_w + heat, u_w) of wall s at order N (b = 0 Gaussian
// projection) per stored population, in FP64; in D = 3 the z-factor of the
// isotropic Gaussian's coefficients is E[He_l(Z)] = 1, th, 3 th^2 for l = 0,
// 2, 4 (Z ~ N(0, T_w), u_z = 0).  The D = 3 sets store the z-even half:
// levels c_z = c[nr/2 + iz] > 0.
void wall_equilibrium(const Setup &h, double heat, int s, double *S) {
  using namespace lesbgk_tables;
  const int nr = h.nroots, N = h.order;
  const double *c = h.c, *w = h.w;
  const double fact[kMaxOrder + 1] = {1, 1, 2, 6, 24};
  const int nz = h.dim == 3 ? nr / 2 : 1;
  double e[kMaxOrder + 1][kMaxOrder + 1];
  const double th = h.wall_T[s] + heat - 1.0;
  gaussian_hermite_moments(N, 1.0, h.wall_ux[s], 0.0, th, 0.0, th, e);
  const double zf[kMaxOrder + 1] = {1.0, 0.0, th, 0.0, 3.0 * th * th};
  for (int iz = 0; iz < nz; ++iz)
    for (int ix = 0; ix < nr; ++ix) {
      double hx[kMaxOrder + 1], hz[kMaxOrder + 1];
      hermite_values(kMaxOrder, c[ix], hx);
      hermite_values(kMaxOrder, h.dim == 3 ? c[nr / 2 + iz] : 0.0, hz);
      for (int iy = 0; iy < nr; ++iy) {
        double hy[kMaxOrder + 1];
        hermite_values(kMaxOrder, c[iy], hy);
        double sum = 0.0;
        for (int m = 0; m <= N; ++m)
          for (int k = 0; m + k <= N; ++k) {
            if (h.dim != 3) {
              sum += e[m][k] * hx[m] * hy[k] / (fact[m] * fact[k]);
              continue;
            }
            for (int l = 0; m + k + l <= N; l += 2)
              sum += e[m][k] * zf[l] * hx[m] * hy[k] * hz[l] / (fact[m] * fact[k] * fact[l]);
          }
        const double wa = w[ix] * w[iy] * (h.dim == 3 ? w[nr / 2 + iz] : 1.0);
        S[(iz * nr + ix) * nr + iy] = wa * sum;
      }
    }
}

int stored_q(const Setup &h) { return h.nroots * h.nroots * (h.dim == 3 ? h.nroots / 2 : 1); }

double stored_w(const Setup &h, int a) {
  const int nr = h.nroots, iy = a % nr, ix = (a / nr) % nr, iz = a / (nr * nr);
  return h.w[ix] * h.w[iy] * (h.dim == 3 ? h.w[nr / 2 + iz] : 1.0);
}

bool outgoing_y(const Setup &h, int s, int a) {
  const double cy = h.c[a % h.nroots];
  return s == 0 ? cy > 0.0 : cy < 0.0;
}

}  // namespace

void heat_poly(Setup *h) {
  HeatPoly &P = h->heat;
  std::memset(&P, 0, sizeof P);
  P.amp = h->wall_T_amp;
  P.freq = h->wall_T_freq;
  P.dt = h->dt;
  const int q = stored_q(*h);
  for (int a = 0; a < q; ++a) P.w[a] = stored_w(*h, a);
  // the polynomial through heat = -1, 0, 1 (exact for degree 2)
  for (int s = 0; s < 2; ++s) {
    double Sm[kMaxWQ], S0[kMaxWQ], Sp[kMaxWQ];
    wall_equilibrium(*h, -1.0, s, Sm);
    wall_equilibrium(*h, 0.0, s, S0);
    wall_equilibrium(*h, 1.0, s, Sp);
    for (int a = 0; a < q; ++a) {
      P.S[s][0][a] = S0[a];
      P.S[s][1][a] = 0.5 * (Sp[a] - Sm[a]);
      P.S[s][2][a] = 0.5 * (Sp[a] + Sm[a]) - S0[a];
    }
    for (int k = 0; k < 3; ++k) {
      double ao = 0.0, zo = 0.0;
      for (int a = 0; a < q; ++a)
        if (outgoing_y(*h, s, a)) {
          const double cn = std::fabs(h->c[a % h->nroots]);
          ao += cn * (k == 0 ? P.S[s][0][a] - P.w[a] : P.S[s][k][a]);
          zo += cn * P.S[s][k][a];
        }
      P.Aout[s][k] = ao;
      P.Zout[s][k] = zo;
    }
  }
}

void set_wall_time(const Setup &h, double t, KArgs *out) {
  KArgs &A = *out;
  const int q = stored_q(h);
  if (h.wall_T_amp != 0.0) {  // heated: the polynomial tables at h = amp sin(freq t)
    const HeatPoly &P = h.heat;
    const double hv = wall_heating(P, t);
    for (int s = 0; s < 2; ++s) {
      for (int a = 0; a < q; ++a) {
        const double S = std::fma(std::fma(P.S[s][2][a], hv, P.S[s][1][a]), hv, P.S[s][0][a]);
        A.wS[s][a] = (float)S;
        A.wSdev[s][a] = (float)(S - P.w[a]);
      }
      const double ao = std::fma(std::fma(P.Aout[s][2], hv, P.Aout[s][1]), hv, P.Aout[s][0]);
      const double zo = std::fma(std::fma(P.Zout[s][2], hv, P.Zout[s][1]), hv, P.Zout[s][0]);
      A.wA[s] = (float)ao;
      A.wB[s] = (float)(1.0 / zo);
    }
    return;
  }
  for (int s = 0; s < 2; ++s) {
    double S[kMaxWQ];
    wall_equilibrium(h, 0.0, s, S);
    double A_out = 0.0, Z_out = 0.0;
    for (int a = 0; a < q; ++a) {
      const double wa = stored_w(h, a);
      A.wS[s][a] = (float)S[a];
      A.wSdev[s][a] = (float)(S[a] - wa);
      if (outgoing_y(h, s, a)) {
        A_out += std::fabs(h.c[a % h.nroots]) * (S[a] - wa);
        Z_out += std::fabs(h.c[a % h.nroots]) * S[a];
      }
    }
    A.wA[s] = (float)A_out;
    A.wB[s] = (float)(1.0 / Z_out);
  }
}

}  // namespace lesbgk_setup

extern "C" const char *lesbgk_last_error(void) { return lesbgk_setup::last_error_buffer(); }
