// Host-side set-up shared by the single-domain solver and the batched
// solver: argument checks, the FP64 tables of Sec. 2.2 rounded to the kernels'
// FP32 argument block, the time-step rule, and thread-local error messages.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "lesbgk.h"

namespace lesbgk_setup {

constexpr int kMaxR = 6;
constexpr int kMaxN = 4;
constexpr int kMaxQ = kMaxR * kMaxR;             // values per node of the 2D sets, D3Q64's 32
constexpr int kMaxWQ = kMaxR * kMaxR * kMaxR / 2;  // values per node of D3Q216 (its z-even half)

// Kernel arguments: lattice tables and scalars, passed by value (constant bank).
struct KArgs {
  float c[kMaxR];              // 1D abscissae, ascending; c[NR-1-i] = -c[i]
  float he[kMaxR][kMaxN + 1];  // He_m(c_i)
  float hw[kMaxR][kMaxN + 1];  // w_i He_m(c_i) / m!
  float ax[kMaxR], kx[kMaxR];  // c_i dt/dx and (1 - |c_i| dt/dx)/2
  alignas(8) float ay[kMaxR];  // same along y
  alignas(8) float ky[kMaxR];
  // pair operands of the packed (f32x2) advection, whose pairs are the
  // populations a, a+1 (the same ix, neighbouring iy)
  alignas(8) float nay[kMaxR];      // -ay
  alignas(8) float kx2[kMaxR][2];   // {kx, kx}
  alignas(8) float nax2[kMaxR][2];  // {-ax, -ax}
  float wS[2][kMaxWQ];         // wall equilibrium S_a(T_w, u_w) per stored population, [0] bottom, [1] top
  float wSdev[2][kMaxWQ];      // S_a - w_a
  float wA[2], wB[2];          // sum_out |c_y|(S-w) and 1/sum_out |c_y| S
  float wq[kMaxWQ], iwq[kMaxWQ];  // 16-bit storage: stored = df * iwq, df = stored * wq
  float c_omega;               // dt / (Kn (1-b)):  dt/tau = c_omega rho T^(1-varpi)
  float visc_pow;              // 1 - varpi
  float b, beta;               // b and (1-b)/D
  float dtgx, dtgy;            // dt g
  int nx, ny, walls, has_force, vmode;  // vmode 1: varpi = 1/2, 2: varpi = 1, 0: general
  int rows, nstrips, nseg;
  long long plane;             // nx*ny
  unsigned seed;               // per-launch key of the 16-bit stochastic rounding
  int row_key;                 // global index of row 0 (the rounding is keyed by global row)
  int row_period;              // wrap of the global row (the whole domain's ny if periodic), or 0
  float wspec;                 // specular fraction 1 - gamma of the Maxwell wall (0: fully diffuse)
  int xwalls;                  // diffuse walls at rest on columns 0 and nx-1
  float wSx[2][kMaxWQ];        // x-wall equilibrium S(T_wx, 0), [0] left, [1] right
  float wSxdev[2][kMaxWQ];     // S - w
  float wAx[2], wBx[2];        // as wA, wB with |c_x| over the outgoing half
  float wAc[4], wBc[4];        // corners [yside * 2 + xside]: sum_kept |c.n|(S-w), 1/sum_kept |c.n| S
};

#if defined(__CUDACC__)
#define LESBGK_HD __host__ __device__
#else
#define LESBGK_HD
#endif

// sin x for the heated walls (Sec. 4.2), the same bits on the host and the
// device: Cody and Waite's reduction x = k pi/2 + r (pi/2 as the sum of three
// doubles, every step one fused multiply-add), then the Taylor series of sin
// and cos on |r| <= pi/4 (to r^17 and r^18: the next terms are below 1e-19),
// evaluated by Horner's rule with fused multiply-adds only, so no compiler
// contraction choice can change a result.  Relative error a few 1e-16 for
// |x| < 2^30.
LESBGK_HD inline double wall_sin(double x) {
  // pi/2 = a + b + c to 159 bits; 2/pi rounded; the Taylor coefficients are
  // 1/n! rounded to the nearest double (hexadecimal literals: exact bits)
  const double kPio2a = 0x1.921fb54442d18p+0, kPio2b = 0x1.1a62633145c07p-54, kPio2c = -0x1.f1976b7ed8fbcp-110;
  const double k = rint(x * 0x1.45f306dc9c883p-1);
  double r = fma(-k, kPio2a, x);
  r = fma(-k, kPio2b, r);
  r = fma(-k, kPio2c, r);
  const double r2 = r * r;
  const long long q = (long long)k & 3;
  if (q & 1) {  // cos r
    double p = 0x1.6827863b97d97p-53;  // 1/18!, then -1/16!, 1/14!, ..., 1/2!
    p = fma(p, r2, -0x1.ae7f3e733b81fp-45);
    p = fma(p, r2, 0x1.93974a8c07c9dp-37);
    p = fma(p, r2, -0x1.1eed8eff8d898p-29);
    p = fma(p, r2, 0x1.27e4fb7789f5cp-22);
    p = fma(p, r2, -0x1.a01a01a01a01ap-16);
    p = fma(p, r2, 0x1.6c16c16c16c17p-10);
    p = fma(p, r2, -0x1.5555555555555p-5);
    p = fma(p, r2, 0.5);
    const double c = fma(-r2, p, 1.0);
    return q == 1 ? c : -c;
  }
  double p = 0x1.952c77030ad4ap-49;  // 1/17!, then -1/15!, 1/13!, ..., -1/3!
  p = fma(p, r2, -0x1.ae7f3e733b81fp-41);
  p = fma(p, r2, 0x1.6124613a86d09p-33);
  p = fma(p, r2, -0x1.ae64567f544e4p-26);
  p = fma(p, r2, 0x1.71de3a556c734p-19);
  p = fma(p, r2, -0x1.a01a01a01a01ap-13);
  p = fma(p, r2, 0x1.1111111111111p-7);
  p = fma(p, r2, -0x1.5555555555555p-3);
  const double sn = fma(r * r2, p, r);
  return q == 0 ? sn : -sn;
}

// Heated walls (Sec. 4.2): the wall equilibrium S_a at T_w + h is, to order
// N <= 4, a polynomial of degree 2 in h (the Hermite coefficients of a
// Gaussian are polynomials of degree <= N/2 in its temperature), so per wall
// S_a(h) = S[0][a] + S[1][a] h + S[2][a] h^2, and likewise the two sums the
// wall rule needs.  Both the host (the single-domain solver's per-step tables)
// and the device (the batched solver) evaluate them as
// fma(fma(P2, h, P1), h, P0) with h = amp wall_sin(freq t), t = (n + 1) dt for
// the state step n writes: the same bits on either side.
struct HeatPoly {
  double S[2][3][kMaxWQ];         // per wall, per power of h, per stored population
  double Aout[2][3], Zout[2][3];  // sum_out |c_n| (S_a - w_a), sum_out |c_n| S_a
  double w[kMaxWQ];               // w_a
  double amp, freq, dt;
};

// What one solve's set-up produces.
struct Setup {
  KArgs args;                      // tables and per-solve scalars (nx, ny, plane, walls filled)
  double dt, dx, dy, cmax, tau_ref;
  // what the wall tables are built from (Sec. 3.2; heating of Sec. 4.2)
  int nroots, order, dim;          // dim: velocity-set dimension D (2 or 3)
  double c[kMaxR], w[kMaxR];       // FP64 quadrature
  double wall_T[2], wall_ux[2];    // steady wall temperature and velocity
  double wall_T_amp, wall_T_freq;  // T_w(t) = wall_T + wall_T_amp sin(wall_T_freq t)
  double wall_Tx[2];               // x-wall temperatures (walls in x are steady and at rest)
  HeatPoly heat;                   // heated walls: the tables as polynomials in the heating
};

// Record a message for lesbgk_last_error() and return code.
int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int cuda_fail(cudaError_t e, const char *where);
void clear_error();
const char *last_error_buffer();

int default_order(int nroots);
int check_params(const lesbgk_params *p);

// What the initial fields contribute to the set-up: their largest density and
// temperature (tau_ref), and the first node that is not admissible (rho > 0,
// T > 0, all four fields finite), or -1.
struct FieldStats {
  double rho_max, T_max;
  long long bad_node;
};

// The same from host fields double[4][cells] (a plain loop).
FieldStats field_stats_host(const double *h_init, size_t cells);

// Quadrature, Hermite and wall tables in FP64 (rounded to FP32 in args),
// spacing, tau_ref and dt (Sec. 2.2; the dt rule is the library's reading).
// stats (may be NULL: rest initial state) enters tau_ref and is checked.
int build_setup(const lesbgk_params &p, int order, const FieldStats *stats, Setup *out);

// The heated walls' polynomial tables (h->heat) of a set-up whose wall
// temperature varies (build_setup calls it).
void heat_poly(Setup *h);

// Build the wall tables (wS, wSdev, wA, wB) of *A in FP64 for the wall
// temperature at time t; build_setup calls it for args with t = 0.
void set_wall_time(const Setup &h, double t, KArgs *A);

// Tables of the walls normal to x and of the corners (steady; build_setup
// calls it when bc_x has walls).
void x_wall_tables(const Setup &h, KArgs *A);

// The heating h = amp sin(freq t) at time t (wall_sin).
LESBGK_HD inline double wall_heating(const HeatPoly &hp, double t) { return hp.amp * wall_sin(hp.freq * t); }

// Whether the wall temperature varies in time (the tables then change per step).
inline bool heated_walls(const Setup &h) { return h.args.walls && h.wall_T_amp != 0.0; }

}  // namespace lesbgk_setup
