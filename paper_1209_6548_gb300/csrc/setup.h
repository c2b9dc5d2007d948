// Host-side set-up shared by the single-domain solver and the batched
// solver: argument checks, the FP64 tables of Sec. 2.2 rounded to the kernels'
// FP32 argument block, the time-step rule, and thread-local error messages.
#pragma once

#include <cuda_runtime.h>

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
  float wq[kMaxQ], iwq[kMaxQ]; // 16-bit storage: stored = df * iwq, df = stored * wq
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
  float wSx[2][kMaxQ];         // x-wall equilibrium S(T_wx, 0), [0] left, [1] right
  float wSxdev[2][kMaxQ];      // S - w
  float wAx[2], wBx[2];        // as wA, wB with |c_x| over the outgoing half
  float wAc[4], wBc[4];        // corners [yside * 2 + xside]: sum_kept |c.n|(S-w), 1/sum_kept |c.n| S
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

// Build the wall tables (wS, wSdev, wA, wB) of *A in FP64 for the wall
// temperature at time t; build_setup calls it for args with t = 0.
void set_wall_time(const Setup &h, double t, KArgs *A);

// Tables of the walls normal to x and of the corners (steady; build_setup
// calls it when bc_x has walls).
void x_wall_tables(const Setup &h, KArgs *A);

// Whether the wall temperature varies in time (the tables then change per step).
inline bool heated_walls(const Setup &h) { return h.args.walls && h.wall_T_amp != 0.0; }

}  // namespace lesbgk_setup
