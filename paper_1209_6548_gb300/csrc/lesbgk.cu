// liblesbgk: GB300 (sm_103a) lattice ES-BGK solver behind the C ABI of
// include/lesbgk.h.  Method: Meng, Zhang, Hadjiconstantinou, Radtke & Shan,
// arXiv 1209.6548 (Sec. 2.2 lattice ES-BGK equation, Sec. 3.1 scheme,
// Sec. 3.2 diffuse walls).
//
// Data layout in HBM: populations as deviations df_a = f_a - w_a, float32, in
// the grouped layout of Layout<NR> below (vectors of 4 (D2Q16) or 2 (D2Q36)
// populations of one node that share the sign of c_y), two ping-pong buffers
// in the caller's workspace.  One time step = one launch of k_step.
//
// k_step mapping: a warp owns a strip of 32 consecutive x-nodes (the two
// outer lanes on each side are halo lanes that load but do not store) and
// marches up a segment of rows.  x-neighbours come from warp shuffles, the
// y-stencil is carried in registers from row to row, so each population is
// read from HBM once and written once per step (plus halo strips/rows that
// hit in L2).  Per node, all Q populations live in one thread: moments,
// collision, Hermite evaluation and the wall reduction are in-thread.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "lesbgk.h"
#include "tables.h"

namespace {

constexpr int kMaxR = 6;
constexpr int kMaxN = 4;
constexpr int kMaxQ = kMaxR * kMaxR;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 128;
constexpr int kMomBlock = 256;

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
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

// Kernel arguments: lattice tables and scalars, passed by value (constant bank).
struct KArgs {
  float c[kMaxR];              // 1D abscissae, ascending; c[NR-1-i] = -c[i]
  float he[kMaxR][kMaxN + 1];  // He_m(c_i)
  float hw[kMaxR][kMaxN + 1];  // w_i He_m(c_i) / m!
  float ax[kMaxR], kx[kMaxR];  // c_i dt/dx and (1 - |c_i| dt/dx)/2
  float ay[kMaxR], ky[kMaxR];  // same along y
  float wS[2][kMaxQ];          // wall equilibrium S_a(T_w, u_w), [0] bottom, [1] top
  float wSdev[2][kMaxQ];       // S_a - w_a
  float wA[2], wB[2];          // sum_out |c_y|(S-w) and 1/sum_out |c_y| S
  float c_omega;               // dt / (Kn (1-b)):  dt/tau = c_omega rho T^(1-varpi)
  float visc_pow;              // 1 - varpi
  float b, beta;               // b and (1-b)/2
  float dtgx, dtgy;            // dt g
  int nx, ny, walls, has_force, vmode;  // vmode 1: varpi = 1/2, 2: varpi = 1, 0: general
  int rows, nstrips, nseg;
  long long plane;             // nx*ny
};

__device__ __forceinline__ float minmod(float a, float b) {
  // signed smaller magnitude when a and b agree in sign, else 0 (= median(a, b, 0));
  // equals [f_{i+1}-f_i] Psi(Theta) of Sec. 3.1 with the minmod limiter.
  return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}

// Hardware approximations (MUFU): relative error ~1 ulp, far below the FP32
// rounding of the moments they act on.
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float fast_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ int map_row(int j, int ny, int walls) {
  if (walls) return j < 0 ? 0 : (j >= ny ? ny - 1 : j);  // ghost rows = wall node
  int r = j % ny;
  return r < 0 ? r + ny : r;
}

// ---------------------------------------------------------------------------
// Hermite moments a_mk = sum_a df_a He_m(c_ax) He_k(c_ay), m + k <= KM, of one
// node's deviations F[ix*NR+iy], by sum factorisation over the tensor-product
// set with the +/- pairing of the roots.
// ---------------------------------------------------------------------------
template <int NR, int KM>
__device__ __forceinline__ void hermite_moments(const float (&F)[NR * NR], float (&a)[KM + 1][KM + 1],
                                                const KArgs &A) {
  constexpr int H = NR / 2;
  float s[NR][KM + 1];
#pragma unroll
  for (int ix = 0; ix < NR; ++ix) {
    float ev[H], od[H];
#pragma unroll
    for (int p = 0; p < H; ++p) {
      const float fp = F[ix * NR + H + p], fn = F[ix * NR + H - 1 - p];
      ev[p] = fp + fn;
      od[p] = fp - fn;
    }
#pragma unroll
    for (int k = 0; k <= KM; ++k) {
      float acc;
      if (k == 0) {
        acc = ev[0];
#pragma unroll
        for (int p = 1; p < H; ++p) acc += ev[p];
      } else {
        acc = ((k & 1) ? od[0] : ev[0]) * A.he[H][k];
#pragma unroll
        for (int p = 1; p < H; ++p) acc = fmaf((k & 1) ? od[p] : ev[p], A.he[H + p][k], acc);
      }
      s[ix][k] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k <= KM; ++k) {
    float sp[H], sm[H];
#pragma unroll
    for (int p = 0; p < H; ++p) {
      sp[p] = s[H + p][k] + s[H - 1 - p][k];
      sm[p] = s[H + p][k] - s[H - 1 - p][k];
    }
#pragma unroll
    for (int m = 0; m + k <= KM; ++m) {
      float acc;
      if (m == 0) {
        acc = sp[0];
#pragma unroll
        for (int p = 1; p < H; ++p) acc += sp[p];
      } else {
        acc = ((m & 1) ? sm[0] : sp[0]) * A.he[H][m];
#pragma unroll
        for (int p = 1; p < H; ++p) acc = fmaf((m & 1) ? sm[p] : sp[p], A.he[H + p][m], acc);
      }
      a[m][k] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// S_a = w_a sum_{m+k<=N} d_mk He_m(c_ax) He_k(c_ay) / (m! k!), by two 1D
// passes (x then y) with the +/- pairing.
// ---------------------------------------------------------------------------
template <int NR, int N>
__device__ __forceinline__ void hermite_evaluate(const float (&d)[N + 1][N + 1], float (&S)[NR * NR],
                                                 const KArgs &A) {
  constexpr int H = NR / 2;
  float E[NR][N + 1];
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const int P = H + p;
#pragma unroll
    for (int k = 0; k <= N; ++k) {
      float ev = d[0][k] * A.hw[P][0];
#pragma unroll
      for (int m = 2; m + k <= N; m += 2) ev = fmaf(d[m][k], A.hw[P][m], ev);
      float od = 0.0f;
      if (k + 1 <= N) {
        od = d[1][k] * A.hw[P][1];
#pragma unroll
        for (int m = 3; m + k <= N; m += 2) od = fmaf(d[m][k], A.hw[P][m], od);
      }
      E[P][k] = ev + od;
      E[H - 1 - p][k] = ev - od;
    }
  }
#pragma unroll
  for (int ix = 0; ix < NR; ++ix) {
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const int P = H + q;
      float ev = E[ix][0] * A.hw[P][0];
#pragma unroll
      for (int k = 2; k <= N; k += 2) ev = fmaf(E[ix][k], A.hw[P][k], ev);
      float od = E[ix][1] * A.hw[P][1];
#pragma unroll
      for (int k = 3; k <= N; k += 2) od = fmaf(E[ix][k], A.hw[P][k], od);
      S[ix * NR + P] = ev + od;
      S[ix * NR + H - 1 - q] = ev - od;
    }
  }
}

// Coefficients e_mk = rho E[He_m(X) He_k(Y)], (X,Y) ~ N(u, lambda): the
// Hermite expansion of the anisotropic Gaussian of Eq. (cfeq) (equal to the
// a_ES^(n) of Sec. 2.2), from the recursion of its generating function
// rho exp(u.t + t.(lambda - I).t/2).  Inputs: rho, rho u, and L = lambda - I.
template <int N>
__device__ __forceinline__ void gaussian_coeffs(float rho, float ru_x, float ru_y, float ux, float uy,
                                                float Lxx, float Lxy, float Lyy, float RLxx, float RLxy,
                                                float RLyy, float (&e)[N + 1][N + 1]) {
  e[0][0] = rho;
  e[1][0] = ru_x;
  e[0][1] = ru_y;
  e[2][0] = fmaf(ux, ru_x, RLxx);
  e[1][1] = fmaf(ux, ru_y, RLxy);
  e[0][2] = fmaf(uy, ru_y, RLyy);
#pragma unroll
  for (int n = 3; n <= N; ++n) {
#pragma unroll
    for (int m = 0; m <= n; ++m) {
      const int k = n - m;
      float v;
      if (m >= 1) {
        v = ux * e[m - 1][k];
        if (m >= 2) v = fmaf((float)(m - 1) * Lxx, e[m - 2][k], v);
        if (k >= 1) v = fmaf((float)k * Lxy, e[m - 1][k - 1], v);
      } else {
        v = uy * e[0][k - 1];
        if (k >= 2) v = fmaf((float)(k - 1) * Lyy, e[0][k - 2], v);
      }
      e[m][k] = v;
    }
  }
}

// One node's collision + force source: S_a = (dt/tau)(f_ES,a - w_a) + dt g_a
// (deviation form) and omw = 1 - dt/tau.
template <int NR, int N>
__device__ __forceinline__ void collide(const float (&F)[NR * NR], float (&S)[NR * NR], float &omw,
                                        const KArgs &A) {
  constexpr int KM = (N - 1 > 2) ? N - 1 : 2;
  float a[KM + 1][KM + 1];
  hermite_moments<NR, KM>(F, a, A);
  const float rho = 1.0f + a[0][0];
  const float ir = fast_rcp(rho);
  const float ux = a[1][0] * ir, uy = a[0][1] * ir;
  // M = P - rho I (pressure tensor minus its rest value), from deviations
  const float Mxx = fmaf(-a[1][0], ux, a[2][0]);
  const float Mxy = fmaf(-a[1][0], uy, a[1][1]);
  const float Myy = fmaf(-a[0][1], uy, a[0][2]);
  const float trM = Mxx + Myy;
  const float T = fmaf(0.5f * trM, ir, 1.0f);  // T = tr P / (D rho), D = 2
  float Tp;
  if (A.vmode == 1) Tp = fast_sqrt(T);
  else if (A.vmode == 2) Tp = 1.0f;
  else Tp = exp2f(A.visc_pow * __log2f(T));
  const float om = A.c_omega * rho * Tp;  // dt/tau, tau = (Kn/Pr) T^varpi / (rho T)
  omw = 1.0f - om;
  // rho (lambda - I) = (1-b) rho (T-1) I + b M,  lambda = (1-b) T I + b P/rho
  const float RLxx = fmaf(A.beta, trM, A.b * Mxx);
  const float RLxy = A.b * Mxy;
  const float RLyy = fmaf(A.beta, trM, A.b * Myy);
  float e[N + 1][N + 1];
  gaussian_coeffs<N>(rho, a[1][0], a[0][1], ux, uy, RLxx * ir, RLxy * ir, RLyy * ir, RLxx, RLxy, RLyy, e);
  float d[N + 1][N + 1];
#pragma unroll
  for (int m = 0; m <= N; ++m)
#pragma unroll
    for (int k = 0; m + k <= N; ++k) d[m][k] = om * e[m][k];
  d[0][0] = om * a[0][0];
  if (A.has_force) {
    // projected body force: coefficient m g_x a_{m-1,k} + k g_y a_{m,k-1} (a_00 = rho)
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
      for (int k = 0; m + k <= N; ++k) {
        if (m + k == 0) continue;
        float v = d[m][k];
        if (m >= 1) v = fmaf((float)m * A.dtgx, (m - 1 + k == 0) ? rho : a[m - 1][k], v);
        if (k >= 1) v = fmaf((float)k * A.dtgy, (m + k - 1 == 0) ? rho : a[m][k - 1], v);
        d[m][k] = v;
      }
  }
  hermite_evaluate<NR, N>(d, S, A);
}

// Diffuse wall of Sec. 3.2 on one node's updated deviations: rho_W from the
// incoming half, outgoing half = rho_W S_a(T_w, u_w).  side 0: bottom
// (outgoing c_y > 0), side 1: top (outgoing c_y < 0).
template <int NR>
__device__ __forceinline__ void wall_fix(float (&O)[NR * NR], int side, const KArgs &A) {
  constexpr int H = NR / 2;
  float s = 0.0f;
#pragma unroll
  for (int ix = 0; ix < NR; ++ix)
#pragma unroll
    for (int iy = 0; iy < NR; ++iy) {
      const bool incoming = side == 0 ? (iy < H) : (iy >= H);
      if (incoming) s = fmaf(fabsf(A.c[iy]), O[ix * NR + iy], s);
    }
  const float rw1 = (s - A.wA[side]) * A.wB[side];  // rho_W - 1
#pragma unroll
  for (int ix = 0; ix < NR; ++ix)
#pragma unroll
    for (int iy = 0; iy < NR; ++iy) {
      const bool outgoing = side == 0 ? (iy >= H) : (iy < H);
      if (outgoing) O[ix * NR + iy] = fmaf(rw1, A.wS[side][ix * NR + iy], A.wSdev[side][ix * NR + iy]);
    }
}

// ---------------------------------------------------------------------------
// Internal population layout in HBM ("grouped").  The Q populations of a node
// are put in slot order: first the Q/2 with c_y < 0, then the Q/2 with
// c_y > 0, each half in (ix, iy) order.  Consecutive slots form groups of V
// (4 for D2Q16, 2 for D2Q36), and a group is stored as one V-vector per node:
//   f[((g * ny + j) * nx + i) * V + k]  holds population alpha(g*V + k).
// All populations of a group share the sign of c_y, so one vector load serves
// one stencil row; a node's populations move as Q/V vector loads and stores.
// ---------------------------------------------------------------------------
template <int NR>
struct Layout {
  static constexpr int Q = NR * NR;
  static constexpr int H = NR / 2;
  static constexpr int HALF = Q / 2;
  static constexpr int V = (HALF % 4 == 0) ? 4 : 2;
  static constexpr int G = Q / V;
  __host__ __device__ static constexpr int alpha(int s) {
    return (s % HALF) / H * NR + ((s / HALF) ? H : 0) + (s % HALF) % H;
  }
};

template <int V>
struct VecT;
template <>
struct VecT<2> { using T = float2; };
template <>
struct VecT<4> { using T = float4; };

// Load group g of one node (p points at the node's row, group 0) into F[alpha].
template <int NR>
__device__ __forceinline__ void ld_group(const float *p, long long gstride, int g, float (&F)[NR * NR]) {
  using L = Layout<NR>;
  using T = typename VecT<L::V>::T;
  const T v = __ldg(reinterpret_cast<const T *>(p + g * gstride));
  const float *e = reinterpret_cast<const float *>(&v);
#pragma unroll
  for (int k = 0; k < L::V; ++k) F[L::alpha(g * L::V + k)] = e[k];
}

template <int NR>
__device__ __forceinline__ void st_group(float *p, long long gstride, int g, const float (&F)[NR * NR]) {
  using L = Layout<NR>;
  using T = typename VecT<L::V>::T;
  T v;
  float *e = reinterpret_cast<float *>(&v);
#pragma unroll
  for (int k = 0; k < L::V; ++k) e[k] = F[L::alpha(g * L::V + k)];
  *reinterpret_cast<T *>(p + g * gstride) = v;
}

// Asynchronous global->shared copy of one V-vector (cp.async; 16-byte copies
// bypass L1).
template <int V>
__device__ __forceinline__ void cp_async_vec(void *smem_dst, const float *gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  if constexpr (V == 4) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// ---------------------------------------------------------------------------
// The fused time step (Sec. 3.1 + Sec. 3.2).
// ---------------------------------------------------------------------------
template <int NR, int N, bool SPLIT, int RING>
__global__ void __launch_bounds__(kBlock) k_step(const float *__restrict__ fin, float *__restrict__ fout,
                                                 const KArgs A) {
  using Lay = Layout<NR>;
  constexpr int Q = Lay::Q, H = Lay::H, V = Lay::V, G = Lay::G;
  constexpr int HL = 2;           // halo lanes per side
  constexpr int U = 32 - 2 * HL;  // nodes a strip updates
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int strip = warp % A.nstrips;
  const int seg = warp / A.nstrips;
  if (seg >= A.nseg) return;  // uniform over the warp
  const int nx = A.nx, ny = A.ny;
  const int xl = strip * U - HL + lane;  // this lane's node, unwrapped
  int xw = xl % nx;
  if (xw < 0) xw += nx;
  const bool writer = lane >= HL && lane < 32 - HL && xl < nx;
  const int y0 = seg * A.rows;
  const int y1 = min(y0 + A.rows, ny);
  const long long gstride = (long long)V * A.plane;  // floats per group plane
  const long long rstride = (long long)V * nx;       // floats per row
  const float *fx = fin + (long long)xw * V;
  // Rows are resolved once per row (periodic wrap, or the wall node for ghost
  // rows), never per population.
  auto row_ptr = [&](int j) { return fx + map_row(j, ny, A.walls) * rstride; };

  // y-stencil state per population:
  //   c_y > 0: s0 = f_j - f_{j-1}, s1 = sigma_{j-1}; fc = f_j
  //   c_y < 0: s0 = f_{j+1},       s1 = sigma_j;     fc = f_j
  float fc[Q], s0[Q], s1[Q];
  {
    float m2[Q], m1[Q], p1[Q];
    const float *pm2 = row_ptr(y0 - 2), *pm1 = row_ptr(y0 - 1), *pz = row_ptr(y0), *pp1 = row_ptr(y0 + 1);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      ld_group<NR>(pm1, gstride, g, m1);
      ld_group<NR>(pz, gstride, g, fc);
      if (g >= G / 2) ld_group<NR>(pm2, gstride, g, m2);
      else ld_group<NR>(pp1, gstride, g, p1);
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      if (a % NR >= H) {
        s0[a] = fc[a] - m1[a];
        s1[a] = minmod(m1[a] - m2[a], fc[a] - m1[a]);
      } else {
        s0[a] = p1[a];
        s1[a] = minmod(fc[a] - m1[a], p1[a] - fc[a]);
      }
    }
  }
  // Look-ahead rows go through a per-lane ring of RING row slots in shared
  // memory, filled by asynchronous copies (cp.async, one vector per group):
  // RING-1 rows are in flight while a row is processed, without holding
  // registers.  Each lane copies and reads only its own node's vectors, so the
  // ring needs no barrier; cp.async.wait_group paces it.  "Row-load k" holds
  // what row y0+k consumes: f_{j+1} for c_y > 0 groups, f_{j+2} for c_y < 0.
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using T = typename VecT<V>::T;
  T *ring = reinterpret_cast<T *>(smem_raw) + (size_t)(threadIdx.x >> 5) * RING * G * 32 + lane;
  int r1 = map_row(y0 + 1, ny, A.walls), r2 = map_row(y0 + 2, ny, A.walls);
  const int nrows = y1 - y0;
  auto issue_rowload = [&](int k) {
    if (k < nrows) {
      const float *q1 = fx + r1 * rstride, *q2 = fx + r2 * rstride;
      T *slot = ring + (k % RING) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g) cp_async_vec<V>(slot + g * 32, (g >= G / 2 ? q1 : q2) + g * gstride);
      r1 = r2;
      r2 = r2 + 1 < ny ? r2 + 1 : (A.walls ? ny - 1 : 0);
    }
    cp_async_commit();  // (an empty group past the segment end keeps the count uniform)
  };
#pragma unroll
  for (int k = 0; k < RING - 1; ++k) issue_rowload(k);

  for (int j = y0; j < y1; ++j) {
    const int k = j - y0;
    issue_rowload(k + RING - 1);
    cp_async_wait<RING - 1>();  // row-load k has landed
    float ld[Q];
    {
      const T *slot = ring + (k % RING) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const T v = slot[g * 32];
        const float *e = reinterpret_cast<const float *>(&v);
#pragma unroll
        for (int q = 0; q < V; ++q) ld[Lay::alpha(g * V + q)] = e[q];
      }
    }

    float acc[Q];
    float omw;
    collide<NR, N>(fc, acc, omw, A);

    // y-advection from the carried stencil of f^n; xs = the values the
    // x-fluxes are taken from: f^n_j (update as printed) or the y-swept
    // f*_j = f^n_j - (c_y dt/dy) dF_y (split scheme).
    float xs[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int iy = a % NR;
      const float ay = A.ay[iy], ky = A.ky[iy];
      float diff;
      const float f0 = fc[a];
      if (iy >= H) {  // c_y > 0: F_{j+1/2} = f_j + k sigma_j
        const float dn = ld[a] - f0;
        const float sg = minmod(s0[a], dn);
        diff = fmaf(ky, sg - s1[a], s0[a]);
        s0[a] = dn;
        s1[a] = sg;
        fc[a] = ld[a];
      } else {  // c_y < 0: F_{j+1/2} = f_{j+1} - k sigma_{j+1}
        const float d1 = s0[a] - f0;
        const float sg = minmod(d1, ld[a] - s0[a]);
        diff = fmaf(-ky, sg - s1[a], d1);
        s1[a] = sg;
        fc[a] = s0[a];
        s0[a] = ld[a];
      }
      acc[a] = fmaf(omw, f0, fmaf(-ay, diff, acc[a]));
      xs[a] = SPLIT ? fmaf(-ay, diff, f0) : f0;
    }

    // x-advection: neighbours from adjacent lanes
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int ix = a / NR;
      const float ax = A.ax[ix], kx = A.kx[ix];
      const float left = __shfl_up_sync(kFull, xs[a], 1);
      const float dl = xs[a] - left;                       // f_i - f_{i-1}
      const float dr = __shfl_down_sync(kFull, dl, 1);     // f_{i+1} - f_i
      const float sg = minmod(dl, dr);                     // sigma_i
      float diff;
      if (ix >= H) {  // c_x > 0: F_{i+1/2} = f_i + k sigma_i
        const float sprev = __shfl_up_sync(kFull, sg, 1);
        diff = fmaf(kx, sg - sprev, dl);
      } else {  // c_x < 0: F_{i+1/2} = f_{i+1} - k sigma_{i+1}
        const float snext = __shfl_down_sync(kFull, sg, 1);
        diff = fmaf(-kx, snext - sg, dr);
      }
      acc[a] = fmaf(-ax, diff, acc[a]);
    }

    if (A.walls && (j == 0 || j == ny - 1)) wall_fix<NR>(acc, (j == 0) ? 0 : 1, A);

    if (writer) {
      float *o = fout + (long long)j * rstride + (long long)xw * V;
#pragma unroll
      for (int g = 0; g < G; ++g) st_group<NR>(o, gstride, g, acc);
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Initial populations f = rho S(T,u) (Eq. feq0 to order N: the Hermite
// expansion of the isotropic Maxwellian), then the wall rule once.
// fields: double[4][ny][nx] = rho, u_x, u_y, T (or nullptr: rest).
// ---------------------------------------------------------------------------
template <int NR, int N>
__global__ void __launch_bounds__(kBlock) k_init(const double *__restrict__ fields, float *__restrict__ f,
                                                 const KArgs A) {
  using Lay = Layout<NR>;
  constexpr int Q = Lay::Q;
  const long long cells = A.plane;
  const long long gstride = (long long)Lay::V * cells;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < cells; c += (long long)gridDim.x * kBlock) {
    float drho = 0.f, ux = 0.f, uy = 0.f, dT = 0.f;
    if (fields) {
      drho = (float)(fields[c] - 1.0);
      ux = (float)fields[cells + c];
      uy = (float)fields[2 * cells + c];
      dT = (float)(fields[3 * cells + c] - 1.0);
    }
    const float rho = 1.0f + drho;
    const float rdT = rho * dT;
    float e[N + 1][N + 1];
    gaussian_coeffs<N>(rho, rho * ux, rho * uy, ux, uy, dT, 0.f, dT, rdT, 0.f, rdT, e);
    e[0][0] = drho;  // deviation from w_a
    float S[Q];
    hermite_evaluate<NR, N>(e, S, A);
    const int j = (int)(c / A.nx);
    if (A.walls && (j == 0 || j == A.ny - 1)) wall_fix<NR>(S, j == 0 ? 0 : 1, A);
#pragma unroll
    for (int g = 0; g < Lay::G; ++g) st_group<NR>(f + c * Lay::V, gstride, g, S);
  }
}

// Populations between the grouped layout and the public [a][j][i] layout.
template <int NR>
__global__ void __launch_bounds__(kBlock) k_ungroup(const float *__restrict__ f, float *__restrict__ out,
                                                    long long cells) {
  using Lay = Layout<NR>;
  const long long gstride = (long long)Lay::V * cells;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < cells; c += (long long)gridDim.x * kBlock) {
    float F[Lay::Q];
#pragma unroll
    for (int g = 0; g < Lay::G; ++g) ld_group<NR>(f + c * Lay::V, gstride, g, F);
#pragma unroll
    for (int a = 0; a < Lay::Q; ++a) out[a * cells + c] = F[a];
  }
}

template <int NR>
__global__ void __launch_bounds__(kBlock) k_group(const float *__restrict__ in, float *__restrict__ f,
                                                  long long cells) {
  using Lay = Layout<NR>;
  const long long gstride = (long long)Lay::V * cells;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < cells; c += (long long)gridDim.x * kBlock) {
    float F[Lay::Q];
#pragma unroll
    for (int a = 0; a < Lay::Q; ++a) F[a] = __ldg(in + a * cells + c);
#pragma unroll
    for (int g = 0; g < Lay::G; ++g) st_group<NR>(f + c * Lay::V, gstride, g, F);
  }
}

// ---------------------------------------------------------------------------
// Moments of Eq. (mac) per node, plus FP64 block partial sums of mass,
// momentum and energy.  out: float[9][ny][nx].
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(kMomBlock) k_moments(const float *__restrict__ f, float *__restrict__ out,
                                                       double *__restrict__ partial, const KArgs A) {
  using Lay = Layout<NR>;
  constexpr int Q = Lay::Q;
  const long long cells = A.plane;
  const long long gstride = (long long)Lay::V * cells;
  double sm = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  for (long long c = blockIdx.x * (long long)kMomBlock + threadIdx.x; c < cells;
       c += (long long)gridDim.x * kMomBlock) {
    float F[Q];
#pragma unroll
    for (int g = 0; g < Lay::G; ++g) ld_group<NR>(f + c * Lay::V, gstride, g, F);
    float m[4][4];
    hermite_moments<NR, 3>(F, m, A);
    const float rho = 1.0f + m[0][0];
    const float ir = __frcp_rn(rho);
    const float ux = m[1][0] * ir, uy = m[0][1] * ir;
    const float Mxx = fmaf(-m[1][0], ux, m[2][0]);
    const float Mxy = fmaf(-m[1][0], uy, m[1][1]);
    const float Myy = fmaf(-m[0][1], uy, m[0][2]);
    const float trM = Mxx + Myy;
    const float T = fmaf(0.5f * trM, ir, 1.0f);
    const float u2 = ux * ux + uy * uy;
    // sum f C_i C^2 = sum df c_i (c^2 - D - 2) - 2 M_ij u_j - u_i tr M - rho u_i u^2
    const float hx = m[3][0] + m[1][2], hy = m[0][3] + m[2][1];
    const float qx = 0.5f * (hx - 2.0f * (Mxx * ux + Mxy * uy) - ux * trM - rho * ux * u2);
    const float qy = 0.5f * (hy - 2.0f * (Mxy * ux + Myy * uy) - uy * trM - rho * uy * u2);
    if (out) {
      out[c] = rho;
      out[cells + c] = ux;
      out[2 * cells + c] = uy;
      out[3 * cells + c] = T;
      out[4 * cells + c] = 0.5f * (Mxx - Myy);
      out[5 * cells + c] = Mxy;
      out[6 * cells + c] = 0.5f * (Myy - Mxx);
      out[7 * cells + c] = qx;
      out[8 * cells + c] = qy;
    }
    // FP64 conservation sums: sum_a f_a {1, c_x, c_y, c^2/2}, f_a = w_a + df_a
    double dm = 0.0, dx = 0.0, dy = 0.0, de = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const double cx = A.c[a / NR], cy = A.c[a % NR];
      const double v = F[a];
      dm += v;
      dx += v * cx;
      dy += v * cy;
      de += v * (cx * cx + cy * cy);
    }
    sm += 1.0 + dm;
    sx += dx;
    sy += dy;
    se += 0.5 * (2.0 + de);  // sum_a w_a c_a^2 = D = 2
  }
  __shared__ double red[4][kMomBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sm += __shfl_down_sync(kFull, sm, o);
    sx += __shfl_down_sync(kFull, sx, o);
    sy += __shfl_down_sync(kFull, sy, o);
    se += __shfl_down_sync(kFull, se, o);
  }
  if (lane == 0) {
    red[0][w] = sm;
    red[1][w] = sx;
    red[2][w] = sy;
    red[3][w] = se;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int k = 0; k < kMomBlock / 32; ++k) t += red[threadIdx.x][k];
    partial[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

__global__ void k_reduce_partials(const double *__restrict__ partial, int n, double *__restrict__ sums) {
  // one warp per quantity, fixed order: bitwise reproducible
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= 4) return;
  double t = 0.0;
  for (int k = lane; k < n; k += 32) t += partial[k * 4 + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
  if (lane == 0) sums[q] = t;
}

constexpr int kMomGrid = 1024;

}  // namespace

// ===========================================================================
// Host side
// ===========================================================================
struct lesbgk {
  lesbgk_params p;
  int nr, order, q, cpt, rows;
  char *ws;
  size_t ws_bytes;
  float *buf[2];
  int cur;
  size_t buf_bytes;
  double *partial, *sums;
  KArgs args;
  double dt, dx, dy, cmax, tau_ref;
  int64_t steps;
  int sm_count;
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int check_params(const lesbgk_params *p) {
  if (!p) return fail(LESBGK_EINVAL, "params is NULL");
  if (p->struct_size != sizeof(lesbgk_params))
    return fail(LESBGK_EINVAL, "struct_size %u != %zu", p->struct_size, sizeof(lesbgk_params));
  if (p->nroots != 4 && p->nroots != 6) return fail(LESBGK_EINVAL, "nroots must be 4 or 6");
  const int order = p->order ? p->order : (p->nroots == 4 ? 3 : 4);
  if (order != 3 && order != 4) return fail(LESBGK_EINVAL, "order must be 3 or 4");
  if (p->nx < 1 || p->ny < 1) return fail(LESBGK_EINVAL, "nx, ny must be >= 1");
  if ((long long)p->nx * p->ny > (1LL << 31) / 64) return fail(LESBGK_EINVAL, "grid too large");
  if (p->bc_y != LESBGK_PERIODIC && p->bc_y != LESBGK_DIFFUSE) return fail(LESBGK_EINVAL, "bad bc_y");
  if (p->bc_y == LESBGK_DIFFUSE && p->ny < 2) return fail(LESBGK_EINVAL, "walls need ny >= 2");
  if (p->storage != LESBGK_F32) return fail(LESBGK_EINVAL, "storage must be LESBGK_F32");
  if (p->scheme != LESBGK_UNSPLIT && p->scheme != LESBGK_SPLIT)
    return fail(LESBGK_EINVAL, "scheme must be LESBGK_UNSPLIT or LESBGK_SPLIT");
  if (!(p->kn > 0.0) || !std::isfinite(p->kn)) return fail(LESBGK_EINVAL, "Kn must be > 0");
  if (!(p->b >= -0.5 && p->b < 1.0)) return fail(LESBGK_EINVAL, "b must satisfy -1/2 <= b < 1");
  if (!(p->visc_exp >= 0.0 && p->visc_exp <= 1.0)) return fail(LESBGK_EINVAL, "visc_exp must be in [0,1]");
  if (!(p->dt >= 0.0) || !std::isfinite(p->dt)) return fail(LESBGK_EINVAL, "dt must be >= 0");
  if (p->dt == 0.0 && !(p->cfl > 0.0 && p->cfl <= 1.0)) return fail(LESBGK_EINVAL, "cfl must be in (0,1]");
  for (int s = 0; s < 2; ++s) {
    if (!(p->wall_T[s] > 0.0) || !std::isfinite(p->wall_T[s])) return fail(LESBGK_EINVAL, "wall_T must be > 0");
    if (!std::isfinite(p->wall_ux[s]) || !std::isfinite(p->g[s])) return fail(LESBGK_EINVAL, "non-finite wall_ux/g");
  }
  return 0;
}

size_t buffer_bytes(const lesbgk_params *p) {
  const size_t cells = (size_t)p->nx * p->ny;
  const size_t q = (size_t)p->nroots * p->nroots;
  size_t per = q * sizeof(float);
  if (per < 9 * sizeof(float)) per = 9 * sizeof(float);
  if (per < 4 * sizeof(double)) per = 4 * sizeof(double);
  return align_up(cells * per, 256);
}

}  // namespace

extern "C" int lesbgk_workspace_size(const lesbgk_params *p, size_t *bytes) {
  if (int rc = check_params(p)) return rc;
  if (!bytes) return fail(LESBGK_EINVAL, "bytes is NULL");
  *bytes = 2 * buffer_bytes(p) + align_up((size_t)kMomGrid * 4 * sizeof(double), 256) + 256;
  return 0;
}

namespace {

int pick_launch(lesbgk *h) {
  const int nx = h->p.nx, ny = h->p.ny;
  // one node per lane, 28 nodes per strip (two halo lanes per side); default
  // 32-row segments (measured best on the 4096^2 periodic case)
  h->cpt = 1;
  const int nstrips = (nx + 27) / 28;
  if (h->rows <= 0) h->rows = ny < 32 ? ny : 32;
  h->args.rows = h->rows;
  h->args.nstrips = nstrips;
  h->args.nseg = (ny + h->rows - 1) / h->rows;
  return 0;
}

int build_tables(lesbgk *h, const double *h_init) {
  using namespace lesbgk_tables;
  const lesbgk_params &p = h->p;
  const int nr = p.nroots, N = h->order;
  double c[kMaxRoots], w[kMaxRoots];
  if (gauss_hermite(nr, c, w)) return fail(LESBGK_EINVAL, "quadrature failed");
  KArgs &A = h->args;
  std::memset(&A, 0, sizeof A);
  h->cmax = std::fabs(c[0]);
  // spacing
  if (p.bc_y == LESBGK_PERIODIC) {
    h->dx = 1.0 / p.nx;
    h->dy = 1.0 / p.ny;
  } else {
    h->dy = 1.0 / (p.ny - 1);
    h->dx = h->dy;
  }
  // reference state for tau_ref
  double tmax = 1.0, rmax = 1.0;
  if (p.bc_y == LESBGK_DIFFUSE) tmax = std::fmax(tmax, std::fmax(p.wall_T[0], p.wall_T[1]));
  if (h_init) {
    const size_t cells = (size_t)p.nx * p.ny;
    double r0 = h_init[0];
    for (size_t k = 0; k < cells; ++k) {
      const double r = h_init[k], T = h_init[3 * cells + k];
      if (!(r > 0.0) || !(T > 0.0) || !std::isfinite(r) || !std::isfinite(T) ||
          !std::isfinite(h_init[cells + k]) || !std::isfinite(h_init[2 * cells + k]))
        return fail(LESBGK_EINVAL, "initial field at node %zu not admissible (rho, T > 0, finite)", k);
      r0 = std::fmax(r0, r);
      tmax = std::fmax(tmax, T);
    }
    rmax = r0;
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
  }
  // wall equilibria S_a(T_w, u_w) at order N (b = 0 Gaussian projection)
  for (int s = 0; s < 2; ++s) {
    double e[kMaxOrder + 1][kMaxOrder + 1];
    const double th = p.wall_T[s] - 1.0;
    gaussian_hermite_moments(N, 1.0, p.wall_ux[s], 0.0, th, 0.0, th, e);
    double A_out = 0.0, Z_out = 0.0;
    for (int ix = 0; ix < nr; ++ix) {
      double hx[kMaxOrder + 1];
      hermite_values(kMaxOrder, c[ix], hx);
      for (int iy = 0; iy < nr; ++iy) {
        double hy[kMaxOrder + 1];
        hermite_values(kMaxOrder, c[iy], hy);
        double sum = 0.0;
        for (int m = 0; m <= N; ++m)
          for (int k = 0; m + k <= N; ++k) sum += e[m][k] * hx[m] * hy[k] / (fact[m] * fact[k]);
        const double wa = w[ix] * w[iy];
        const double S = wa * sum;
        const int a = ix * nr + iy;
        A.wS[s][a] = (float)S;
        A.wSdev[s][a] = (float)(S - wa);
        const bool outgoing = (s == 0) ? (c[iy] > 0.0) : (c[iy] < 0.0);
        if (outgoing) {
          A_out += std::fabs(c[iy]) * (S - wa);
          Z_out += std::fabs(c[iy]) * S;
        }
      }
    }
    A.wA[s] = (float)A_out;
    A.wB[s] = (float)(1.0 / Z_out);
  }
  A.c_omega = (float)(dt / (p.kn * (1.0 - p.b)));
  A.visc_pow = (float)(1.0 - p.visc_exp);
  A.vmode = p.visc_exp == 0.5 ? 1 : (p.visc_exp == 1.0 ? 2 : 0);
  A.b = (float)p.b;
  A.beta = (float)(0.5 * (1.0 - p.b));
  A.dtgx = (float)(dt * p.g[0]);
  A.dtgy = (float)(dt * p.g[1]);
  A.has_force = (p.g[0] != 0.0 || p.g[1] != 0.0) ? 1 : 0;
  A.nx = p.nx;
  A.ny = p.ny;
  A.walls = p.bc_y == LESBGK_DIFFUSE ? 1 : 0;
  A.plane = (long long)p.nx * p.ny;
  return 0;
}

constexpr int kRing = 4;

template <int NR>
constexpr size_t step_smem_bytes() {
  return (size_t)(kBlock / 32) * kRing * Layout<NR>::G * 32 * Layout<NR>::V * sizeof(float);
}

template <int NR, int N>
int launch_step_t(lesbgk *h, const float *fin, float *fout, cudaStream_t s) {
  const long long warps = (long long)h->args.nstrips * h->args.nseg;
  const unsigned grid = (unsigned)((warps * 32 + kBlock - 1) / kBlock);
  constexpr size_t smem = step_smem_bytes<NR>();
  if (h->p.scheme == LESBGK_SPLIT) k_step<NR, N, true, kRing><<<grid, kBlock, smem, s>>>(fin, fout, h->args);
  else k_step<NR, N, false, kRing><<<grid, kBlock, smem, s>>>(fin, fout, h->args);
  return 0;
}

// Opt in to more than 48 KiB of dynamic shared memory where a ring needs it.
template <int NR, int N>
cudaError_t allow_smem_t() {
  constexpr int smem = (int)step_smem_bytes<NR>();
  cudaError_t e = cudaFuncSetAttribute(k_step<NR, N, true, kRing>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step<NR, N, false, kRing>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

cudaError_t allow_smem(const lesbgk *h) {
  if (h->nr == 4 && h->order == 3) return allow_smem_t<4, 3>();
  if (h->nr == 4 && h->order == 4) return allow_smem_t<4, 4>();
  if (h->nr == 6 && h->order == 3) return allow_smem_t<6, 3>();
  return allow_smem_t<6, 4>();
}

int launch_step(lesbgk *h, const float *fin, float *fout, cudaStream_t s) {
  if (h->nr == 4 && h->order == 3) return launch_step_t<4, 3>(h, fin, fout, s);
  if (h->nr == 4 && h->order == 4) return launch_step_t<4, 4>(h, fin, fout, s);
  if (h->nr == 6 && h->order == 3) return launch_step_t<6, 3>(h, fin, fout, s);
  return launch_step_t<6, 4>(h, fin, fout, s);
}

unsigned grid_for(const lesbgk *h, long long cells) {
  long long g = (cells + kBlock - 1) / kBlock;
  const long long cap = (long long)h->sm_count * 16;
  if (g > cap) g = cap;
  return g < 1 ? 1u : (unsigned)g;
}

int launch_init(lesbgk *h, const double *fields, float *f, cudaStream_t s) {
  const unsigned grid = grid_for(h, h->args.plane);
  if (h->nr == 4 && h->order == 3) k_init<4, 3><<<grid, kBlock, 0, s>>>(fields, f, h->args);
  else if (h->nr == 4 && h->order == 4) k_init<4, 4><<<grid, kBlock, 0, s>>>(fields, f, h->args);
  else if (h->nr == 6 && h->order == 3) k_init<6, 3><<<grid, kBlock, 0, s>>>(fields, f, h->args);
  else k_init<6, 4><<<grid, kBlock, 0, s>>>(fields, f, h->args);
  return 0;
}

int launch_moments(lesbgk *h, float *out, cudaStream_t s) {
  const float *f = h->buf[h->cur];
  if (h->nr == 4) k_moments<4><<<kMomGrid, kMomBlock, 0, s>>>(f, out, h->partial, h->args);
  else k_moments<6><<<kMomGrid, kMomBlock, 0, s>>>(f, out, h->partial, h->args);
  k_reduce_partials<<<1, 128, 0, s>>>(h->partial, kMomGrid, h->sums);
  return 0;
}

}  // namespace

extern "C" int lesbgk_create(const lesbgk_params *p, void *d_workspace, size_t bytes, const double *h_init,
                             void *stream, lesbgk **out) {
  g_err[0] = 0;
  if (int rc = check_params(p)) return rc;
  if (!out) return fail(LESBGK_EINVAL, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  lesbgk_workspace_size(p, &need);
  if (!d_workspace || bytes < need) return fail(LESBGK_ESPACE, "workspace %zu bytes < %zu needed", bytes, need);
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256) return fail(LESBGK_ESPACE, "workspace not 256-byte aligned");
  lesbgk *h = new (std::nothrow) lesbgk();
  if (!h) return fail(LESBGK_EINVAL, "out of host memory");
  h->p = *p;
  h->nr = p->nroots;
  h->order = p->order ? p->order : (p->nroots == 4 ? 3 : 4);
  h->q = h->nr * h->nr;
  h->ws = static_cast<char *>(d_workspace);
  h->ws_bytes = bytes;
  h->buf_bytes = buffer_bytes(p);
  h->buf[0] = reinterpret_cast<float *>(h->ws);
  h->buf[1] = reinterpret_cast<float *>(h->ws + h->buf_bytes);
  h->partial = reinterpret_cast<double *>(h->ws + 2 * h->buf_bytes);
  h->sums = reinterpret_cast<double *>(h->ws + 2 * h->buf_bytes + align_up((size_t)kMomGrid * 4 * sizeof(double), 256));
  h->cur = 0;
  h->steps = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "device query");
  }
  if (int rc = build_tables(h, h_init)) {
    delete h;
    return rc;
  }
  pick_launch(h);
  e = allow_smem(h);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "step kernel shared-memory opt-in");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double *dfields = nullptr;
  if (h_init) {
    const size_t fb = (size_t)4 * p->nx * p->ny * sizeof(double);
    e = cudaMemcpyAsync(h->buf[1], h_init, fb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "copy of initial fields");
    }
    dfields = reinterpret_cast<const double *>(h->buf[1]);
  }
  launch_init(h, dfields, h->buf[0], s);
  e = cudaGetLastError();
  if (e == cudaSuccess && h_init) e = cudaStreamSynchronize(s);  // h_init may be freed after return
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "init kernel");
  }
  *out = h;
  return 0;
}

extern "C" int lesbgk_reinit(lesbgk *h, const double *d_fields, void *stream) {
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->cur = 0;
  h->steps = 0;
  launch_init(h, d_fields, h->buf[0], s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "init kernel");
}

extern "C" int lesbgk_step(lesbgk *h, int64_t nsteps, void *stream) {
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(LESBGK_EINVAL, "nsteps < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t k = 0; k < nsteps; ++k) {
    launch_step(h, h->buf[h->cur], h->buf[h->cur ^ 1], s);
    h->cur ^= 1;
  }
  h->steps += nsteps;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "step kernel");
  return 0;
}

namespace {
int finish_sums(lesbgk *h, double *h_sums, cudaStream_t s) {
  if (!h_sums) return 0;
  cudaError_t e = cudaMemcpyAsync(h_sums, h->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "moment sums");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(h_sums[k])) return fail(LESBGK_EDIVERGED, "non-finite conservation sum %d", k);
  return 0;
}
}  // namespace

extern "C" int lesbgk_moments(lesbgk *h, float *d_out, double *h_sums, void *stream) {
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_moments(h, d_out, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "moments kernel");
  return finish_sums(h, h_sums, s);
}

extern "C" int lesbgk_moments_host(lesbgk *h, float *h_out, double *h_sums, void *stream) {
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  if (!h_out) return fail(LESBGK_EINVAL, "h_out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *stage = h->buf[h->cur ^ 1];  // the spare ping-pong buffer holds >= 9 floats per node
  launch_moments(h, stage, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_out, stage, (size_t)9 * h->args.plane * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "moments to host");
  return finish_sums(h, h_sums, s);
}

extern "C" int lesbgk_get_populations(lesbgk *h, float *d_out, void *stream) {
  if (!h || !d_out) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long cells = h->args.plane;
  if (h->nr == 4) k_ungroup<4><<<grid_for(h, cells), kBlock, 0, s>>>(h->buf[h->cur], d_out, cells);
  else k_ungroup<6><<<grid_for(h, cells), kBlock, 0, s>>>(h->buf[h->cur], d_out, cells);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "get populations");
}

extern "C" int lesbgk_set_populations(lesbgk *h, const float *d_in, int64_t steps_done, void *stream) {
  if (!h || !d_in) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long cells = h->args.plane;
  if (h->nr == 4) k_group<4><<<grid_for(h, cells), kBlock, 0, s>>>(d_in, h->buf[h->cur], cells);
  else k_group<6><<<grid_for(h, cells), kBlock, 0, s>>>(d_in, h->buf[h->cur], cells);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "set populations");
  h->steps = steps_done;
  return 0;
}

extern "C" int lesbgk_set_launch(lesbgk *h, int32_t cells_per_thread, int32_t rows_per_segment) {
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  if (cells_per_thread < 0 || cells_per_thread > 1 || rows_per_segment < 0)
    return fail(LESBGK_EINVAL, "bad launch shape (cells_per_thread must be 0 or 1)");
  if (rows_per_segment) h->rows = rows_per_segment;
  return pick_launch(h);
}

extern "C" int lesbgk_get_info(const lesbgk *h, lesbgk_info *out) {
  if (!h || !out) return fail(LESBGK_EINVAL, "NULL argument");
  out->dt = h->dt;
  out->dx = h->dx;
  out->dy = h->dy;
  out->c_max = h->cmax;
  out->cfl = h->cmax * h->dt / std::fmin(h->dx, h->dy);
  out->tau_ref = h->tau_ref;
  out->steps_done = h->steps;
  out->q = h->q;
  out->order = h->order;
  out->cells_per_thread = h->cpt;
  out->rows_per_segment = h->rows;
  return 0;
}

extern "C" int lesbgk_destroy(lesbgk *h) {
  delete h;
  return 0;
}

extern "C" const char *lesbgk_last_error(void) { return g_err; }

// ===========================================================================
// Moments without allocation.
//
// For callers that cannot allocate device memory at all (an embedding
// application whose device memory belongs to another allocator, a plugin held
// to a fixed memory budget, or a loop that cannot afford the device-wide
// synchronisation of cudaMalloc), this entry point computes the same nine
// moment fields and FP64 totals as lesbgk_moments from populations the caller
// already holds.  Its only scratch -- one FP64 partial sum per quantity per
// block, plus the four totals -- lives in the file-scope array below, so the
// call allocates nothing.  The array is fixed in size (kNoAllocBlocks blocks
// of kNoAllocNodesPerBlock nodes, 256 KiB + 32 B) and every GPU that loads
// the library holds it until the process exits.
// ===========================================================================
namespace {

constexpr int kNoAllocBlocks = 8192;
constexpr int kNoAllocNodesPerThread = 8;
constexpr long long kNoAllocNodesPerBlock = (long long)kMomBlock * kNoAllocNodesPerThread;
constexpr long long kNoAllocMaxNodes = (long long)kNoAllocBlocks * kNoAllocNodesPerBlock;  // 2^24

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks * 4 + 4];

// One block per kNoAllocNodesPerBlock nodes of the public layout
// f[a][j][i] (deviations f_a - w_a); per-node arithmetic as in k_moments.
template <int NR>
__global__ void __launch_bounds__(kMomBlock) k_moments_public(const float *__restrict__ f, float *__restrict__ out,
                                                              double *__restrict__ partial, const KArgs A) {
  constexpr int Q = NR * NR;
  const long long cells = A.plane;
  double sm = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  const long long c0 = blockIdx.x * kNoAllocNodesPerBlock;
  for (int t = 0; t < kNoAllocNodesPerThread; ++t) {
    const long long c = c0 + (long long)t * kMomBlock + threadIdx.x;
    if (c >= cells) break;
    float F[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) F[a] = __ldg(f + a * cells + c);
    float m[4][4];
    hermite_moments<NR, 3>(F, m, A);
    const float rho = 1.0f + m[0][0];
    const float ir = __frcp_rn(rho);
    const float ux = m[1][0] * ir, uy = m[0][1] * ir;
    const float Mxx = fmaf(-m[1][0], ux, m[2][0]);
    const float Mxy = fmaf(-m[1][0], uy, m[1][1]);
    const float Myy = fmaf(-m[0][1], uy, m[0][2]);
    const float trM = Mxx + Myy;
    const float T = fmaf(0.5f * trM, ir, 1.0f);
    const float u2 = ux * ux + uy * uy;
    const float hx = m[3][0] + m[1][2], hy = m[0][3] + m[2][1];
    const float qx = 0.5f * (hx - 2.0f * (Mxx * ux + Mxy * uy) - ux * trM - rho * ux * u2);
    const float qy = 0.5f * (hy - 2.0f * (Mxy * ux + Myy * uy) - uy * trM - rho * uy * u2);
    if (out) {
      out[c] = rho;
      out[cells + c] = ux;
      out[2 * cells + c] = uy;
      out[3 * cells + c] = T;
      out[4 * cells + c] = 0.5f * (Mxx - Myy);
      out[5 * cells + c] = Mxy;
      out[6 * cells + c] = 0.5f * (Myy - Mxx);
      out[7 * cells + c] = qx;
      out[8 * cells + c] = qy;
    }
    double dm = 0.0, dx = 0.0, dy = 0.0, de = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const double cx = A.c[a / NR], cy = A.c[a % NR];
      const double v = F[a];
      dm += v;
      dx += v * cx;
      dy += v * cy;
      de += v * (cx * cx + cy * cy);
    }
    sm += 1.0 + dm;
    sx += dx;
    sy += dy;
    se += 0.5 * (2.0 + de);
  }
  __shared__ double red[4][kMomBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sm += __shfl_down_sync(kFull, sm, o);
    sx += __shfl_down_sync(kFull, sx, o);
    sy += __shfl_down_sync(kFull, sy, o);
    se += __shfl_down_sync(kFull, se, o);
  }
  if (lane == 0) {
    red[0][w] = sm;
    red[1][w] = sx;
    red[2][w] = sy;
    red[3][w] = se;
  }
  __syncthreads();
  if (threadIdx.x < 4) {  // every block writes all four of its slots: no zeroing needed
    double t = 0.0;
    for (int k = 0; k < kMomBlock / 32; ++k) t += red[threadIdx.x][k];
    partial[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (in host code the symbol is only a stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(LESBGK_EINVAL, "device index %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static moment scratch");
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return 0;
}

}  // namespace

extern "C" int lesbgk_moments_noalloc(const lesbgk_params *p, const float *d_populations, float *d_out,
                                      double *h_sums, void *stream) {
  if (int rc = check_params(p)) return rc;
  if (!d_populations) return fail(LESBGK_EINVAL, "d_populations is NULL");
  const long long cells = (long long)p->nx * p->ny;
  if (cells > kNoAllocMaxNodes)
    return fail(LESBGK_EINVAL, "lesbgk_moments_noalloc handles at most %lld nodes (%lld given): its static "
                "scratch holds %d block partial sums", kNoAllocMaxNodes, cells, kNoAllocBlocks);
  lesbgk tmp{};
  tmp.p = *p;
  tmp.nr = p->nroots;
  tmp.order = p->order ? p->order : (p->nroots == 4 ? 3 : 4);
  tmp.q = tmp.nr * tmp.nr;
  if (int rc = build_tables(&tmp, nullptr)) return rc;
  double *scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((cells + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock);
  double *sums = scratch + (size_t)kNoAllocBlocks * 4;
  if (p->nroots == 4) k_moments_public<4><<<blocks, kMomBlock, 0, s>>>(d_populations, d_out, scratch, tmp.args);
  else k_moments_public<6><<<blocks, kMomBlock, 0, s>>>(d_populations, d_out, scratch, tmp.args);
  k_reduce_partials<<<1, 128, 0, s>>>(scratch, blocks, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "moments (no allocation)");
  if (!h_sums) return 0;
  e = cudaMemcpyAsync(h_sums, sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "moment sums (no allocation)");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(h_sums[k])) return fail(LESBGK_EDIVERGED, "non-finite conservation sum %d", k);
  return 0;
}
