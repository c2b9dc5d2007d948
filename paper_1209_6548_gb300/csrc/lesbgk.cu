// liblesbgk: GB300 (sm_103a) lattice ES-BGK solver behind the C ABI of
// include/lesbgk.h.  Method: Meng, Zhang, Hadjiconstantinou, Radtke & Shan,
// arXiv 1209.6548 (Sec. 2.2 lattice ES-BGK equation, Sec. 3.1 scheme,
// Sec. 3.2 walls, Sec. 4.2 heated walls).
//
// Data layout in HBM: populations as deviations df_a = f_a - w_a (FP32, or
// 16-bit relative deviations), in the grouped layout of Layout<NR, S, NZ>
// (device.cuh: vectors of 2, 4 or 8 populations of one node that share the
// sign of c_y), two ping-pong buffers in the caller's workspace.  The D = 3
// sets store their z-even half.  One time step = one launch of k_step (or
// k_step_z for D3Q216).
//
// k_step mapping: a warp owns a strip of 32 consecutive x-nodes (the two
// outer lanes on each side are halo lanes that load but do not store) and
// marches up a segment of rows.  x-neighbours come from warp shuffles, the
// y-stencil is carried in registers from row to row, so each population is
// read from HBM once and written once per step (plus halo strips/rows that
// hit in L2).  Per node, all stored values live in one thread: moments,
// collision, Hermite evaluation and the wall reduction are in-thread.  The
// D3Q216 step spreads a node's three stored z-levels over three warps.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>

#include "lesbgk.h"
#include "device.cuh"
#include "internal.h"
#include "setup.h"

namespace {

using namespace lesbgk_dev;
using namespace lesbgk_setup;

constexpr int kBlock = 128;
constexpr int kMomBlock = 256;



// ---------------------------------------------------------------------------
// The fused time step (Sec. 3.1 + Sec. 3.2).
// ---------------------------------------------------------------------------
template <int NR, int N, bool SPLIT, int RING, class S, int WM, int NZ = 1>
__global__ void __launch_bounds__(kBlock) k_step(const S *__restrict__ fin, S *__restrict__ fout,
                                                 const KArgs A) {
  using Lay = Layout<NR, S, NZ>;
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
  int xw;
  if constexpr (WM == 2) {
    xw = min(max(xl, 0), nx - 1);  // walls in x: ghost columns hold the wall node
  } else {
    xw = xl % nx;
    if (xw < 0) xw += nx;
  }
  const bool writer = lane >= HL && lane < 32 - HL && xl < nx;
  const int y0 = seg * A.rows;
  const int y1 = min(y0 + A.rows, ny);
  const long long gstride = (long long)V * A.plane;  // elements per group plane
  const long long rstride = (long long)V * nx;       // elements per row
  const S *fx = fin + (long long)xw * V;
  // Rows are resolved once per row (periodic wrap, or the wall node for ghost
  // rows), never per population.
  auto row_ptr = [&](int j) { return fx + map_row(j, ny, A.walls) * rstride; };

  // y-stencil state per population:
  //   c_y > 0: s0 = f_j - f_{j-1}, s1 = sigma_{j-1}; fc = f_j
  //   c_y < 0: s0 = f_{j+1},       s1 = sigma_j;     fc = f_j
  float fc[Q], s0[Q], s1[Q];
  {
    float m2[Q], m1[Q], p1[Q];
    const S *pm2 = row_ptr(y0 - 2), *pm1 = row_ptr(y0 - 1), *pz = row_ptr(y0), *pp1 = row_ptr(y0 + 1);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      ld_group_s<NR, S>(pm1, gstride, g, m1, A);
      ld_group_s<NR, S>(pz, gstride, g, fc, A);
      if (g >= G / 2) ld_group_s<NR, S>(pm2, gstride, g, m2, A);
      else ld_group_s<NR, S>(pp1, gstride, g, p1, A);
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
  using T = typename Raw<Lay::VB>::T;
  T *ring = reinterpret_cast<T *>(smem_raw) + (size_t)(threadIdx.x >> 5) * RING * G * 32 + lane;
  int r1 = map_row(y0 + 1, ny, A.walls), r2 = map_row(y0 + 2, ny, A.walls);
  const int nrows = y1 - y0;
  auto issue_rowload = [&](int k) {
    if (k < nrows) {
      const S *q1 = fx + r1 * rstride, *q2 = fx + r2 * rstride;
      T *slot = ring + (k % RING) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g) cp_async_raw<Lay::VB>(slot + g * 32, (g >= G / 2 ? q1 : q2) + g * gstride);
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
      for (int g = 0; g < G; ++g) unpack_group<NR, S>(slot[g * 32], g, ld, A);
    }

    float acc[Q];
    float omw;
    collide_any<NR, N>(fc, acc, omw, A, A);

    // y-advection from the carried stencil of f^n; xs = the values the
    // x-fluxes are taken from: f^n_j (update as printed) or the y-swept
    // f*_j = f^n_j - (c_y dt/dy) dF_y (split scheme).  Both sweeps run on
    // packed f32x2 pairs of populations (a, a+1): one instruction issues two
    // additions or FMAs, each rounded as the scalar one, so the results are
    // bitwise those of the scalar form; the kernel is issue-bound, and this
    // takes 7% off the D2Q16 step.  The limiter and the shuffles stay scalar.
    // The pair operands are read before the flux code (as here, the step
    // measured 2% faster than with them read after it).
    float xs[Q];
    const float2 omw2 = make_float2(omw, omw);
#pragma unroll
    for (int a = 0; a < Q; a += 2) {
      const int iy = a % NR;
      if ((iy >= H) != (iy + 1 >= H)) {  // a pair across c_y = 0 (D2Q36): one at a time
#pragma unroll
        for (int b = a; b < a + 2; ++b) {
          float f0;
          const float diff = yflux(b % NR >= H, b, fc, s0, s1, ld, A.ky[b % NR], f0);
          acc[b] = fmaf(omw, f0, fmaf(-A.ay[b % NR], diff, acc[b]));
          xs[b] = SPLIT ? fmaf(-A.ay[b % NR], diff, f0) : f0;
        }
        continue;
      }
      const float2 nay = make_float2(A.nay[iy], A.nay[iy + 1]);
      float2 f0;
      const float2 diff = yflux2(iy >= H, a, fc, s0, s1, ld, make_float2(A.ky[iy], A.ky[iy + 1]), f0);
      const float2 ac = fma2(omw2, f0, fma2(nay, diff, make_float2(acc[a], acc[a + 1])));
      const float2 x2 = SPLIT ? fma2(nay, diff, f0) : f0;
      acc[a] = ac.x;
      acc[a + 1] = ac.y;
      xs[a] = x2.x;
      xs[a + 1] = x2.y;
    }

    // x-advection of xs: neighbours from adjacent lanes; a and a+1 share ix
#pragma unroll
    for (int a = 0; a < Q; a += 2) {
      const int ix = (a / NR) % NR;
      const float2 kx = make_float2(A.kx2[ix][0], A.kx2[ix][1]);
      const float2 nax = make_float2(A.nax2[ix][0], A.nax2[ix][1]);
      const float2 diff = xflux2(ix >= H, make_float2(xs[a], xs[a + 1]), kx, StripLanes{});
      const float2 ac = fma2(nax, diff, make_float2(acc[a], acc[a + 1]));
      acc[a] = ac.x;
      acc[a + 1] = ac.y;
    }

    // the Maxwell wall (specular share) and walls in x are separate
    // instantiations so that the hot loop of everything else keeps its code
    apply_walls_node<NR, WM>(acc, xw, j, A);

    if (writer) {
      S *o = fout + (long long)j * rstride + (long long)xw * V;
      // rounding key per step and row (not per column): a flow uniform in x stays
      // exactly uniform, so rounding noise cannot seed the x-varying modes the
      // printed unsplit update amplifies
      int gr = j + A.row_key;  // the global row (a y-slab's halo rows may wrap around)
      if (A.row_period) {
        gr %= A.row_period;
        if (gr < 0) gr += A.row_period;
      }
      const unsigned key = mix32(A.seed ^ mix32((unsigned)gr));
#pragma unroll
      for (int g = 0; g < G; ++g) st_group_sr<NR, S>(o, gstride, g, acc, A, key);
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// The fused time step for D3Q216 (N = 4): 108 stored values per node (the
// z-even half), too many for one thread.  A block of three warps shares one
// strip of nodes, warp iz holding z-level iz (c_z = c[3 + iz]) -- 36 values
// laid out like D2Q36 -- and running the step of k_step on them.  The levels
// meet in the collision, whose moments are sums over all levels (each warp
// adds its in-plane Hermite moments weighted by 2 He_l(c_z) into shared
// memory, one barrier per row, every warp sums the three in the same order),
// and in the wall rules' incoming flux (one more barrier on wall rows, and on
// every row of the strips that hold a wall column).  The advection does not
// depend on the collision, so a warp publishes its share, advects, and only
// then waits for the others: the barrier no longer lines the three warps up
// for the shuffle-heavy x-sweep (5.41 -> 3.98 ms per 4096^2 step).
// Storage S: FP32 deviations, or FP16/BF16 relative deviations stochastically
// rounded like k_step's (level iz's stored populations are iz*36 .. iz*36+35
// of the node, so its scale factors and random words are those of the
// one-thread layout).  WM: 0 y-walls (fully diffuse) if any, 1 y-walls with
// a specular share, 2 walls in x as well (y-walls diffuse; corners as in
// wall_corner).
// ---------------------------------------------------------------------------
constexpr int kBlockZ = 96;  // three warps: one per stored z-level
constexpr int kXch = 13;     // moments a level contributes: l = 0, m + k <= 3 (10); l = 2, m + k <= 1 (3)
constexpr int kXch4 = 4;     // ... held as four float4 per thread (16 slots)

template <int RING, class S = float>
constexpr size_t stepz_smem_bytes() {
  return (size_t)3 * RING * 18 * 32 * (2 * sizeof(S)) + (size_t)2 * 3 * kXch4 * 32 * sizeof(float4) +
         3 * 32 * sizeof(float);
}

template <bool SPLIT, int RING, int WM, class S>
__global__ void __launch_bounds__(kBlockZ) k_step_z(const S *__restrict__ fin, S *__restrict__ fout,
                                                    const KArgs A) {
  constexpr int NR = 6, N = 4, H = 3, Q = 36, V = 2, GL = 18, KM = 3;
  constexpr int HL = 2, U = 32 - 2 * HL;
  using LL = LayoutQ<NR, S, Q>;  // one level: the D2Q36 slot order
  static_assert(LL::V == V && LL::G == GL, "a level holds 18 pairs");
  using T = typename Raw<LL::VB>::T;
  constexpr bool kScaled = Store<S>::kScaled;
  const int lane = threadIdx.x & 31;
  const int iz = threadIdx.x >> 5;  // stored z-level of this warp
  const int zo = iz * Q;            // its first stored population
  const int strip = blockIdx.x % A.nstrips;
  const int seg = blockIdx.x / A.nstrips;
  if (seg >= A.nseg) return;  // uniform over the block
  const int nx = A.nx, ny = A.ny;
  const int xl = strip * U - HL + lane;
  int xw;
  if constexpr (WM == 2) {
    xw = min(max(xl, 0), nx - 1);  // walls in x: ghost columns hold the wall node
  } else {
    xw = xl % nx;
    if (xw < 0) xw += nx;
  }
  const bool writer = lane >= HL && lane < 32 - HL && xl < nx;
  // the strip holds a wall column (uniform over the block): its rows take the wall exchange
  const bool xstrip = WM == 2 && (strip == 0 || (strip + 1) * U >= nx);
  const int y0 = seg * A.rows;
  const int y1 = min(y0 + A.rows, ny);
  const long long gstride = (long long)V * A.plane;
  const long long rstride = (long long)V * nx;
  // level iz's 18 group planes: c_y < 0 groups at 9 iz + gl (gl < 9), c_y > 0
  // groups at 27 + 9 iz + (gl - 9)
  const long long lo = (long long)(9 * iz) * gstride, hi = (long long)(18 + 9 * iz) * gstride;
  const S *fx = fin + (long long)xw * V;
  auto row_ptr = [&](int j) { return fx + map_row(j, ny, A.walls) * rstride; };
  // a level's raw vector -> FP32 deviations (scale of stored population zo + a)
  auto unpack_z = [&](const T &raw, int g, float (&F)[Q]) {
    const S *e = reinterpret_cast<const S *>(&raw);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int a = LL::alpha(g * V + k);
      F[a] = Store<S>::get(e[k], kScaled ? A.wq[zo + a] : 1.0f);
    }
  };
  auto load_z = [&](const S *p, int g, float (&F)[Q]) {
    const T raw = __ldg(reinterpret_cast<const T *>(p + g * gstride));
    unpack_z(raw, g, F);
  };

  float fc[Q], s0[Q], s1[Q];
  {
    float m2[Q], m1[Q], p1[Q];
    const S *pm2 = row_ptr(y0 - 2), *pm1 = row_ptr(y0 - 1), *pz = row_ptr(y0), *pp1 = row_ptr(y0 + 1);
#pragma unroll
    for (int g = 0; g < GL; ++g) {
      const long long off = g < GL / 2 ? lo : hi;
      load_z(pm1 + off, g, m1);
      load_z(pz + off, g, fc);
      if (g >= GL / 2) load_z(pm2 + off, g, m2);
      else load_z(pp1 + off, g, p1);
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ring = reinterpret_cast<T *>(smem_raw) + (size_t)iz * RING * GL * 32 + lane;
  // exchange buffer [row parity][level][float4 k][lane]: consecutive lanes read
  // consecutive 16-byte words (no bank conflicts)
  float4 *xch = reinterpret_cast<float4 *>(smem_raw + (size_t)3 * RING * GL * 32 * sizeof(T));
  float *wsum = reinterpret_cast<float *>(xch + 2 * 3 * kXch4 * 32);
  // this level's z-weights, read once: 2 He_2(c_z) and w_z He_l(c_z)/l!, l = 0, 2, 4
  const float he2 = 2.0f * A.he[H + iz][2];
  const float hz[3] = {A.hw[H + iz][0], A.hw[H + iz][2], A.hw[H + iz][4]};
  int r1 = map_row(y0 + 1, ny, A.walls), r2 = map_row(y0 + 2, ny, A.walls);
  const int nrows = y1 - y0;
  auto issue_rowload = [&](int k) {
    if (k < nrows) {
      const S *q1 = fx + r1 * rstride, *q2 = fx + r2 * rstride;
      T *slot = ring + (k % RING) * GL * 32;
#pragma unroll
      for (int g = 0; g < GL; ++g)
        cp_async_raw<LL::VB>(slot + g * 32, (g >= GL / 2 ? q1 + hi : q2 + lo) + g * gstride);
      r1 = r2;
      r2 = r2 + 1 < ny ? r2 + 1 : (A.walls ? ny - 1 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < RING - 1; ++k) issue_rowload(k);

  for (int j = y0; j < y1; ++j) {
    const int k = j - y0;
    issue_rowload(k + RING - 1);
    cp_async_wait<RING - 1>();
    float ld[Q];
    {
      const T *slot = ring + (k % RING) * GL * 32;
#pragma unroll
      for (int g = 0; g < GL; ++g) unpack_z(slot[g * 32], g, ld);
    }

    // this level's share of the moments into shared memory; the barrier and
    // the sum come after the advection, which does not depend on them
    {
      float a2[KM + 1][KM + 1];
      hermite_moments<NR, KM>(fc, a2, A);
      float part[4 * kXch4];
      int v = 0;
#pragma unroll
      for (int m = 0; m <= KM; ++m)
#pragma unroll
        for (int q = 0; m + q <= KM; ++q) part[v++] = 2.0f * a2[m][q];
#pragma unroll
      for (int m = 0; m <= KM - 2; ++m)
#pragma unroll
        for (int q = 0; m + q <= KM - 2; ++q) part[v++] = he2 * a2[m][q];
#pragma unroll
      for (; v < 4 * kXch4; ++v) part[v] = 0.0f;
      float4 *x = xch + ((k & 1) * 3 + iz) * kXch4 * 32 + lane;
#pragma unroll
      for (int q = 0; q < kXch4; ++q)
        x[q * 32] = make_float4(part[4 * q], part[4 * q + 1], part[4 * q + 2], part[4 * q + 3]);
    }

    float f0v[Q], acc[Q];  // f^n_j and the advective change
    {
      float xs[Q];
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const int iy = a % NR;
        if ((iy >= H) != (iy + 1 >= H)) {  // a pair across c_y = 0: one at a time
#pragma unroll
          for (int b = a; b < a + 2; ++b) {
            float f0;
            const float diff = yflux(b % NR >= H, b, fc, s0, s1, ld, A.ky[b % NR], f0);
            f0v[b] = f0;
            acc[b] = -A.ay[b % NR] * diff;
            xs[b] = SPLIT ? fmaf(-A.ay[b % NR], diff, f0) : f0;
          }
          continue;
        }
        const float2 nay = make_float2(A.nay[iy], A.nay[iy + 1]);
        float2 f0;
        const float2 diff = yflux2(iy >= H, a, fc, s0, s1, ld, make_float2(A.ky[iy], A.ky[iy + 1]), f0);
        const float2 ac = __fmul2_rn(nay, diff);
        const float2 x2 = SPLIT ? fma2(nay, diff, f0) : f0;
        f0v[a] = f0.x;
        f0v[a + 1] = f0.y;
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
        xs[a] = x2.x;
        xs[a + 1] = x2.y;
      }
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const int ix = a / NR;
        const float2 kx = make_float2(A.kx2[ix][0], A.kx2[ix][1]);
        const float2 nax = make_float2(A.nax2[ix][0], A.nax2[ix][1]);
        const float2 diff = xflux2(ix >= H, make_float2(xs[a], xs[a + 1]), kx, StripLanes{});
        const float2 ac = fma2(nax, diff, make_float2(acc[a], acc[a + 1]));
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
      }
    }

    // the moments summed over the levels, then collision and force
    {
      __syncthreads();
      float tot[4 * kXch4];
      const float4 *x0 = xch + (k & 1) * 3 * kXch4 * 32 + lane;
#pragma unroll
      for (int q = 0; q < kXch4; ++q) {
        const float4 p0 = x0[q * 32], p1 = x0[(kXch4 + q) * 32], p2 = x0[(2 * kXch4 + q) * 32];
        tot[4 * q] = (p0.x + p1.x) + p2.x;  // the levels in a fixed order
        tot[4 * q + 1] = (p0.y + p1.y) + p2.y;
        tot[4 * q + 2] = (p0.z + p1.z) + p2.z;
        tot[4 * q + 3] = (p0.w + p1.w) + p2.w;
      }
      float b[3][KM + 1][KM + 1];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int m = 0; m <= KM; ++m)
#pragma unroll
          for (int q = 0; q <= KM; ++q) b[l][m][q] = 0.0f;
      int v = 0;
#pragma unroll
      for (int m = 0; m <= KM; ++m)
#pragma unroll
        for (int q = 0; m + q <= KM; ++q) b[0][m][q] = tot[v++];
#pragma unroll
      for (int m = 0; m <= KM - 2; ++m)
#pragma unroll
        for (int q = 0; m + q <= KM - 2; ++q) b[1][m][q] = tot[v++];
      float d[3][N + 1][N + 1];
      float omw;
      es_coefficients3<NR, N, KM>(b, d, omw, A);
      float dz[N + 1][N + 1];
#pragma unroll
      for (int m = 0; m <= N; ++m)
#pragma unroll
        for (int q = 0; m + q <= N; ++q) {
          float t = d[0][m][q] * hz[0];
          if (m + q + 2 <= N) t = fmaf(d[1][m][q], hz[1], t);
          if (m + q + 4 <= N) t = fmaf(d[2][m][q], hz[2], t);
          dz[m][q] = t;
        }
      float src[Q];
      hermite_evaluate<NR, N>(dz, src, A);
      const float2 omw2 = make_float2(omw, omw);
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const float2 ac = fma2(omw2, make_float2(f0v[a], f0v[a + 1]),
                               __fadd2_rn(make_float2(acc[a], acc[a + 1]), make_float2(src[a], src[a + 1])));
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
      }
    }

    // the wall rules of wall_fix, wall_fix_x and wall_corner with the
    // incoming flux summed over the levels
    const bool yrow = A.walls && (j == 0 || j == ny - 1);  // uniform over the block
    if (yrow || xstrip) {
      const int ys = j == 0 ? 0 : 1, xs = xw == 0 ? 0 : 1;
      const bool xn = WM == 2 && (xw == 0 || xw == nx - 1);  // this lane's node is on an x-wall
      const float nxs = xs == 0 ? 1.0f : -1.0f, nys = ys == 0 ? 1.0f : -1.0f;
      float sl = 0.0f;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int ix = a / NR, iy = a % NR;
        const bool kx_in = xs == 0 ? ix < H : ix >= H, ky_in = ys == 0 ? iy < H : iy >= H;
        if (xn && yrow) {
          if (kx_in && ky_in) sl = fmaf(fabsf(fmaf(A.c[ix], nxs, A.c[iy] * nys)), acc[a], sl);
        } else if (xn) {
          if (kx_in) sl = fmaf(fabsf(A.c[ix]), acc[a], sl);
        } else if (ky_in) {
          sl = fmaf(fabsf(A.c[iy]), acc[a], sl);
        }
      }
      wsum[iz * 32 + lane] = sl;
      __syncthreads();
      const float s = (wsum[lane] + wsum[32 + lane]) + wsum[64 + lane];
      if (xn) {
        const float rw1 = yrow ? (s - A.wAc[ys * 2 + xs]) * A.wBc[ys * 2 + xs] : (s - A.wAx[xs]) * A.wBx[xs];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const int ix = a / NR, iy = a % NR;
          const bool kx_in = xs == 0 ? ix < H : ix >= H, ky_in = ys == 0 ? iy < H : iy >= H;
          const bool keep = yrow ? (kx_in && ky_in) : kx_in;
          if (!keep) acc[a] = fmaf(rw1, A.wSx[xs][zo + a], A.wSxdev[xs][zo + a]);
        }
      } else if (yrow) {
        const float rw1 = (s - A.wA[ys]) * A.wB[ys];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const int iy = a % NR;
          const bool outgoing = ys == 0 ? (iy >= H) : (iy < H);
          if (outgoing) {
            const float diffuse = fmaf(rw1, A.wS[ys][zo + a], A.wSdev[ys][zo + a]);
            if constexpr (WM == 1) acc[a] = fmaf(A.wspec, acc[a + (NR - 1 - 2 * iy)] - diffuse, diffuse);
            else acc[a] = diffuse;
          }
        }
      }
    }

    if (writer) {
      S *o = fout + (long long)j * rstride + (long long)xw * V;
      if constexpr (kScaled) {
        // the random words of st_group_sr: one per pair, keyed by the step,
        // the global row and the node's group (9 iz + g, or 18 + 9 iz + g)
        int gr = j + A.row_key;
        if (A.row_period) {
          gr %= A.row_period;
          if (gr < 0) gr += A.row_period;
        }
        const unsigned key = mix32(A.seed ^ mix32((unsigned)gr));
#pragma unroll
        for (int g = 0; g < GL; ++g) {
          const int a0 = LL::alpha(g * V), a1 = LL::alpha(g * V + 1);
          const int gg = 9 * iz + g + (g < GL / 2 ? 0 : 18);
          const unsigned bits = mix32(key ^ ((unsigned)gg * 0x9e3779b9u));
          *reinterpret_cast<T *>(o + (g < GL / 2 ? lo : hi) + g * gstride) =
              Store<S>::put_sr2(acc[a0] * A.iwq[zo + a0], acc[a1] * A.iwq[zo + a1], bits);
        }
      } else {
#pragma unroll
        for (int g = 0; g < GL; ++g) st_group_s<NR, float>(o + (g < GL / 2 ? lo : hi), gstride, g, acc, A);
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// The fused time step with compensated FP32 storage (tag Comp: D2Q16 and
// D3Q64, N = 3, periodic or fully diffuse walls).  The mapping of k_step
// (32-node strips, a segment of rows per warp, a per-lane cp.async ring of
// look-ahead rows), with every stored value carried as hi + lo:
//   - differences of stored values, the TVD slopes and fluxes of Sec. 3.1,
//     take (hi_1 - hi_0) + (lo_1 - lo_0), which keeps the stored precision;
//   - the collision and force source of Sec. 2.2 read hi alone (the source
//     is dt/tau times the non-equilibrium part, so leaving lo out costs that
//     fraction of one FP32 rounding);
//   - the update adds the step's increment t to hi + lo with an error-free
//     two-sum: s = hi + (lo + t), e = (hi - s) + (lo + t); hi = s, lo = e.
// A step's storage error is then the FP16 rounding of the remainder, 2^-11
// of at most half an FP32 ulp, instead of half an FP32 ulp.  The x-advection
// of each population follows its y-advection at once (it needs only that
// population's neighbours), so the per-population temporaries stay short.
// ---------------------------------------------------------------------------
template <bool SPLIT, int RING, int NZ>
__global__ void __launch_bounds__(kBlock, NZ == 1 ? 3 : 1) k_step_c(const float *__restrict__ fin, float *__restrict__ fout,
                                                   const KArgs A) {
  constexpr int NR = 4, N = 3;
  using LH = Layout<NR, float, NZ>;   // hi plane: 4 FP32 per 16-byte vector
  using LL = Layout<NR, __half, NZ>;  // lo plane: 8 FP16 per 16-byte vector
  constexpr int Q = LH::Q, H = LH::H, GH = LH::G, GL = LL::G, VH = LH::V, VL = LL::V, G = GH + GL;
  static_assert(VL == 2 * VH, "hi and lo vectors of 16 bytes");
  constexpr int HL = 2;
  constexpr int U = 32 - 2 * HL;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int strip = warp % A.nstrips;
  const int seg = warp / A.nstrips;
  if (seg >= A.nseg) return;  // uniform over the warp
  const int nx = A.nx, ny = A.ny;
  const int xl = strip * U - HL + lane;
  int xw = xl % nx;
  if (xw < 0) xw += nx;
  const bool writer = lane >= HL && lane < 32 - HL && xl < nx;
  const int y0 = seg * A.rows;
  const int y1 = min(y0 + A.rows, ny);
  // both planes as 16-byte vectors: vector g < GH of a node is hi group g,
  // vector GH + g lo group g; each group plane holds nx ny vectors
  const long long plane = A.plane;
  const uint4 *vx = reinterpret_cast<const uint4 *>(fin) + xw;
  auto up_group = [](int g) { return g < GH ? g >= GH / 2 : (g - GH) >= GL / 2; };  // c_y > 0
  auto unpack = [&](const uint4 (&v)[G], float (&hi)[Q], float (&lo)[Q]) {
#pragma unroll
    for (int g = 0; g < GH; ++g) {
      const float *e = reinterpret_cast<const float *>(&v[g]);
#pragma unroll
      for (int k = 0; k < VH; ++k) hi[LH::alpha(g * VH + k)] = e[k];
    }
#pragma unroll
    for (int g = 0; g < GL; ++g) {
      const __half *e = reinterpret_cast<const __half *>(&v[GH + g]);
#pragma unroll
      for (int k = 0; k < VL; ++k) {
        const int a = LL::alpha(g * VL + k);
        // a rounded product (never contracted into a later subtraction): a
        // row's lo values are then the same numbers whether a segment's
        // prologue loads the row or the ring brings it, whatever the segment
        // boundaries -- slabs and launch shapes give bitwise the same result
        lo[a] = __fmul_rn(__half2float(e[k]), A.wq[a]);
      }
    }
  };
  auto load_row = [&](int j, float (&hi)[Q], float (&lo)[Q]) {
    const uint4 *p = vx + (long long)map_row(j, ny, A.walls) * nx;
    uint4 v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = __ldg(p + g * plane);
    unpack(v, hi, lo);
  };

  // y-stencil per population, as in k_step, with hi and lo parts of values:
  //   c_y > 0: s0 = f_j - f_{j-1} (a difference), s1 = sigma_{j-1}; fc = f_j
  //   c_y < 0: s0 = f_{j+1} (s0h + s0l),        s1 = sigma_j;     fc = f_j
  float fch[Q], fcl[Q], s0h[Q], s0l[Q], s1[Q];
  {
    float m2h[Q], m2l[Q], m1h[Q], m1l[Q], p1h[Q], p1l[Q];
    load_row(y0 - 2, m2h, m2l);
    load_row(y0 - 1, m1h, m1l);
    load_row(y0, fch, fcl);
    load_row(y0 + 1, p1h, p1l);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const float d0 = (fch[a] - m1h[a]) + (fcl[a] - m1l[a]);  // f_j - f_{j-1}
      if (a % NR >= H) {
        s0h[a] = d0;
        s0l[a] = 0.0f;
        s1[a] = minmod((m1h[a] - m2h[a]) + (m1l[a] - m2l[a]), d0);
      } else {
        s0h[a] = p1h[a];
        s0l[a] = p1l[a];
        s1[a] = minmod(d0, (p1h[a] - fch[a]) + (p1l[a] - fcl[a]));
      }
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint4 *ring = reinterpret_cast<uint4 *>(smem_raw) + (size_t)(threadIdx.x >> 5) * RING * G * 32 + lane;
  int r1 = map_row(y0 + 1, ny, A.walls), r2 = map_row(y0 + 2, ny, A.walls);
  const int nrows = y1 - y0;
  auto issue_rowload = [&](int k) {
    if (k < nrows) {
      uint4 *slot = ring + (k % RING) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g)
        cp_async_raw<16>(slot + g * 32, vx + (long long)(up_group(g) ? r1 : r2) * nx + g * plane);
      r1 = r2;
      r2 = r2 + 1 < ny ? r2 + 1 : (A.walls ? ny - 1 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < RING - 1; ++k) issue_rowload(k);

  for (int j = y0; j < y1; ++j) {
    const int k = j - y0;
    issue_rowload(k + RING - 1);
    cp_async_wait<RING - 1>();
    float ldh[Q], ldl[Q];
    {
      uint4 v[G];
      const uint4 *slot = ring + (k % RING) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g) v[g] = slot[g * 32];
      unpack(v, ldh, ldl);
    }
    float src[Q], om;
    collide_om<NR, N>(fch, src, om, A, A);

    // populations a and a + 1 (a even) share ix and the sign of c_y, so the
    // whole update runs on packed FP32 pairs (each half rounded as the scalar
    // operation); the limiters and the lane shuffles stay scalar
    float nh[Q], nl[Q];  // f^{n+1} as hi + lo
    const float2 nom = make_float2(-om, -om);
    const StripLanes nb;
    auto left2 = [&](float2 v) { return make_float2(nb.left(v.x), nb.left(v.y)); };
    auto right2 = [&](float2 v) { return make_float2(nb.right(v.x), nb.right(v.y)); };
    auto minmod2 = [](float2 u, float2 v) { return make_float2(minmod(u.x, v.x), minmod(u.y, v.y)); };
#pragma unroll
    for (int a = 0; a < Q; a += 2) {
      const int iy = a % NR, ix = (a / NR) % NR;
      static_assert(NR % 2 == 0 && H % 2 == 0, "pairs of populations share the sign of c_y");
      const float2 f0h = make_float2(fch[a], fch[a + 1]), f0l = make_float2(fcl[a], fcl[a + 1]);
      const float2 lh = make_float2(ldh[a], ldh[a + 1]), ll = make_float2(ldl[a], ldl[a + 1]);
      const float2 S0h = make_float2(s0h[a], s0h[a + 1]), S1 = make_float2(s1[a], s1[a + 1]);
      const float2 ky = make_float2(A.ky[iy], A.ky[iy + 1]);
      float2 diff;
      if (iy >= H) {  // c_y > 0
        const float2 dn = __fadd2_rn(sub2(lh, f0h), sub2(ll, f0l));
        const float2 sg = minmod2(S0h, dn);
        diff = fma2(ky, sub2(sg, S1), S0h);
        s0h[a] = dn.x;
        s0h[a + 1] = dn.y;
        s1[a] = sg.x;
        s1[a + 1] = sg.y;
        fch[a] = lh.x;
        fch[a + 1] = lh.y;
        fcl[a] = ll.x;
        fcl[a + 1] = ll.y;
      } else {  // c_y < 0
        const float2 S0l = make_float2(s0l[a], s0l[a + 1]);
        const float2 d1 = __fadd2_rn(sub2(S0h, f0h), sub2(S0l, f0l));
        const float2 sg = minmod2(d1, __fadd2_rn(sub2(lh, S0h), sub2(ll, S0l)));
        diff = fma2(ky, sub2(S1, sg), d1);  // (-k)(sg - s1) = k (s1 - sg), exactly
        s1[a] = sg.x;
        s1[a + 1] = sg.y;
        fch[a] = S0h.x;
        fch[a + 1] = S0h.y;
        fcl[a] = S0l.x;
        fcl[a + 1] = S0l.y;
        s0h[a] = lh.x;
        s0h[a + 1] = lh.y;
        s0l[a] = ll.x;
        s0l[a + 1] = ll.y;
      }
      // -(c_y dt/dy)(F_{j+1/2} - F_{j-1/2}) joins the collision increment
      const float2 nay = make_float2(A.nay[iy], A.nay[iy + 1]);
      float2 inc = fma2(nay, diff, fma2(nom, f0h, make_float2(src[a], src[a + 1])));
      // x-fluxes of f^n (printed update) or of f* = f^n - ady (split), whose
      // hi part is f0h and whose change goes to the lo part
      const float2 xlo = SPLIT ? fma2(nay, diff, f0l) : f0l;
      const float2 dl = __fadd2_rn(sub2(f0h, left2(f0h)), sub2(xlo, left2(xlo)));
      const float2 dr = right2(dl);
      const float2 sg = minmod2(dl, dr);
      const float2 kx = make_float2(A.kx2[ix][0], A.kx2[ix][1]);
      // c_x < 0: (-k)(sigma_{i+1} - sigma_i) = k (sigma_i - sigma_{i+1}), exactly
      const float2 dxf = ix >= H ? fma2(kx, sub2(sg, left2(sg)), dl) : fma2(kx, sub2(sg, right2(sg)), dr);
      inc = fma2(make_float2(A.nax2[ix][0], A.nax2[ix][1]), dxf, inc);
      // error-free update of hi + lo
      const float2 t = __fadd2_rn(f0l, inc);
      const float2 sh = __fadd2_rn(f0h, t);
      const float2 lo2 = __fadd2_rn(sub2(f0h, sh), t);
      nh[a] = sh.x;
      nh[a + 1] = sh.y;
      nl[a] = lo2.x;
      nl[a + 1] = lo2.y;
    }

    if (A.walls && (j == 0 || j == ny - 1)) {
      // the wall rule of wall_fix on hi + lo: rho_W from the incoming half
      // (two sums), the outgoing half rho_W S as hi with its FMA remainder as lo
      const int side = j == 0 ? 0 : 1;
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int iy = a % NR;
        if (side == 0 ? (iy < H) : (iy >= H)) {
          sh = fmaf(fabsf(A.c[iy]), nh[a], sh);
          sl = fmaf(fabsf(A.c[iy]), nl[a], sl);
        }
      }
      const float rw1 = ((sh - A.wA[side]) + sl) * A.wB[side];  // rho_W - 1
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int iy = a % NR;
        if (side == 0 ? (iy >= H) : (iy < H)) {
          const float h = fmaf(rw1, A.wS[side][a], A.wSdev[side][a]);
          nl[a] = fmaf(rw1, A.wS[side][a], A.wSdev[side][a] - h);
          nh[a] = h;
        }
      }
    }

    if (writer) {
      uint4 *o = reinterpret_cast<uint4 *>(fout) + (long long)j * nx + xw;
#pragma unroll
      for (int g = 0; g < GH; ++g) {
        float4 v;
        v.x = nh[LH::alpha(g * VH)];
        v.y = nh[LH::alpha(g * VH + 1)];
        v.z = nh[LH::alpha(g * VH + 2)];
        v.w = nh[LH::alpha(g * VH + 3)];
        *reinterpret_cast<float4 *>(o + g * plane) = v;
      }
#pragma unroll
      for (int g = 0; g < GL; ++g) {
        uint4 raw;
        unsigned *w = reinterpret_cast<unsigned *>(&raw);
#pragma unroll
        for (int k2 = 0; k2 < VL; k2 += 2) {
          const int a0 = LL::alpha(g * VL + k2), a1 = LL::alpha(g * VL + k2 + 1);
          const __half2 h2 = __floats2half2_rn(nl[a0] * A.iwq[a0], nl[a1] * A.iwq[a1]);
          w[k2 / 2] = *reinterpret_cast<const unsigned *>(&h2);
        }
        o[(GH + g) * plane] = raw;
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Initial populations f = rho S(T,u) (Eq. feq0 to order N: the Hermite
// expansion of the isotropic Maxwellian), then the wall rule once.
// fields: double[4][ny][nx] = rho, u_x, u_y, T (or nullptr: rest).
// ---------------------------------------------------------------------------
template <int NR, int N, class S, int NZ = 1>
__global__ void __launch_bounds__(kBlock) k_init(const double *__restrict__ fields,
                                                 typename Elem<S>::T *__restrict__ f, const KArgs A) {
  constexpr int Q = NZ * NR * NR;
  const long long cells = A.plane;
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
    float Sv[Q];
    if constexpr (NZ == 1) {
      e[0][0] = drho;  // deviation from w_a
      hermite_evaluate<NR, N>(e, Sv, A);
    } else {  // D = 3: isotropic, so lambda_zz - 1 = T - 1 as in-plane
      float d[3][N + 1][N + 1];
      z_factor<N>(e, dT, 1.0f, d);
      d[0][0][0] = drho;
      hermite_evaluate3<NR, N>(d, Sv, A);
    }
    const int j = (int)(c / A.nx), i = (int)(c - (long long)j * A.nx);
    if (A.xwalls) apply_walls_node<NR, 2>(Sv, i, j, A);
    else if (A.wspec != 0.0f) apply_walls_node<NR, 1>(Sv, i, j, A);
    else apply_walls_node<NR, 0>(Sv, i, j, A);
    st_node<NR, S, NZ>(f, c, cells, Sv, A);
  }
}

// Largest density and temperature of initial fields double[4][cells] and the
// first node that is not admissible (rho, T > 0, all four finite):
// st[0], st[1] = bits of the maxima (non-negative doubles order like their
// bits), st[2] = the node index (or all ones).  st set to {0, 0, ~0} before.
__global__ void __launch_bounds__(kBlock) k_field_stats(const double *__restrict__ f, long long cells,
                                                        unsigned long long *__restrict__ st) {
  double rmax = 0.0, tmax = 0.0;
  unsigned long long bad = ~0ull;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < cells; c += (long long)gridDim.x * kBlock) {
    const double r = f[c], ux = f[cells + c], uy = f[2 * cells + c], T = f[3 * cells + c];
    if (!(r > 0.0) || !(T > 0.0) || !isfinite(r) || !isfinite(T) || !isfinite(ux) || !isfinite(uy)) {
      bad = min(bad, (unsigned long long)c);
    } else {
      rmax = fmax(rmax, r);
      tmax = fmax(tmax, T);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(kFull, rmax, o));
    tmax = fmax(tmax, __shfl_xor_sync(kFull, tmax, o));
    bad = min(bad, __shfl_xor_sync(kFull, bad, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st[0], (unsigned long long)__double_as_longlong(rmax));
    atomicMax(&st[1], (unsigned long long)__double_as_longlong(tmax));
    if (bad != ~0ull) atomicMin(&st[2], bad);
  }
}

// Populations between the grouped layout and the public [a][j][i] layout.
template <int NR, class S, int NZ = 1>
__global__ void __launch_bounds__(kBlock) k_ungroup(const typename Elem<S>::T *__restrict__ f,
                                                    float *__restrict__ out, long long cells, const KArgs A) {
  constexpr int Q = NZ * NR * NR;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < cells; c += (long long)gridDim.x * kBlock) {
    float F[Q];
    ld_node<NR, S, NZ>(f, c, cells, F, A);
#pragma unroll
    for (int a = 0; a < Q; ++a) out[a * cells + c] = F[a];
  }
}

template <int NR, class S, int NZ = 1>
__global__ void __launch_bounds__(kBlock) k_group(const float *__restrict__ in, typename Elem<S>::T *__restrict__ f,
                                                  long long cells, const KArgs A) {
  constexpr int Q = NZ * NR * NR;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < cells; c += (long long)gridDim.x * kBlock) {
    float F[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) F[a] = __ldg(in + a * cells + c);
    st_node<NR, S, NZ>(f, c, cells, F, A);
  }
}

// Conservation totals: per-node sums in FP32 (above), summed in FP32 over
// runs of kSumRun nodes, the runs in FP64 (GB300 issues about two FP64
// operations per SM and clock, so one FP64 add per node and quantity would
// cost as much as reading the populations).  Fixed order: reproducible.
constexpr int kSumRun = 16;

struct ConsSums {
  float run[4] = {0.f, 0.f, 0.f, 0.f};
  double tot[4] = {0.0, 0.0, 0.0, 0.0};
  int n = 0;          // nodes in the current run
  long long nodes = 0;
  __device__ __forceinline__ void add(const float (&d)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) run[k] += d[k];
    if (++n == kSumRun) flush();
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      tot[k] += (double)run[k];
      run[k] = 0.f;
    }
    nodes += n;
    n = 0;
  }
  // Block totals of mass, x/y momentum and energy (sum f {1, c_x, c_y, c^2/2},
  // f = w + df, sum_a w_a = 1, sum_a w_a c_a^2 = D) into partial[4 * block].
  __device__ __forceinline__ void write_block(double *__restrict__ partial, int D) {
    flush();
    double v[4] = {(double)nodes + tot[0], tot[1], tot[2], 0.5 * ((double)D * (double)nodes + tot[3])};
    __shared__ double red[4][kMomBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] += __shfl_down_sync(kFull, v[k], o);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {  // every block writes all four of its slots: no zeroing needed
      double t = 0.0;
      for (int k = 0; k < kMomBlock / 32; ++k) t += red[threadIdx.x][k];
      partial[blockIdx.x * 4 + threadIdx.x] = t;
    }
  }
};

// Moments per node of the grouped layout, plus the block partial sums, over
// `cells` consecutive nodes from f (a whole grid, or a range of its rows);
// plane: nodes of the whole grid (nx ny, the distance between group planes in
// vectors).  out: float[9][cells] or nullptr.
template <int NR, class S, int NZ = 1>
__global__ void __launch_bounds__(kMomBlock) k_moments(const typename Elem<S>::T *__restrict__ f,
                                                       float *__restrict__ out, double *__restrict__ partial,
                                                       long long cells, long long plane, const KArgs A) {
  constexpr int Q = NZ * NR * NR;
  ConsSums cs;
  for (long long c = blockIdx.x * (long long)kMomBlock + threadIdx.x; c < cells;
       c += (long long)gridDim.x * kMomBlock) {
    float F[Q];
    ld_node<NR, S, NZ>(f, c, plane, F, A);
    float d[4];
    node_moments<NR>(F, out, cells, c, A, d);
    cs.add(d);
  }
  cs.write_block(partial, NZ == 1 ? 2 : 3);
}

// Fields rho, u_x, u_y, T of each node against a snapshot: r_max (bits of a
// non-negative float in *rbits, atomic max) of |d rho| + |d u| + |d T| (a
// non-finite change counts as +Inf), and the snapshot overwritten with the
// current fields (residual of lesbgk_residual); mpart[block] receives the
// block's sum of rho - 1 (FP32 per thread, FP64 across the block).
template <int NR, class S, int NZ = 1>
__global__ void __launch_bounds__(kMomBlock) k_residual(const typename Elem<S>::T *__restrict__ f,
                                                        float *__restrict__ snap, int update_only,
                                                        unsigned *__restrict__ rbits, double *__restrict__ mpart,
                                                        const KArgs A) {
  constexpr int Q = NZ * NR * NR;
  const long long cells = A.plane;
  float rmax = 0.0f, dm = 0.0f;
  for (long long c = blockIdx.x * (long long)kMomBlock + threadIdx.x; c < cells;
       c += (long long)gridDim.x * kMomBlock) {
    float F[Q];
    ld_node<NR, S, NZ>(f, c, cells, F, A);
    float m[3][3], mzz = 0.0f;
    if constexpr (NZ == 1) {
      hermite_moments<NR, 2>(F, m, A);
    } else {
      float b[3][3][3];
      hermite_moments3<NR, 2>(F, b, A);
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; p + q < 3; ++q) m[p][q] = b[0][p][q];
      mzz = b[1][0][0];
    }
    const float rho = 1.0f + m[0][0];
    const float ir = __frcp_rn(rho);
    const float ux = m[1][0] * ir, uy = m[0][1] * ir;
    const float trM = fmaf(-m[1][0], ux, m[2][0]) + fmaf(-m[0][1], uy, m[0][2]) + mzz;
    const float T = fmaf((NZ == 1 ? 0.5f : 1.0f / 3.0f) * trM, ir, 1.0f);
    const float d = fabsf(rho - snap[c]) + fabsf(ux - snap[cells + c]) + fabsf(uy - snap[2 * cells + c]) +
                    fabsf(T - snap[3 * cells + c]);
    rmax = update_only ? 0.0f : fmaxf(rmax, d != d ? __int_as_float(0x7f800000) : d);  // NaN counts as Inf
    dm += m[0][0];
    snap[c] = rho;
    snap[cells + c] = ux;
    snap[2 * cells + c] = uy;
    snap[3 * cells + c] = T;
  }
  double dmd = (double)dm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmaxf(rmax, __shfl_xor_sync(kFull, rmax, o));
    dmd += __shfl_down_sync(kFull, dmd, o);
  }
  __shared__ double wsum[kMomBlock / 32];
  if ((threadIdx.x & 31) == 0) {
    if (rmax > 0.0f) atomicMax(rbits, __float_as_uint(rmax));
    wsum[threadIdx.x >> 5] = dmd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kMomBlock / 32; ++w) t += wsum[w];  // fixed order
    mpart[blockIdx.x] = t;
  }
}

// Sum of n doubles in a fixed order (one warp): bitwise reproducible.
__global__ void k_reduce_one(const double *__restrict__ part, int n, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double t = 0.0;
  for (int k = lane; k < n; k += 32) t += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
  if (lane == 0) *out = t;
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

constexpr int kMomGrid = lesbgk_internal::kMomentPartials;

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
  Setup su;  // FP64 inputs of the wall tables (rebuilt per step for heated walls)
  double dt, dx, dy, cmax, tau_ref;
  int64_t steps;
  int sm_count;
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t buffer_bytes(const lesbgk_params *p) {
  const size_t cells = (size_t)p->nx * p->ny;
  const size_t q = (size_t)p->nroots * p->nroots * (p->dim == 3 ? p->nroots / 2 : 1);  // values per node
  size_t per = q * (p->storage == LESBGK_F32 ? sizeof(float) : p->storage == LESBGK_F32C ? 6 : 2);
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
  // segments of 32 rows (D2Q16, D3Q64) or 128 rows (D2Q36): measured best on
  // the 4096^2 periodic case (D2Q36: 961 us per step at 128 rows, 988 us at
  // 32, where the three prologue rows per segment weigh more)
  h->cpt = 1;
  const int nstrips = (nx + 27) / 28;
  const int rows_default = h->q >= 36 ? 128 : 32;
  if (h->rows <= 0) h->rows = ny < rows_default ? ny : rows_default;
  h->args.rows = h->rows;
  h->args.nstrips = nstrips;
  h->args.nseg = (ny + h->rows - 1) / h->rows;
  return 0;
}

int build_tables(lesbgk *h, const FieldStats *stats) {
  Setup s;
  if (int rc = build_setup(h->p, h->order, stats, &s)) return rc;
  h->args = s.args;
  h->su = s;
  h->dt = s.dt;
  h->dx = s.dx;
  h->dy = s.dy;
  h->cmax = s.cmax;
  h->tau_ref = s.tau_ref;
  return 0;
}

constexpr int kRing = 4;

template <int NR, class S, int NZ>
constexpr size_t step_smem_bytes() {
  if constexpr (kIsComp<S>)  // both planes' 16-byte vectors
    return (size_t)(kBlock / 32) * kRing * (Layout<NR, float, NZ>::G + Layout<NR, __half, NZ>::G) * 32 * 16;
  else
    return (size_t)(kBlock / 32) * kRing * Layout<NR, S, NZ>::G * 32 * Layout<NR, S, NZ>::VB;
}

// Call fn(NR, N, storage tag, NZ) with compile-time constants for the built
// combinations: every (nroots, order) of the 2D sets in FP32, the default
// orders also in FP16 and BF16 (NZ = 1), D2Q16 also compensated (Comp);
// D3Q64, N = 3, in FP32, FP16, BF16 and compensated (NZ = 2 stored z-levels);
// D3Q216, N = 4, in FP32, FP16 and BF16 (NZ = 3).
template <class Fn>
void dispatch(int nr, int order, int storage, int dim, Fn &&fn) {
  using R4 = std::integral_constant<int, 4>;
  using R6 = std::integral_constant<int, 6>;
  using N3 = std::integral_constant<int, 3>;
  using N4 = std::integral_constant<int, 4>;
  using Z1 = std::integral_constant<int, 1>;
  using Z2 = std::integral_constant<int, 2>;
  using Z3 = std::integral_constant<int, 3>;
  if (dim == 3 && nr == 6) {
    if (storage == LESBGK_F16) fn(R6{}, N4{}, __half{}, Z3{});
    else if (storage == LESBGK_BF16) fn(R6{}, N4{}, __nv_bfloat16{}, Z3{});
    else fn(R6{}, N4{}, float{}, Z3{});
  } else if (dim == 3) {
    if (storage == LESBGK_F32C) fn(R4{}, N3{}, Comp{}, Z2{});
    else if (storage == LESBGK_F16) fn(R4{}, N3{}, __half{}, Z2{});
    else if (storage == LESBGK_BF16) fn(R4{}, N3{}, __nv_bfloat16{}, Z2{});
    else fn(R4{}, N3{}, float{}, Z2{});
  } else if (nr == 4 && order == 3) {
    if (storage == LESBGK_F32C) fn(R4{}, N3{}, Comp{}, Z1{});
    else if (storage == LESBGK_F16) fn(R4{}, N3{}, __half{}, Z1{});
    else if (storage == LESBGK_BF16) fn(R4{}, N3{}, __nv_bfloat16{}, Z1{});
    else fn(R4{}, N3{}, float{}, Z1{});
  } else if (nr == 6 && order == 4) {
    if (storage == LESBGK_F16) fn(R6{}, N4{}, __half{}, Z1{});
    else if (storage == LESBGK_BF16) fn(R6{}, N4{}, __nv_bfloat16{}, Z1{});
    else fn(R6{}, N4{}, float{}, Z1{});
  } else if (nr == 4) {
    fn(R4{}, N4{}, float{}, Z1{});
  } else {
    fn(R6{}, N3{}, float{}, Z1{});
  }
}

// Opt in to more than 48 KiB of dynamic shared memory where a ring needs it.
cudaError_t allow_smem(const lesbgk *h) {
  cudaError_t e = cudaSuccess;
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto n, auto st, auto z) {
    constexpr int NR = decltype(r)::value, N = decltype(n)::value, NZ = decltype(z)::value;
    using S = decltype(st);
    auto allow = [&](auto kernel, int smem) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    if constexpr (kIsComp<S>) {
      constexpr int smem = (int)step_smem_bytes<NR, S, NZ>();
      allow(k_step_c<true, kRing, NZ>, smem);
      allow(k_step_c<false, kRing, NZ>, smem);
    } else if constexpr (NZ == 3) {  // D3Q216: one warp per stored z-level
      constexpr int smem = (int)stepz_smem_bytes<kRing, S>();
      allow(k_step_z<true, kRing, 0, S>, smem);
      allow(k_step_z<false, kRing, 0, S>, smem);
      allow(k_step_z<true, kRing, 1, S>, smem);
      allow(k_step_z<false, kRing, 1, S>, smem);
      allow(k_step_z<true, kRing, 2, S>, smem);
      allow(k_step_z<false, kRing, 2, S>, smem);
    } else {
      constexpr int smem = (int)step_smem_bytes<NR, S, NZ>();
      allow(k_step<NR, N, true, kRing, S, 0, NZ>, smem);
      allow(k_step<NR, N, false, kRing, S, 0, NZ>, smem);
      allow(k_step<NR, N, true, kRing, S, 2, NZ>, smem);
      allow(k_step<NR, N, false, kRing, S, 2, NZ>, smem);
      if constexpr (std::is_same<S, float>::value) {
        allow(k_step<NR, N, true, kRing, S, 1, NZ>, smem);
        allow(k_step<NR, N, false, kRing, S, 1, NZ>, smem);
      }
    }
  });
  return e;
}

int launch_step(lesbgk *h, const void *fin, void *fout, cudaStream_t s) {
  const long long warps = (long long)h->args.nstrips * h->args.nseg;
  const unsigned grid = (unsigned)((warps * 32 + kBlock - 1) / kBlock);
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto n, auto st, auto z) {
    constexpr int NR = decltype(r)::value, N = decltype(n)::value, NZ = decltype(z)::value;
    using S = decltype(st);
    using E = typename Elem<S>::T;
    const E *fi = static_cast<const E *>(fin);
    E *fo = static_cast<E *>(fout);
    const bool split = h->p.scheme == LESBGK_SPLIT;
    if constexpr (kIsComp<S>) {  // compensated storage: hi + lo planes
      constexpr size_t smem = step_smem_bytes<NR, S, NZ>();
      if (split) k_step_c<true, kRing, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
      else k_step_c<false, kRing, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
      return;
    } else if constexpr (NZ == 3) {  // D3Q216: a block of three warps per strip and segment
      constexpr size_t smem = stepz_smem_bytes<kRing, S>();
      const unsigned gz = (unsigned)warps;
      const int wm = h->args.xwalls ? 2 : (h->args.walls && h->args.wspec != 0.0f ? 1 : 0);
      if (wm == 2) {  // walls in x
        if (split) k_step_z<true, kRing, 2, S><<<gz, kBlockZ, smem, s>>>(fi, fo, h->args);
        else k_step_z<false, kRing, 2, S><<<gz, kBlockZ, smem, s>>>(fi, fo, h->args);
        return;
      }
      if (split) {
        if (wm == 1) k_step_z<true, kRing, 1, S><<<gz, kBlockZ, smem, s>>>(fi, fo, h->args);
        else k_step_z<true, kRing, 0, S><<<gz, kBlockZ, smem, s>>>(fi, fo, h->args);
      } else {
        if (wm == 1) k_step_z<false, kRing, 1, S><<<gz, kBlockZ, smem, s>>>(fi, fo, h->args);
        else k_step_z<false, kRing, 0, S><<<gz, kBlockZ, smem, s>>>(fi, fo, h->args);
      }
      return;
    } else {
      constexpr size_t smem = step_smem_bytes<NR, S, NZ>();
      if (h->args.xwalls) {  // walls in x (cavity)
        if (split) k_step<NR, N, true, kRing, S, 2, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
        else k_step<NR, N, false, kRing, S, 2, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
        return;
      }
      if constexpr (std::is_same<S, float>::value) {  // Maxwell walls: FP32 storage (checked at set-up)
        if (h->args.walls && h->args.wspec != 0.0f) {  // Maxwell walls
          if (split) k_step<NR, N, true, kRing, S, 1, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
          else k_step<NR, N, false, kRing, S, 1, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
          return;
        }
      }
      if (split) k_step<NR, N, true, kRing, S, 0, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
      else k_step<NR, N, false, kRing, S, 0, NZ><<<grid, kBlock, smem, s>>>(fi, fo, h->args);
    }
  });
  return 0;
}

unsigned grid_for(const lesbgk *h, long long cells) {
  long long g = (cells + kBlock - 1) / kBlock;
  const long long cap = (long long)h->sm_count * 16;
  if (g > cap) g = cap;
  return g < 1 ? 1u : (unsigned)g;
}

int launch_init(lesbgk *h, const double *fields, void *f, cudaStream_t s) {
  const unsigned grid = grid_for(h, h->args.plane);
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto n, auto st, auto z) {
    constexpr int NR = decltype(r)::value, N = decltype(n)::value, NZ = decltype(z)::value;
    using S = decltype(st);
    k_init<NR, N, S, NZ><<<grid, kBlock, 0, s>>>(fields, static_cast<typename Elem<S>::T *>(f), h->args);
  });
  return 0;
}

int launch_moments(lesbgk *h, float *out, cudaStream_t s) {
  const void *f = h->buf[h->cur];
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto, auto st, auto z) {
    constexpr int NR = decltype(r)::value, NZ = decltype(z)::value;
    using S = decltype(st);
    k_moments<NR, S, NZ><<<kMomGrid, kMomBlock, 0, s>>>(static_cast<const typename Elem<S>::T *>(f), out,
                                                        h->partial, h->args.plane, h->args.plane, h->args);
  });
  k_reduce_partials<<<1, 128, 0, s>>>(h->partial, kMomGrid, h->sums);
  return 0;
}

}  // namespace

namespace lesbgk_internal {

// (storage: LESBGK_F32, LESBGK_F16 or LESBGK_BF16, the 2D sets; A supplies the
// 16-bit scale tables)
cudaError_t launch_init(const KArgs &A, int nr, int order, int storage, int dim, const double *fields, void *f,
                        int sm_count, cudaStream_t s) {
  long long g = (A.plane + kBlock - 1) / kBlock;
  if (g > (long long)sm_count * 16) g = (long long)sm_count * 16;
  const unsigned grid = g < 1 ? 1u : (unsigned)g;
  dispatch(nr, order, storage, dim, [&](auto r, auto n, auto st, auto z) {
    using S = decltype(st);
    if constexpr (!kIsComp<S> && decltype(z)::value < 3)
      k_init<decltype(r)::value, decltype(n)::value, S, decltype(z)::value>
          <<<grid, kBlock, 0, s>>>(fields, static_cast<S *>(f), A);
  });
  return cudaGetLastError();
}

cudaError_t launch_moments(const KArgs &A, int nr, int order, int storage, int dim, const void *f, float *out,
                           double *partial, double *sums, cudaStream_t s) {
  dispatch(nr, order, storage, dim, [&](auto r, auto, auto st, auto z) {
    using S = decltype(st);
    if constexpr (!kIsComp<S> && decltype(z)::value < 3)
      k_moments<decltype(r)::value, S, decltype(z)::value>
          <<<kMomGrid, kMomBlock, 0, s>>>(static_cast<const S *>(f), out, partial, A.plane, A.plane, A);
  });
  k_reduce_partials<<<1, 128, 0, s>>>(partial, kMomGrid, sums);
  return cudaGetLastError();
}

cudaError_t launch_ungroup(const KArgs &A, int nr, int order, int storage, int dim, const void *f, float *out,
                           long long cells, int sm_count, cudaStream_t s) {
  long long g = (cells + kBlock - 1) / kBlock;
  if (g > (long long)sm_count * 16) g = (long long)sm_count * 16;
  const unsigned grid = g < 1 ? 1u : (unsigned)g;
  dispatch(nr, order, storage, dim, [&](auto r, auto, auto st, auto z) {
    using S = decltype(st);
    if constexpr (!kIsComp<S> && decltype(z)::value < 3)
      k_ungroup<decltype(r)::value, S, decltype(z)::value><<<grid, kBlock, 0, s>>>(static_cast<const S *>(f), out, cells, A);
  });
  return cudaGetLastError();
}

}  // namespace lesbgk_internal

extern "C" int lesbgk_create(const lesbgk_params *p, void *d_workspace, size_t bytes, const double *h_init,
                             void *stream, lesbgk **out) {
  lesbgk_internal::Range range_("lesbgk_create");
  clear_error();
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
  h->order = p->order ? p->order : default_order(p->nroots);
  h->q = h->nr * h->nr * (p->dim == 3 ? h->nr / 2 : 1);
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double *dfields = nullptr;
  FieldStats stats{1.0, 1.0, -1};
  if (h_init) {
    // fields to the device, then their check and maxima there (a host loop
    // over 4 nx ny values would cost more than the copy)
    const long long cells = (long long)p->nx * p->ny;
    const size_t fb = (size_t)4 * cells * sizeof(double);
    unsigned long long *st = reinterpret_cast<unsigned long long *>(h->sums);
    unsigned long long hs[3] = {0, 0, 0};
    e = cudaMemcpyAsync(h->buf[1], h_init, fb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st + 2, 0xff, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      dfields = reinterpret_cast<const double *>(h->buf[1]);
      k_field_stats<<<grid_for(h, cells), kBlock, 0, s>>>(dfields, cells, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, st, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // also: h_init may be freed after return
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "copy and check of initial fields");
    }
    double r, t;
    std::memcpy(&r, &hs[0], sizeof r);
    std::memcpy(&t, &hs[1], sizeof t);
    stats = FieldStats{r, t, hs[2] == ~0ull ? -1 : (long long)hs[2]};
  }
  if (int rc = build_tables(h, h_init ? &stats : nullptr)) {
    delete h;
    return rc;
  }
  pick_launch(h);
  e = allow_smem(h);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "step kernel shared-memory opt-in");
  }
  launch_init(h, dfields, h->buf[0], s);  // reads the device copy: no wait for the host
  e = cudaGetLastError();
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
  if (heated_walls(h->su)) set_wall_time(h->su, 0.0, &h->args);
  launch_init(h, d_fields, h->buf[0], s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "init kernel");
}

extern "C" int lesbgk_step(lesbgk *h, int64_t nsteps, void *stream) {
  lesbgk_internal::Range range_("lesbgk_step");
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(LESBGK_EINVAL, "nsteps < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t k = 0; k < nsteps; ++k) {
    h->args.seed = (unsigned)(h->steps + k) * 0x9e3779b9u + 0x7f4a7c15u;  // a new rounding key per step
    if (heated_walls(h->su))  // wall tables at the time of the state written
      set_wall_time(h->su, (double)(h->steps + k + 1) * h->dt, &h->args);
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
  lesbgk_internal::Range range_("lesbgk_moments");
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_moments(h, d_out, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "moments kernel");
  return finish_sums(h, h_sums, s);
}

extern "C" int lesbgk_moments_host(lesbgk *h, float *h_out, double *h_sums, void *stream) {
  lesbgk_internal::Range range_("lesbgk_moments_host");
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

extern "C" int lesbgk_residual(lesbgk *h, float *d_snap, int64_t steps, double *h_r, double *h_mass,
                               void *stream) {
  lesbgk_internal::Range range_("lesbgk_residual");
  if (!h || !d_snap || !h_r) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch in the handle's reduction area (no moments call runs meanwhile):
  // the residual's bits in sums[0], the mass in sums[1], block partials in partial
  unsigned *rbits = reinterpret_cast<unsigned *>(h->sums);
  cudaError_t e = cudaMemsetAsync(rbits, 0, sizeof(unsigned), s);
  const void *f = h->buf[h->cur];
  if (e == cudaSuccess) {
    dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto, auto st, auto z) {
      using S = decltype(st);
      k_residual<decltype(r)::value, S, decltype(z)::value><<<kMomGrid, kMomBlock, 0, s>>>(
          static_cast<const typename Elem<S>::T *>(f), d_snap, steps <= 0 ? 1 : 0, rbits, h->partial, h->args);
    });
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_reduce_one<<<1, 32, 0, s>>>(h->partial, kMomGrid, h->sums + 1);
    e = cudaGetLastError();
  }
  double hb[2] = {0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb, h->sums, sizeof hb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "residual");
  float rmax;
  std::memcpy(&rmax, &hb[0], sizeof rmax);
  *h_r = steps <= 0 ? std::nan("") : (double)rmax / ((double)steps * h->dt);
  if (h_mass) *h_mass = (double)h->args.plane + hb[1];
  return 0;
}

extern "C" int lesbgk_get_populations(lesbgk *h, float *d_out, void *stream) {
  if (!h || !d_out) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long cells = h->args.plane;
  const void *f = h->buf[h->cur];
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto, auto st, auto z) {
    using S = decltype(st);
    k_ungroup<decltype(r)::value, S, decltype(z)::value>
        <<<grid_for(h, cells), kBlock, 0, s>>>(static_cast<const typename Elem<S>::T *>(f), d_out, cells, h->args);
  });
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "get populations");
}

extern "C" int lesbgk_set_populations(lesbgk *h, const float *d_in, int64_t steps_done, void *stream) {
  if (!h || !d_in) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long cells = h->args.plane;
  void *f = h->buf[h->cur];
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto, auto st, auto z) {
    using S = decltype(st);
    k_group<decltype(r)::value, S, decltype(z)::value>
        <<<grid_for(h, cells), kBlock, 0, s>>>(d_in, static_cast<typename Elem<S>::T *>(f), cells, h->args);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "set populations");
  h->steps = steps_done;
  return 0;
}

namespace {
// Bytes of one stored vector and the number of group planes of the solver's layout.
void row_geometry(const lesbgk *h, int *vb, int *groups) {
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto, auto st, auto z) {
    using S = decltype(st);
    constexpr int NR = decltype(r)::value, NZ = decltype(z)::value;
    if constexpr (kIsComp<S>) {  // the lo plane's groups follow the hi plane's, 16-byte vectors in both
      *vb = 16;
      *groups = Layout<NR, float, NZ>::G + Layout<NR, __half, NZ>::G;
    } else {
      *vb = Layout<NR, S, NZ>::VB;
      *groups = Layout<NR, S, NZ>::G;
    }
  });
}

int check_rows(const lesbgk *h, int32_t j0, int32_t nrows) {
  if (!h) return fail(LESBGK_EINVAL, "handle is NULL");
  if (nrows < 0 || j0 < 0 || (long long)j0 + nrows > h->p.ny)
    return fail(LESBGK_EINVAL, "rows [%d, %d) outside [0, %d)", j0, j0 + nrows, h->p.ny);
  return 0;
}

// One 2D copy: G planes of nrows x nx vectors, between the current buffer and
// a packed array.
int copy_rows(lesbgk *h, int32_t j0, int32_t nrows, void *packed, bool to_packed, cudaStream_t s) {
  int vb = 0, groups = 0;
  row_geometry(h, &vb, &groups);
  const size_t width = (size_t)nrows * h->p.nx * vb, pitch = (size_t)h->args.plane * vb;
  char *base = reinterpret_cast<char *>(h->buf[h->cur]) + (size_t)j0 * h->p.nx * vb;
  if (!width) return 0;
  cudaError_t e = to_packed ? cudaMemcpy2DAsync(packed, width, base, pitch, width, groups, cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpy2DAsync(base, pitch, packed, width, width, groups, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? 0 : cuda_fail(e, "row copy");
}
}  // namespace

extern "C" int lesbgk_rows_bytes(const lesbgk *h, int32_t nrows, size_t *bytes) {
  if (!h || !bytes || nrows < 0) return fail(LESBGK_EINVAL, "bad argument");
  int vb = 0, groups = 0;
  row_geometry(h, &vb, &groups);
  *bytes = (size_t)groups * nrows * h->p.nx * vb;
  return 0;
}

extern "C" int lesbgk_get_rows(lesbgk *h, int32_t j0, int32_t nrows, void *d_out, void *stream) {
  if (int rc = check_rows(h, j0, nrows)) return rc;
  if (!d_out) return fail(LESBGK_EINVAL, "d_out is NULL");
  return copy_rows(h, j0, nrows, d_out, true, static_cast<cudaStream_t>(stream));
}

extern "C" int lesbgk_set_rows(lesbgk *h, int32_t j0, int32_t nrows, const void *d_in, void *stream) {
  if (int rc = check_rows(h, j0, nrows)) return rc;
  if (!d_in) return fail(LESBGK_EINVAL, "d_in is NULL");
  return copy_rows(h, j0, nrows, const_cast<void *>(d_in), false, static_cast<cudaStream_t>(stream));
}

extern "C" int lesbgk_moments_rows(lesbgk *h, int32_t j0, int32_t nrows, float *d_out, double *h_sums,
                                   void *stream) {
  if (int rc = check_rows(h, j0, nrows)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const void *f = h->buf[h->cur];
  const long long cells = (long long)nrows * h->p.nx;
  dispatch(h->nr, h->order, h->p.storage, h->p.dim, [&](auto r, auto, auto st, auto z) {
    constexpr int NR = decltype(r)::value, NZ = decltype(z)::value;
    using S = decltype(st);
    using E = typename Elem<S>::T;
    constexpr int V = Layout<NR, E, NZ>::V;  // (for Comp the hi plane's; the lo plane shares its byte offsets)
    const E *fr = static_cast<const E *>(f) + (long long)j0 * h->p.nx * V;
    k_moments<NR, S, NZ><<<kMomGrid, kMomBlock, 0, s>>>(fr, d_out, h->partial, cells, h->args.plane, h->args);
  });
  k_reduce_partials<<<1, 128, 0, s>>>(h->partial, kMomGrid, h->sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "moments of rows");
  return finish_sums(h, h_sums, s);
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
template <int NR, int NZ = 1>
__global__ void __launch_bounds__(kMomBlock) k_moments_public(const float *__restrict__ f, float *__restrict__ out,
                                                              double *__restrict__ partial, const KArgs A) {
  constexpr int Q = NZ * NR * NR;
  const long long cells = A.plane;
  ConsSums cs;
  const long long c0 = blockIdx.x * kNoAllocNodesPerBlock;
  for (int t = 0; t < kNoAllocNodesPerThread; ++t) {
    const long long c = c0 + (long long)t * kMomBlock + threadIdx.x;
    if (c >= cells) break;
    float F[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) F[a] = __ldg(f + a * cells + c);
    float d[4];
    node_moments<NR>(F, out, cells, c, A, d);
    cs.add(d);
  }
  cs.write_block(partial, NZ == 1 ? 2 : 3);
}

// Device address of g_noalloc_scratch (in host code the symbol is only a
// stand-in).  An address belongs to one CUDA context, not to a device: a
// device reset, or a caller that runs its own context on the same device,
// loads the module again at another address.  So the cache is keyed by the
// current context's process-unique ID (cuCtxGetId, reached through the
// runtime's driver entry points, so that the library does not link libcuda),
// and each new context gets its own cudaGetSymbolAddress.  If those driver
// entry points are unavailable the address is looked up on every call.
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);
constexpr int kNoAllocCache = 64;  // contexts remembered (oldest replaced first)
std::mutex g_noalloc_mutex;
struct NoAllocEntry {
  unsigned long long ctx_id;
  double *ptr;
};
NoAllocEntry g_noalloc_cache[kNoAllocCache] = {};
int g_noalloc_next = 0;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_looked_up = false;

// The current context's unique ID; false if there is none (or no way to ask).
bool current_context_id(unsigned long long *id) {
  if (!g_ctx_fns_looked_up) {
    g_ctx_fns_looked_up = true;
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
      g_ctx_id = reinterpret_cast<CtxGetIdFn>(g);
    }
    cudaGetLastError();  // a failed query leaves no sticky error
  }
  if (!g_ctx_current || !g_ctx_id) return false;
  void *ctx = nullptr;
  if (g_ctx_current(&ctx) != 0 || !ctx) return false;
  return g_ctx_id(ctx, id) == 0;
}

int noalloc_scratch(double **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  unsigned long long id = 0;
  bool have = current_context_id(&id);
  if (have)
    for (const NoAllocEntry &e : g_noalloc_cache)
      if (e.ptr && e.ctx_id == id) {
        *out = e.ptr;
        return 0;
      }
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static moment scratch");
  if (!have) have = current_context_id(&id);  // the lookup made the device's primary context current
  if (have) {
    g_noalloc_cache[g_noalloc_next] = NoAllocEntry{id, static_cast<double *>(p)};
    g_noalloc_next = (g_noalloc_next + 1) % kNoAllocCache;
  }
  *out = static_cast<double *>(p);
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
  tmp.order = p->order ? p->order : default_order(p->nroots);
  tmp.q = tmp.nr * tmp.nr * (p->dim == 3 ? tmp.nr / 2 : 1);
  if (int rc = build_tables(&tmp, nullptr)) return rc;
  double *scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((cells + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock);
  double *sums = scratch + (size_t)kNoAllocBlocks * 4;
  if (p->dim == 3 && p->nroots == 6)
    k_moments_public<6, 3><<<blocks, kMomBlock, 0, s>>>(d_populations, d_out, scratch, tmp.args);
  else if (p->dim == 3) k_moments_public<4, 2><<<blocks, kMomBlock, 0, s>>>(d_populations, d_out, scratch, tmp.args);
  else if (p->nroots == 4) k_moments_public<4><<<blocks, kMomBlock, 0, s>>>(d_populations, d_out, scratch, tmp.args);
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
