// Batched lattice ES-BGK solver: many independent narrow solves (nx a power of
// two <= 32, e.g. the 1D-in-y channel flows of Sec. 4 of the paper) advanced
// together, one launch per lattice per time step, replayed from CUDA graphs.
//
// Device memory: the caller's workspace holds fixed tables (per-slot
// descriptors, the work list, residual and moment scratch) and a pool from
// which each instance gets its two population buffers and a residual
// snapshot; the pool is managed on the host (first fit, 256-byte aligned).
//
// k_batch_step: a warp holds 32/W lane groups of W = nx lanes; each group owns
// one work item (an instance and a segment of its rows) and marches it like
// the single-domain kernel (y-stencil in registers, look-ahead rows through a
// per-lane cp.async ring), with the periodic x-neighbours taken by shuffles
// inside the group.  Work items are sorted by length so the groups of a warp
// run the same number of rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "lesbgk.h"
#include "setup.h"

using namespace lesbgk_dev;
using namespace lesbgk_setup;

namespace {

constexpr int kBBlock = 128;
constexpr int kBRing = 4;
// classes: velocity set x storage x wall heating -- class lat + 3 st + 9 h
// with lat 0 D2Q16 (order 3), 1 D2Q36 (order 4), 2 D3Q64 (order 3, its z-even
// half stored); st 0 FP32, 1 FP16, 2 BF16; h 1 for heated walls (their
// kernels carry the FP64 wall-table code, the others none of it)
constexpr int kNumClasses = 18;
constexpr int kGraphSteps = 64;
constexpr size_t kGuardBytes = 256;       // guard words after each slot's pool block
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kBuckets = 6;  // resident instances by height: ny <= 16, 32, ..., 512 (smem permitting)

// Per-instance descriptor (device memory).
struct InstDesc {
  float *f[2];  // population buffers, grouped layout
  float *snap;  // residual snapshot: rho, ux, uy, T per node
  const HeatPoly *heat;  // heated walls (Sec. 4.2): the wall tables' polynomials, or null
  int nx, ny, walls, split;
  int vmode, has_force, pad0, pad1;
  float c_omega, visc_pow, b, beta, dtgx, dtgy, dt, wspec;  // wspec: Maxwell walls' specular share
  float ax[kMaxR], kx[kMaxR], ay[kMaxR], ky[kMaxR];
  float wS[2][kMaxQ], wSdev[2][kMaxQ], wA[2], wB[2];
};

struct WorkItem {
  int inst, y0, rows, pad;
};

struct LatTables {
  float c[kMaxR];
  float he[kMaxR][kMaxN + 1];
  float hw[kMaxR][kMaxN + 1];
  float wq[kMaxQ], iwq[kMaxQ];  // 16-bit storage scale (stored = df * iwq), as in KArgs
};

struct BatchArgs {
  LatTables lat;
  const InstDesc *desc;
  const WorkItem *items;
  const int *range;  // {first item, item count} of this lattice class
  long long *nstep;  // per slot, per buffer parity: the steps that led to that buffer's state
};

// Per-solve scalars of one instance, held in registers (collide's TP).
struct InstRegs {
  float c_omega, visc_pow, b, beta, dtgx, dtgy;
  int vmode, has_force;
};

template <int NR, class S = float, int NZ = 1>
constexpr size_t batch_smem_bytes() {
  return (size_t)(kBBlock / 32) * kBRing * Layout<NR, S, NZ>::G * 32 * Layout<NR, S, NZ>::VB;
}

// neighbour lanes inside a lane group of W lanes (periodic in x)
struct GroupLanes {
  int srcL, srcR;
  __device__ __forceinline__ float left(float v) const { return __shfl_sync(kFull, v, srcL); }
  __device__ __forceinline__ float right(float v) const { return __shfl_sync(kFull, v, srcR); }
};

// wall_fix of a heated wall (Sec. 4.2): the tables evaluated at heating hv
// from the polynomials of HeatPoly by the arithmetic of set_wall_time, so the
// values are bitwise those the single-domain solver passes for the same step.
template <int NR, bool SPEC, int Q, class TT>
__device__ __forceinline__ void wall_fix_heated(float (&O)[Q], int side, const TT &T, const HeatPoly &P, double hv,
                                                float wspec) {
  constexpr int H = NR / 2;
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int iy = a % NR;
    const bool incoming = side == 0 ? (iy < H) : (iy >= H);
    if (incoming) s = fmaf(fabsf(T.c[iy]), O[a], s);
  }
  const double ao = fma(fma(P.Aout[side][2], hv, P.Aout[side][1]), hv, P.Aout[side][0]);
  const double zo = fma(fma(P.Zout[side][2], hv, P.Zout[side][1]), hv, P.Zout[side][0]);
  const float rw1 = (s - (float)ao) * (float)(1.0 / zo);  // rho_W - 1
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int iy = a % NR;
    const bool outgoing = side == 0 ? (iy >= H) : (iy < H);
    if (outgoing) {
      const double S = fma(fma(P.S[side][2][a], hv, P.S[side][1][a]), hv, P.S[side][0][a]);
      const float diffuse = fmaf(rw1, (float)S, (float)(S - P.w[a]));
      if constexpr (SPEC) O[a] = fmaf(wspec, O[a + (NR - 1 - 2 * iy)] - diffuse, diffuse);
      else O[a] = diffuse;
    }
  }
}

// One time step of every work item of a class (velocity set and storage S:
// FP32 deviations, or FP16/BF16 relative deviations rounded stochastically
// with the random words of k_step, keyed by the instance's step count and row).
template <int NR, int N, int W, class S, bool HEAT, int NZ>
__global__ void __launch_bounds__(kBBlock) k_batch_step(const BatchArgs B, const int par) {
  using Lay = Layout<NR, S, NZ>;
  constexpr int Q = Lay::Q, H = Lay::H, V = Lay::V, G = Lay::G;
  constexpr int GPW = 32 / W;
  const int lane = threadIdx.x & 31;
  const int gi = lane / W, lx = lane % W;
  const int warp = (blockIdx.x * kBBlock + threadIdx.x) >> 5;
  const int first = B.range[0], count = B.range[1];
  const int base = warp * GPW;
  if (base >= count) return;  // uniform over the warp
  int it = base + gi;
  const bool live = it < count;
  if (!live) it = base;  // idle group: repeats the warp's first item, stores nothing
  const WorkItem wi = B.items[first + it];
  const InstDesc &D = B.desc[wi.inst];
  const int ny = D.ny, walls = D.walls;
  const bool split = D.split != 0;
  InstRegs P{D.c_omega, D.visc_pow, D.b, D.beta, D.dtgx, D.dtgy, D.vmode, D.has_force};
  float ax[NR], kx[NR], ay[NR], ky[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    ax[i] = D.ax[i];
    kx[i] = D.kx[i];
    ay[i] = D.ay[i];
    ky[i] = D.ky[i];
  }
  const S *fin = reinterpret_cast<const S *>(D.f[par]);
  S *fout = reinterpret_cast<S *>(D.f[par ^ 1]);
  const long long gstride = (long long)V * W * ny;
  const long long rstride = (long long)V * W;
  const S *fx = fin + (long long)lx * V;
  const int y0 = wi.y0;
  const int rows = live ? wi.rows : 0;
  int nrows = rows;  // the warp runs its longest item's rows
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrows = max(nrows, __shfl_xor_sync(kFull, nrows, o));
  const int srcL = gi * W + ((lx + W - 1) & (W - 1));
  const int srcR = gi * W + ((lx + 1) & (W - 1));
  auto row_ptr = [&](int j) { return fx + map_row(j, ny, walls) * rstride; };

  float fc[Q], s0[Q], s1[Q];
  {
    float m2[Q], m1[Q], p1[Q];
    const S *pm2 = row_ptr(y0 - 2), *pm1 = row_ptr(y0 - 1), *pz = row_ptr(y0), *pp1 = row_ptr(y0 + 1);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      ld_group_s<NR, S>(pm1, gstride, g, m1, B.lat);
      ld_group_s<NR, S>(pz, gstride, g, fc, B.lat);
      if (g >= G / 2) ld_group_s<NR, S>(pm2, gstride, g, m2, B.lat);
      else ld_group_s<NR, S>(pp1, gstride, g, p1, B.lat);
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
  using T = typename Raw<Lay::VB>::T;
  T *ring = reinterpret_cast<T *>(smem_raw) + (size_t)(threadIdx.x >> 5) * kBRing * G * 32 + lane;
  int r1 = map_row(y0 + 1, ny, walls), r2 = map_row(y0 + 2, ny, walls);
  auto issue_rowload = [&](int k) {
    if (k < nrows) {
      const S *q1 = fx + r1 * rstride, *q2 = fx + r2 * rstride;
      T *slot = ring + (k % kBRing) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g) cp_async_raw<Lay::VB>(slot + g * 32, (g >= G / 2 ? q1 : q2) + g * gstride);
      r1 = r2;
      r2 = r2 + 1 < ny ? r2 + 1 : (walls ? ny - 1 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < kBRing - 1; ++k) issue_rowload(k);

  for (int k = 0; k < nrows; ++k) {
    const int j = y0 + k;
    issue_rowload(k + kBRing - 1);
    cp_async_wait<kBRing - 1>();
    float ld[Q];
    {
      const T *slot = ring + (k % kBRing) * G * 32;
#pragma unroll
      for (int g = 0; g < G; ++g) unpack_group<NR, S>(slot[g * 32], g, ld, B.lat);
    }
    float acc[Q];
    float omw;
    collide_any<NR, N>(fc, acc, omw, B.lat, P);
    float xs[Q];
    const GroupLanes nb{srcL, srcR};
    if constexpr (NR == 4) {  // packed pairs a, a+1 (same ix, c_y of one sign)
      const float2 omw2 = make_float2(omw, omw);
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const int iy = a % NR;
        const float2 nay = make_float2(-ay[iy], -ay[iy + 1]);
        float2 f0;
        const float2 diff = yflux2(iy >= H, a, fc, s0, s1, ld, make_float2(ky[iy], ky[iy + 1]), f0);
        const float2 ac = fma2(omw2, f0, fma2(nay, diff, make_float2(acc[a], acc[a + 1])));
        const float2 x2 = split ? fma2(nay, diff, f0) : f0;
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
        xs[a] = x2.x;
        xs[a + 1] = x2.y;
      }
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const int ix = (a / NR) % NR;
        const float2 nax = make_float2(-ax[ix], -ax[ix]);
        const float2 diff = xflux2(ix >= H, make_float2(xs[a], xs[a + 1]), make_float2(kx[ix], kx[ix]), nb);
        const float2 ac = fma2(nax, diff, make_float2(acc[a], acc[a + 1]));
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
      }
    } else {  // D2Q36: one population at a time (the pair constants would spill)
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int iy = a % NR;
        float f0;
        const float diff = yflux(iy >= H, a, fc, s0, s1, ld, ky[iy], f0);
        acc[a] = fmaf(omw, f0, fmaf(-ay[iy], diff, acc[a]));
        xs[a] = split ? fmaf(-ay[iy], diff, f0) : f0;
      }
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int ix = (a / NR) % NR;
        acc[a] = fmaf(-ax[ix], xflux(ix >= H, xs[a], kx[ix], nb), acc[a]);
      }
    }
    if (walls && (j == 0 || j == ny - 1)) {
      const int side = j == 0 ? 0 : 1;
      if constexpr (HEAT) {  // the wall temperature of the time this step writes
        const HeatPoly &hp = *D.heat;
        const double hv = wall_heating(hp, (double)(B.nstep[2 * wi.inst + par] + 1) * hp.dt);
        if (D.wspec != 0.0f) wall_fix_heated<NR, true>(acc, side, B.lat, hp, hv, D.wspec);
        else wall_fix_heated<NR, false>(acc, side, B.lat, hp, hv, D.wspec);
      } else if (D.wspec != 0.0f) {
        wall_fix<NR, true>(acc, side, B.lat, D);
      } else {
        wall_fix<NR, false>(acc, side, B.lat, D);
      }
    }
    if (k < rows) {
      S *o = fout + (long long)j * rstride + (long long)lx * V;
      if constexpr (Store<S>::kScaled) {  // the key of k_step: step count and row
        const unsigned seed = (unsigned)B.nstep[2 * wi.inst + par] * 0x9e3779b9u + 0x7f4a7c15u;
        const unsigned key = mix32(seed ^ mix32((unsigned)j));
#pragma unroll
        for (int g = 0; g < G; ++g) st_group_sr<NR, S>(o, gstride, g, acc, B.lat, key);
      } else {
#pragma unroll
        for (int g = 0; g < G; ++g) st_group_s<NR, S>(o, gstride, g, acc, B.lat);
      }
    }
  }
  cp_async_wait<0>();
  // the instance's step count (the clock of heated walls, the key of 16-bit
  // rounding) follows its state into the other buffer: one thread per
  // instance, while every thread of this launch reads parity par only
  if constexpr (HEAT || Store<S>::kScaled)
    if (live && wi.y0 == 0 && lx == 0) B.nstep[2 * wi.inst + (par ^ 1)] = B.nstep[2 * wi.inst + par] + 1;
}

// ---------------------------------------------------------------------------
// Resident batched step (D2Q16, order 3): one block holds one whole instance
// in shared memory -- two buffers of Q planes of ny x W values -- and takes K
// time steps there, reading the instance from device memory once and writing
// it once per launch.  Per step every thread updates the nodes of its row
// (its lane's column) pass after pass, 128/W rows at a time, then one barrier
// swaps the buffers.  Each thread rebuilds, from the five rows j-2..j+2 of its
// column, the y-stencil state that k_batch_step carries from row to row (fc,
// s0, s1 and the incoming row, each by the same floating-point operations) and
// runs the same yflux2 / xflux2 / collide / wall_fix: the result is bitwise
// that of the per-step kernel, so a solve's answer does not depend on which
// path stepped it.  rlist: the instances, one per block; smem holds the
// largest of them.  Reads buffer p_in, writes buffer p_out (p_in ^ (K & 1)
// when stepping; the spare buffer when the autotuner times it).
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kBBlock) k_batch_resident(const BatchArgs B, const int *__restrict__ rlist,
                                                            const int *__restrict__ rrange, int K, int p_in,
                                                            int p_out) {
  constexpr int NR = 4, N = 3, Q = 16, H = 2;
  constexpr int R = kBBlock / W;  // rows per pass
  if ((int)blockIdx.x >= rrange[1]) return;  // the bucket's count, read from device memory
  const int inst = rlist[rrange[0] + blockIdx.x];
  const InstDesc &D = B.desc[inst];
  const int ny = D.ny, walls = D.walls;
  const bool split = D.split != 0;
  const long long cells = (long long)W * ny;
  InstRegs P{D.c_omega, D.visc_pow, D.b, D.beta, D.dtgx, D.dtgy, D.vmode, D.has_force};
  float ax[NR], kx[NR], ay[NR], ky[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    ax[i] = D.ax[i];
    kx[i] = D.kx[i];
    ay[i] = D.ay[i];
    ky[i] = D.ky[i];
  }
  extern __shared__ __align__(16) float sm[];
  float *buf[2] = {sm, sm + (size_t)Q * cells};  // [a][j][i] planes
  // the instance into buffer 0
  for (long long c = threadIdx.x; c < cells; c += kBBlock) {
    float F[Q];
    ld_node<NR, float, 1>(D.f[p_in], c, cells, F, B.lat);
#pragma unroll
    for (int a = 0; a < Q; ++a) buf[0][a * cells + c] = F[a];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int lx = threadIdx.x % W;
  const int gi = lane / W;  // group of W lanes within the warp
  const GroupLanes nb{gi * W + ((lx + W - 1) & (W - 1)), gi * W + ((lx + 1) & (W - 1))};
  int cur = 0;
  for (int step = 0; step < K; ++step) {
    const float *fi = buf[cur];
    float *fo = buf[cur ^ 1];
    for (int j0 = 0; j0 < ny; j0 += R) {
      const int j = j0 + (int)threadIdx.x / W;
      const bool live = j < ny;
      const int jj = live ? j : ny - 1;  // a spare group computes a real row and stores nothing
      const int rm2 = map_row(jj - 2, ny, walls), rm1 = map_row(jj - 1, ny, walls);
      const int rp1 = map_row(jj + 1, ny, walls), rp2 = map_row(jj + 2, ny, walls);
      auto at = [&](int a, int r) { return fi[a * cells + (long long)r * W + lx]; };
      float fc[Q], s0[Q], s1[Q], ld[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const float m2 = at(a, rm2), m1 = at(a, rm1), c0 = at(a, jj), p1 = at(a, rp1);
        fc[a] = c0;
        if (a % NR >= H) {  // c_y > 0: s0 = f_j - f_{j-1}, s1 = sigma_{j-1}, incoming f_{j+1}
          s0[a] = c0 - m1;
          s1[a] = minmod(m1 - m2, c0 - m1);
          ld[a] = p1;
        } else {  // c_y < 0: s0 = f_{j+1}, s1 = sigma_j, incoming f_{j+2}
          s0[a] = p1;
          s1[a] = minmod(c0 - m1, p1 - c0);
          ld[a] = at(a, rp2);
        }
      }
      float acc[Q];
      float omw;
      collide<NR, N>(fc, acc, omw, B.lat, P);
      float xs[Q];
      const float2 omw2 = make_float2(omw, omw);
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const int iy = a % NR;
        const float2 nay = make_float2(-ay[iy], -ay[iy + 1]);
        float2 f0;
        const float2 diff = yflux2(iy >= H, a, fc, s0, s1, ld, make_float2(ky[iy], ky[iy + 1]), f0);
        const float2 ac = fma2(omw2, f0, fma2(nay, diff, make_float2(acc[a], acc[a + 1])));
        const float2 x2 = split ? fma2(nay, diff, f0) : f0;
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
        xs[a] = x2.x;
        xs[a + 1] = x2.y;
      }
#pragma unroll
      for (int a = 0; a < Q; a += 2) {
        const int ix = a / NR;
        const float2 nax = make_float2(-ax[ix], -ax[ix]);
        const float2 diff = xflux2(ix >= H, make_float2(xs[a], xs[a + 1]), make_float2(kx[ix], kx[ix]), nb);
        const float2 ac = fma2(nax, diff, make_float2(acc[a], acc[a + 1]));
        acc[a] = ac.x;
        acc[a + 1] = ac.y;
      }
      if (walls && (jj == 0 || jj == ny - 1)) {
        if (D.wspec != 0.0f) wall_fix<NR, true>(acc, (jj == 0) ? 0 : 1, B.lat, D);
        else wall_fix<NR, false>(acc, (jj == 0) ? 0 : 1, B.lat, D);
      }
      if (live) {
#pragma unroll
        for (int a = 0; a < Q; ++a) fo[a * cells + (long long)j * W + lx] = acc[a];
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  float *out = D.f[p_out];
  for (long long c = threadIdx.x; c < cells; c += kBBlock) {
    float F[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) F[a] = buf[cur][a * cells + c];
    st_node<NR, float, 1>(out, c, cells, F, B.lat);
  }
}

// Residual of every work item: max over its nodes of
// |d rho| + |d u_x| + |d u_y| + |d T| since the snapshot, folded into
// res_bits[instance] (non-negative floats order like their bit patterns; a
// node whose change is not finite counts as +Inf, so a diverged slot reports
// r = Inf); the snapshot is refreshed.  mass[item] receives the item's sum of
// rho - 1 over its nodes (FP32 per thread, FP64 across the block).  One block
// per item.
template <int NR, class S, int NZ>
__global__ void __launch_bounds__(kBBlock) k_batch_residual(const BatchArgs B, const int par,
                                                            unsigned *__restrict__ res_bits,
                                                            double *__restrict__ mass) {
  constexpr int Q = NZ * NR * NR;
  const int first = B.range[0], count = B.range[1];
  if ((int)blockIdx.x >= count) return;
  const WorkItem wi = B.items[first + blockIdx.x];
  const InstDesc &D = B.desc[wi.inst];
  const int nx = D.nx, ny = D.ny;
  const long long cells = (long long)nx * ny;
  const S *f = reinterpret_cast<const S *>(D.f[par]);
  float r = 0.0f, dm = 0.0f;
  for (int t = threadIdx.x; t < wi.rows * nx; t += kBBlock) {
    const long long c = (long long)wi.y0 * nx + t;
    float F[Q];
    ld_node<NR, S, NZ>(f, c, cells, F, B.lat);
    float m[3][3], mzz = 0.0f;
    if constexpr (NZ == 1) {
      hermite_moments<NR, 2>(F, m, B.lat);
    } else {  // D = 3: the in-plane moments summed over the z-levels, and m002
      float b[3][3][3];
      hermite_moments3<NR, 2>(F, b, B.lat);
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; p + q < 3; ++q) m[p][q] = b[0][p][q];
      mzz = b[1][0][0];
    }
    const float rho = 1.0f + m[0][0];
    const float ir = 1.0f / rho;
    const float ux = m[1][0] * ir, uy = m[0][1] * ir;
    const float trM = fmaf(-m[1][0], ux, m[2][0]) + fmaf(-m[0][1], uy, m[0][2]) + mzz;
    const float T = fmaf((NZ == 1 ? 0.5f : 1.0f / 3.0f) * trM, ir, 1.0f);
    float *s = D.snap + 4 * c;
    const float d = fabsf(rho - s[0]) + fabsf(ux - s[1]) + fabsf(uy - s[2]) + fabsf(T - s[3]);
    r = fmaxf(r, d != d ? __int_as_float(0x7f800000) : d);  // NaN counts as Inf
    dm += m[0][0];
    s[0] = rho;
    s[1] = ux;
    s[2] = uy;
    s[3] = T;
  }
  double dmd = (double)dm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r = fmaxf(r, __shfl_xor_sync(kFull, r, o));
    dmd += __shfl_down_sync(kFull, dmd, o);
  }
  __shared__ double wsum[kBBlock / 32];
  if ((threadIdx.x & 31) == 0) {
    atomicMax(res_bits + wi.inst, __float_as_uint(r));
    wsum[threadIdx.x >> 5] = dmd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBBlock / 32; ++w) t += wsum[w];  // fixed order
    mass[first + blockIdx.x] = t;
  }
}

// Initial populations of newly admitted slots, one block per slot of the
// list: f = rho S(T,u) (Eq. feq0 to order N) from the slot's fields (device
// double[4][ny][nx] in its spare buffer when list entry bit 30 is set, else
// rest), then the wall rule -- the arithmetic of the single-domain k_init.
template <int NR, int N, class S, int NZ>
__global__ void __launch_bounds__(kBBlock) k_batch_init(const BatchArgs B, const int *__restrict__ list, int n,
                                                        const int par) {
  if ((int)blockIdx.x >= n) return;
  const int entry = list[blockIdx.x];
  const InstDesc &D = B.desc[entry & 0x3fffffff];
  const bool has_fields = (entry >> 30) & 1;
  const int nx = D.nx, ny = D.ny;
  const long long cells = (long long)nx * ny;
  const double *fields = has_fields ? reinterpret_cast<const double *>(D.f[par ^ 1]) : nullptr;
  S *f = reinterpret_cast<S *>(D.f[par]);
  if (threadIdx.x == 0) B.nstep[2 * (entry & 0x3fffffff) + par] = 0;
  for (long long c = threadIdx.x; c < cells; c += kBBlock) {
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
    float Sv[NZ * NR * NR];
    if constexpr (NZ == 1) {
      e[0][0] = drho;
      hermite_evaluate<NR, N>(e, Sv, B.lat);
    } else {  // D = 3, as k_init: isotropic, so lambda_zz - 1 = T - 1 as in-plane
      float d[3][N + 1][N + 1];
      z_factor<N>(e, dT, 1.0f, d);
      d[0][0][0] = drho;
      hermite_evaluate3<NR, N>(d, Sv, B.lat);
    }
    const int j = (int)(c / nx);
    if (D.walls && (j == 0 || j == ny - 1)) {
      if (D.wspec != 0.0f) wall_fix<NR, true>(Sv, j == 0 ? 0 : 1, B.lat, D);
      else wall_fix<NR, false>(Sv, j == 0 ? 0 : 1, B.lat, D);
    }
    st_node<NR, S, NZ>(f, c, cells, Sv, B.lat);
  }
}

// Moments (Eq. mac) of every node of every work item whose slot has an output
// in outs[slot] (DEVICE float[9][ny][nx] each, or null): the per-node
// arithmetic of lesbgk_moments, one block per item.
template <int NR, class S, int NZ>
__global__ void __launch_bounds__(kBBlock) k_batch_moments(const BatchArgs B, const int par,
                                                           float *const *__restrict__ outs) {
  const int first = B.range[0], count = B.range[1];
  if ((int)blockIdx.x >= count) return;
  const WorkItem wi = B.items[first + blockIdx.x];
  float *out = outs[wi.inst];
  if (!out) return;
  const InstDesc &D = B.desc[wi.inst];
  const int nx = D.nx;
  const long long cells = (long long)nx * D.ny;
  const S *f = reinterpret_cast<const S *>(D.f[par]);
  for (int t = threadIdx.x; t < wi.rows * nx; t += kBBlock) {
    const long long c = (long long)wi.y0 * nx + t;
    float F[NZ * NR * NR];
    ld_node<NR, S, NZ>(f, c, cells, F, B.lat);
    float d[4];
    node_moments<NR>(F, out, cells, c, B.lat, d);
  }
}

// Guard check: block k compares the kGuardBytes after slot list[k]'s pool
// block (guards[k]) with the pattern written at admission and sets bad[slot]
// when any byte differs.
__global__ void k_batch_guards(const unsigned *const *__restrict__ guards, const int *__restrict__ list, int n,
                               unsigned *__restrict__ bad) {
  if ((int)blockIdx.x >= n) return;
  constexpr unsigned pat = 0x01010101u * kGuardByte;
  const unsigned *g = guards[blockIdx.x];
  bool diff = false;
  for (int t = threadIdx.x; t < (int)(kGuardBytes / 4); t += blockDim.x) diff |= g[t] != pat;
  if (__syncthreads_or(diff) && threadIdx.x == 0) bad[list[blockIdx.x]] = 1u;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, cap) in 256-byte units, coalescing on release.
class Pool {
 public:
  explicit Pool(size_t cap = 0) : cap_(cap) {
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = align_up(bytes, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes, 256);
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest_free() const {
    size_t m = 0;
    for (auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t total_free() const {
    size_t m = 0;
    for (auto &kv : free_) m += kv.second;
    return m;
  }

 private:
  size_t cap_;
  std::map<size_t, size_t> free_;
};

int class_of(int nr, int order, int storage, bool heated, int dim) {
  const int st = storage == LESBGK_F32 ? 0 : storage == LESBGK_F16 ? 1 : storage == LESBGK_BF16 ? 2 : -1;
  if (st < 0) return -1;
  int lat = -1;
  if (dim == 3) lat = nr == 4 && order == 3 ? 2 : -1;
  else if (nr == 4 && order == 3) lat = 0;
  else if (nr == 6 && order == 4) lat = 1;
  if (lat < 0) return -1;
  return lat + 3 * st + (heated ? 9 : 0);
}

// Call fn(NR, N, storage tag, heated, NZ) with the compile-time constants of class cls.
template <class Fn>
void with_class(int cls, Fn &&fn) {
  using R4 = std::integral_constant<int, 4>;
  using R6 = std::integral_constant<int, 6>;
  using N3 = std::integral_constant<int, 3>;
  using N4 = std::integral_constant<int, 4>;
  using Z1 = std::integral_constant<int, 1>;
  using Z2 = std::integral_constant<int, 2>;
  const int lat = cls % 3, st = (cls / 3) % 3;
  const bool heated = cls >= 9;
  auto by_heat = [&](auto r, auto n, auto s, auto z) {
    if (heated) fn(r, n, s, std::true_type{}, z);
    else fn(r, n, s, std::false_type{}, z);
  };
  auto by_storage = [&](auto r, auto n, auto z) {
    if (st == 0) by_heat(r, n, float{}, z);
    else if (st == 1) by_heat(r, n, __half{}, z);
    else by_heat(r, n, __nv_bfloat16{}, z);
  };
  if (lat == 0) by_storage(R4{}, N3{}, Z1{});
  else if (lat == 1) by_storage(R6{}, N4{}, Z1{});
  else by_storage(R4{}, N3{}, Z2{});
}

}  // namespace

struct lesbgk_batch {
  struct Slot {
    bool used = false;
    lesbgk_params p;
    int nr = 0, order = 0, cls = 0;
    size_t off = 0, bytes = 0;
    InstDesc desc;
    KArgs args;
    std::vector<HeatPoly> heat;  // heated walls: the host copy of the slot's polynomials (one), else empty
    double dt = 0, dx = 0, dy = 0, cmax = 0, tau_ref = 0;
    int64_t steps = 0, snap_step = -1;
  };
  char *ws = nullptr;
  size_t ws_bytes = 0;
  int capacity = 0, nx = 0, W = 0;
  InstDesc *d_desc = nullptr;
  WorkItem *d_items = nullptr;
  int *d_range = nullptr;      // {first, count} per class of the items the per-step kernel takes
  int *d_range_all = nullptr;  // {first, count} per class of all items (residuals, moments)
  int *d_rlist = nullptr;      // resident instances, bucket after bucket
  int *d_rrange = nullptr;     // {first, count} per bucket
  unsigned *d_res = nullptr;
  double *d_mass = nullptr;
  int *d_list = nullptr;
  float **d_outs = nullptr;
  double *d_partial = nullptr, *d_sums = nullptr;
  long long *d_nstep = nullptr;
  char *pool_base = nullptr;
  size_t pool_bytes = 0;
  Pool pool;
  std::vector<Slot> slots;
  std::vector<WorkItem> items;
  int range[kNumClasses][2] = {};
  int range_all[kNumClasses][2] = {};
  int rrange[kBuckets][2] = {};
  int max_items = 0;
  bool resident = true;      // D2Q16 instances that fit in shared memory take the resident kernel
  int resident_k = 64;       // time steps per resident launch (divides kGraphSteps)
  int resident_ny = 0;       // tallest instance the resident kernel can hold (shared memory)
  int resident_limit = 128;  // tallest instance it takes (autotuned: a tall one is one block's serial work)
  int graph_rgrid[kBuckets] = {};
  int rows = 32;
  int par = 0;
  int sm_count = 0;
  LatTables lat[kNumClasses];
  bool lat_ready[kNumClasses] = {};
  cudaGraphExec_t graph = nullptr;
  int graph_grid[kNumClasses] = {};
  bool graph_dirty = true;
  bool items_dirty = false;  // slots changed since the work list was uploaded
};

namespace {

constexpr size_t kItemsPerSlot = 1024;  // work-list room: items per slot (rows/8 for ny <= 8192)

struct Layout0 {
  size_t desc, items, mass, range, range_all, rlist, rrange, res, partial, sums, list, outs, nstep, pool;
};

Layout0 fixed_layout(int capacity) {
  Layout0 L{};
  size_t o = 0;
  L.desc = o;
  o = align_up(o + sizeof(InstDesc) * (size_t)capacity, 256);
  L.items = o;
  o = align_up(o + sizeof(WorkItem) * (size_t)capacity * kItemsPerSlot, 256);
  L.mass = o;  // per-item mass partial of the residual pass
  o = align_up(o + sizeof(double) * (size_t)capacity * kItemsPerSlot, 256);
  L.range = o;
  o = align_up(o + sizeof(int) * 2 * kNumClasses, 256);
  L.range_all = o;
  o = align_up(o + sizeof(int) * 2 * kNumClasses, 256);
  L.rlist = o;
  o = align_up(o + sizeof(int) * (size_t)capacity, 256);
  L.rrange = o;
  o = align_up(o + sizeof(int) * 2 * kBuckets, 256);
  L.res = o;
  o = align_up(o + sizeof(unsigned) * (size_t)capacity, 256);
  L.partial = o;
  o = align_up(o + sizeof(double) * 4 * lesbgk_internal::kMomentPartials, 256);
  L.sums = o;
  o = align_up(o + sizeof(double) * 4, 256);
  L.list = o;  // slots to initialise (lesbgk_batch_add_many)
  o = align_up(o + sizeof(int) * (size_t)capacity, 256);
  L.outs = o;  // per-slot moment outputs (lesbgk_batch_moments_many)
  o = align_up(o + sizeof(float *) * (size_t)capacity, 256);
  L.nstep = o;  // per slot and buffer parity: steps done (the heated walls' clock)
  o = align_up(o + sizeof(long long) * 2 * (size_t)capacity, 256);
  L.pool = o;
  return L;
}

size_t elem_bytes(int storage) { return storage == LESBGK_F32 ? sizeof(float) : 2; }

// values stored per node (D = 3: the z-even half)
size_t stored_values(const lesbgk_params &p) {
  return (size_t)p.nroots * p.nroots * (p.dim == 3 ? p.nroots / 2 : 1);
}

size_t slot_bytes(const lesbgk_params &p) {
  const size_t cells = (size_t)p.nx * p.ny;
  const size_t q = stored_values(p);
  const size_t buf = align_up(cells * std::max<size_t>(q * elem_bytes(p.storage), 36), 256);
  const size_t heat = p.wall_T_amp != 0.0 ? align_up(sizeof(HeatPoly), 256) : 0;
  return 2 * buf + align_up(cells * 4 * sizeof(float), 256) + heat + kGuardBytes;
}

// The guard words of a slot: the last kGuardBytes of its pool block.
char *guard_of(const lesbgk_batch *b, const lesbgk_batch::Slot &sl) {
  return b->pool_base + sl.off + sl.bytes - kGuardBytes;
}

bool pow2_le32(int n) { return n >= 1 && n <= 32 && (n & (n - 1)) == 0; }

template <int NR, int N, class S, bool HEAT, int NZ>
void *step_fn(int W) {
  switch (W) {
    case 1: return (void *)k_batch_step<NR, N, 1, S, HEAT, NZ>;
    case 2: return (void *)k_batch_step<NR, N, 2, S, HEAT, NZ>;
    case 4: return (void *)k_batch_step<NR, N, 4, S, HEAT, NZ>;
    case 8: return (void *)k_batch_step<NR, N, 8, S, HEAT, NZ>;
    case 16: return (void *)k_batch_step<NR, N, 16, S, HEAT, NZ>;
    default: return (void *)k_batch_step<NR, N, 32, S, HEAT, NZ>;
  }
}

void *step_kernel(int cls, int W) {
  void *fn = nullptr;
  with_class(cls, [&](auto r, auto n, auto st, auto ht, auto z) {
    fn = step_fn<decltype(r)::value, decltype(n)::value, decltype(st), decltype(ht)::value, decltype(z)::value>(W);
  });
  return fn;
}

size_t step_smem(int cls) {
  size_t b = 0;
  with_class(cls, [&](auto r, auto, auto st, auto, auto z) {
    b = batch_smem_bytes<decltype(r)::value, decltype(st), decltype(z)::value>();
  });
  return b;
}

BatchArgs make_args(const lesbgk_batch *b, int cls) {
  BatchArgs a;
  a.lat = b->lat[cls];
  a.desc = b->d_desc;
  a.items = b->d_items;
  a.range = b->d_range + 2 * cls;
  a.nstep = b->d_nstep;
  return a;
}

// The same over every item of the class, resident instances included
// (residuals, moments).
BatchArgs make_args_all(const lesbgk_batch *b, int cls) {
  BatchArgs a = make_args(b, cls);
  a.range = b->d_range_all + 2 * cls;
  return a;
}

void *resident_fn(int W) {
  switch (W) {
    case 1: return (void *)k_batch_resident<1>;
    case 2: return (void *)k_batch_resident<2>;
    case 4: return (void *)k_batch_resident<4>;
    case 8: return (void *)k_batch_resident<8>;
    case 16: return (void *)k_batch_resident<16>;
    default: return (void *)k_batch_resident<32>;
  }
}

// Rows of bucket k: instances with ny in (bucket_ny(k-1), bucket_ny(k)].
int bucket_ny(const lesbgk_batch *b, int k) { return std::min(16 << k, b->resident_ny); }

size_t resident_smem(const lesbgk_batch *b, int k) {
  return (size_t)2 * 16 * b->nx * bucket_ny(b, k) * sizeof(float);  // two buffers of Q planes
}

bool is_resident(const lesbgk_batch *b, const lesbgk_batch::Slot &sl) {
  return b->resident && sl.cls == 0 &&  // D2Q16 in FP32, steady walls
         sl.p.ny <= std::min(b->resident_ny, b->resident_limit);
}

// K steps of every resident instance: one launch per non-empty bucket.
cudaError_t launch_resident(lesbgk_batch *b, int K, int p_in, int p_out, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  BatchArgs a = make_args(b, 0);
  for (int k = 0; k < kBuckets && e == cudaSuccess; ++k) {
    const int n = b->rrange[k][1];
    if (!n) continue;
    const int *rr = b->d_rrange + 2 * k;
    const int *rl = b->d_rlist;
    void *args[] = {&a, &rl, &rr, &K, &p_in, &p_out};
    e = cudaLaunchKernel(resident_fn(b->W), dim3(n), dim3(kBBlock), args, resident_smem(b, k), s);
  }
  return e;
}

unsigned step_grid(const lesbgk_batch *b, int n_items) {
  const int gpw = 32 / b->W;
  const long long warps = (n_items + gpw - 1) / gpw;
  const long long blocks = (warps * 32 + kBBlock - 1) / kBBlock;
  return (unsigned)std::max<long long>(blocks, 1);
}

cudaError_t launch_one_step(lesbgk_batch *b, int cls, int par, unsigned grid, cudaStream_t s) {
  BatchArgs a = make_args(b, cls);
  void *args[] = {&a, &par};
  return cudaLaunchKernel(step_kernel(cls, b->W), dim3(grid), dim3(kBBlock), args, step_smem(cls), s);
}

// Rebuild the host work list and copy it with the class ranges to the device:
// per class, the items of the instances the per-step kernel takes (sorted by
// length), then those of the resident instances (whose items only the
// residual and moment kernels visit); and the resident instances by bucket.
int rebuild_items(lesbgk_batch *b, cudaStream_t s) {
  b->items.clear();
  for (int cls = 0; cls < kNumClasses; ++cls) {
    const int first = (int)b->items.size();
    std::vector<WorkItem> mine, res;
    for (int i = 0; i < b->capacity; ++i) {
      const auto &sl = b->slots[i];
      if (!sl.used || sl.cls != cls) continue;
      auto &dst = is_resident(b, sl) ? res : mine;
      for (int y0 = 0; y0 < sl.p.ny; y0 += b->rows) dst.push_back({i, y0, std::min(b->rows, sl.p.ny - y0), 0});
    }
    std::stable_sort(mine.begin(), mine.end(), [](const WorkItem &x, const WorkItem &y) { return x.rows > y.rows; });
    b->items.insert(b->items.end(), mine.begin(), mine.end());
    b->items.insert(b->items.end(), res.begin(), res.end());
    b->range[cls][0] = first;
    b->range[cls][1] = (int)mine.size();
    b->range_all[cls][0] = first;
    b->range_all[cls][1] = (int)(mine.size() + res.size());
  }
  if ((long long)b->items.size() > (long long)b->capacity * (long long)kItemsPerSlot)
    return fail(LESBGK_ESPACE, "work list of %zu items exceeds its room", b->items.size());
  std::vector<int> rlist;
  for (int k = 0; k < kBuckets; ++k) {
    b->rrange[k][0] = (int)rlist.size();
    for (int i = 0; i < b->capacity; ++i) {
      const auto &sl = b->slots[i];
      if (sl.used && is_resident(b, sl) && sl.p.ny <= bucket_ny(b, k) && (k == 0 || sl.p.ny > bucket_ny(b, k - 1)))
        rlist.push_back(i);
    }
    b->rrange[k][1] = (int)rlist.size() - b->rrange[k][0];
  }
  cudaError_t e = cudaSuccess;
  if (!b->items.empty())
    e = cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(WorkItem) * b->items.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_range, b->range, sizeof(b->range), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_range_all, b->range_all, sizeof(b->range_all), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !rlist.empty())
    e = cudaMemcpyAsync(b->d_rlist, rlist.data(), sizeof(int) * rlist.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_rrange, b->rrange, sizeof(b->rrange), cudaMemcpyHostToDevice, s);
  // (pageable sources: the copies are staged before cudaMemcpyAsync returns,
  // so the host vectors may change afterwards)
  if (e != cudaSuccess) return cuda_fail(e, "work list upload");
  b->items_dirty = false;
  for (int cls = 0; cls < kNumClasses; ++cls)
    if ((int)step_grid(b, b->range[cls][1]) > b->graph_grid[cls]) b->graph_dirty = true;
  for (int k = 0; k < kBuckets; ++k)
    if (b->rrange[k][1] > b->graph_rgrid[k]) b->graph_dirty = true;
  return 0;
}

int ensure_items(lesbgk_batch *b, cudaStream_t s) { return b->items_dirty ? rebuild_items(b, s) : 0; }

void drop_graph(lesbgk_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_dirty = true;
}

// A graph of kGraphSteps steps: per step one launch per lattice class present,
// each step after the previous one; grids sized with head room for the
// current work list (kernels read their item counts from device memory, so
// the graph stays valid while slots come and go).
int build_graph(lesbgk_batch *b) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  BatchArgs args[kNumClasses];
  int pars[2] = {0, 1};
  std::vector<cudaGraphNode_t> prev;
  for (int cls = 0; cls < kNumClasses; ++cls) {
    const int n = b->range[cls][1];
    b->graph_grid[cls] = n ? (int)step_grid(b, n + n / 4 + 64) : 0;
    args[cls] = make_args(b, cls);
  }
  for (int st = 0; st < kGraphSteps && e == cudaSuccess; ++st) {
    std::vector<cudaGraphNode_t> cur;
    for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls) {
      if (!b->graph_grid[cls]) continue;
      cudaKernelNodeParams kp{};
      void *kargs[] = {&args[cls], &pars[st & 1]};
      kp.func = step_kernel(cls, b->W);
      kp.gridDim = dim3(b->graph_grid[cls]);
      kp.blockDim = dim3(kBBlock);
      kp.sharedMemBytes = (unsigned)step_smem(cls);
      kp.kernelParams = kargs;
      cudaGraphNode_t node;
      e = cudaGraphAddKernelNode(&node, g, prev.empty() ? nullptr : prev.data(), prev.size(), &kp);
      cur.push_back(node);
    }
    if (!cur.empty()) prev = cur;
  }
  // resident instances: per bucket a chain of kGraphSteps / resident_k launches,
  // each taking resident_k steps in place (an even count: parity 0 to 0),
  // independent of the per-step chain (they touch other instances)
  BatchArgs a0 = make_args(b, 0);
  const int *rl = b->d_rlist;
  int K = b->resident_k, p0 = 0;
  for (int k = 0; k < kBuckets && e == cudaSuccess; ++k) {
    const int n = b->rrange[k][1];
    b->graph_rgrid[k] = n ? n + n / 4 + 8 : 0;
    if (!n) continue;
    const int *rr = b->d_rrange + 2 * k;
    cudaGraphNode_t last = nullptr;
    for (int c = 0; c < kGraphSteps / K && e == cudaSuccess; ++c) {
      cudaKernelNodeParams kp{};
      void *kargs[] = {&a0, &rl, &rr, &K, &p0, &p0};
      kp.func = resident_fn(b->W);
      kp.gridDim = dim3(b->graph_rgrid[k]);
      kp.blockDim = dim3(kBBlock);
      kp.sharedMemBytes = (unsigned)resident_smem(b, k);
      kp.kernelParams = kargs;
      cudaGraphNode_t node;
      e = cudaGraphAddKernelNode(&node, g, last ? &last : nullptr, last ? 1 : 0, &kp);
      last = node;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return cuda_fail(e, "building the step graph");
  }
  b->graph_dirty = false;
  return 0;
}

}  // namespace

extern "C" int lesbgk_batch_workspace_size(int32_t capacity, size_t pool_bytes, size_t *bytes) {
  if (capacity < 1 || capacity > (1 << 20)) return fail(LESBGK_EINVAL, "capacity must be in [1, 2^20]");
  if (!bytes) return fail(LESBGK_EINVAL, "bytes is NULL");
  *bytes = fixed_layout(capacity).pool + align_up(pool_bytes, 256);
  return 0;
}

extern "C" int lesbgk_batch_slot_bytes(const lesbgk_params *p, size_t *bytes) {
  if (int rc = check_params(p)) return rc;
  if (!bytes) return fail(LESBGK_EINVAL, "bytes is NULL");
  *bytes = align_up(slot_bytes(*p), 256);
  return 0;
}

extern "C" int lesbgk_batch_create(int32_t capacity, int32_t nx, void *d_workspace, size_t bytes, void *stream,
                                   lesbgk_batch **out) {
  clear_error();
  if (!out) return fail(LESBGK_EINVAL, "out is NULL");
  *out = nullptr;
  if (capacity < 1 || capacity > (1 << 20)) return fail(LESBGK_EINVAL, "capacity must be in [1, 2^20]");
  if (!pow2_le32(nx)) return fail(LESBGK_EINVAL, "batched instances need nx in {1, 2, 4, 8, 16, 32}");
  const Layout0 L = fixed_layout(capacity);
  if (!d_workspace || bytes < L.pool + 256) return fail(LESBGK_ESPACE, "workspace %zu bytes < %zu", bytes, L.pool + 256);
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256) return fail(LESBGK_ESPACE, "workspace not 256-byte aligned");
  lesbgk_batch *b = new (std::nothrow) lesbgk_batch();
  if (!b) return fail(LESBGK_EINVAL, "out of host memory");
  b->ws = static_cast<char *>(d_workspace);
  b->ws_bytes = bytes;
  b->capacity = capacity;
  b->nx = nx;
  b->W = nx;
  b->d_desc = reinterpret_cast<InstDesc *>(b->ws + L.desc);
  b->d_items = reinterpret_cast<WorkItem *>(b->ws + L.items);
  b->d_range = reinterpret_cast<int *>(b->ws + L.range);
  b->d_range_all = reinterpret_cast<int *>(b->ws + L.range_all);
  b->d_rlist = reinterpret_cast<int *>(b->ws + L.rlist);
  b->d_rrange = reinterpret_cast<int *>(b->ws + L.rrange);
  b->d_res = reinterpret_cast<unsigned *>(b->ws + L.res);
  b->d_mass = reinterpret_cast<double *>(b->ws + L.mass);
  b->d_list = reinterpret_cast<int *>(b->ws + L.list);
  b->d_outs = reinterpret_cast<float **>(b->ws + L.outs);
  b->d_nstep = reinterpret_cast<long long *>(b->ws + L.nstep);
  b->d_partial = reinterpret_cast<double *>(b->ws + L.partial);
  b->d_sums = reinterpret_cast<double *>(b->ws + L.sums);
  b->pool_base = b->ws + L.pool;
  b->pool_bytes = bytes - L.pool;
  b->pool = Pool(b->pool_bytes / 256 * 256);
  b->slots.resize(capacity);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  for (int w : {1, 2, 4, 8, 16, 32})
    for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls)
      e = cudaFuncSetAttribute(step_kernel(cls, w), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem(cls));
  // the resident kernel: as tall an instance as two buffers of Q planes fit in
  // the opt-in shared memory of a block
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  b->resident_ny = std::min(16 << (kBuckets - 1), optin / (2 * 16 * nx * (int)sizeof(float)));
  for (int w : {1, 2, 4, 8, 16, 32})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(resident_fn(w), cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_range, 0, sizeof(int) * 2 * kNumClasses, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_range_all, 0, sizeof(int) * 2 * kNumClasses, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_rrange, 0, sizeof(int) * 2 * kBuckets, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch set-up");
  }
  *out = b;
  return 0;
}

namespace {

// Validate p, build its tables and take a slot and pool memory for it; the
// slot's descriptor is filled on the host (sl.desc), not yet on the device.
int prepare_slot(lesbgk_batch *b, const lesbgk_params *p, const double *h_init, int *slot_out) {
  if (int rc = check_params(p)) return rc;
  const int order = p->order ? p->order : default_order(p->nroots);
  if (p->storage == LESBGK_F32C) return fail(LESBGK_EINVAL, "batched instances store FP32, FP16 or BF16 populations");
  const int cls = class_of(p->nroots, order, p->storage, p->wall_T_amp != 0.0, p->dim == 3 ? 3 : 2);
  if (cls < 0) return fail(LESBGK_EINVAL, "batched instances take D2Q16 (order 3), D2Q36 (order 4) or D3Q64");
  if (p->nx != b->nx) return fail(LESBGK_EINVAL, "instance nx %d differs from the batch's %d", p->nx, b->nx);
  if (p->bc_x != LESBGK_PERIODIC) return fail(LESBGK_EINVAL, "batched instances are periodic in x");
  if ((long long)(p->ny + b->rows - 1) / b->rows > (long long)kItemsPerSlot)
    return fail(LESBGK_EINVAL, "ny %d too large for the batch work list", p->ny);
  int slot = -1;
  for (int i = 0; i < b->capacity; ++i)
    if (!b->slots[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) return fail(LESBGK_ESPACE, "all %d slots are in use", b->capacity);
  Setup su;
  FieldStats stats{1.0, 1.0, -1};
  if (h_init) stats = field_stats_host(h_init, (size_t)p->nx * p->ny);  // small instances: a host loop
  if (int rc = build_setup(*p, order, h_init ? &stats : nullptr, &su)) return rc;
  size_t off = 0;
  const size_t need = slot_bytes(*p);
  if (!b->pool.alloc(need, &off))
    return fail(LESBGK_ESPACE, "pool has no free block of %zu bytes (largest %zu)", need, b->pool.largest_free());
  auto &sl = b->slots[slot];
  sl = lesbgk_batch::Slot();
  sl.p = *p;
  sl.nr = p->nroots;
  sl.order = order;
  sl.cls = cls;
  sl.off = off;
  sl.bytes = need;
  sl.args = su.args;
  sl.dt = su.dt;
  sl.dx = su.dx;
  sl.dy = su.dy;
  sl.cmax = su.cmax;
  sl.tau_ref = su.tau_ref;
  const size_t cells = (size_t)p->nx * p->ny;
  const size_t q = stored_values(*p);
  const size_t buf = align_up(cells * std::max<size_t>(q * elem_bytes(p->storage), 36), 256);
  char *base = b->pool_base + off;
  InstDesc &D = sl.desc;
  std::memset(&D, 0, sizeof D);
  D.f[b->par] = reinterpret_cast<float *>(base);
  D.f[b->par ^ 1] = reinterpret_cast<float *>(base + buf);
  D.snap = reinterpret_cast<float *>(base + 2 * buf);
  if (p->wall_T_amp != 0.0) {  // the polynomials follow the snapshot (uploaded with the descriptor)
    sl.heat.assign(1, su.heat);
    D.heat = reinterpret_cast<const HeatPoly *>(base + 2 * buf + align_up(cells * 4 * sizeof(float), 256));
  }
  const KArgs &A = su.args;
  D.nx = p->nx;
  D.ny = p->ny;
  D.walls = A.walls;
  D.split = p->scheme == LESBGK_SPLIT;
  D.vmode = A.vmode;
  D.has_force = A.has_force;
  D.c_omega = A.c_omega;
  D.visc_pow = A.visc_pow;
  D.b = A.b;
  D.beta = A.beta;
  D.dtgx = A.dtgx;
  D.dtgy = A.dtgy;
  D.dt = (float)su.dt;
  D.wspec = A.wspec;
  std::memcpy(D.ax, A.ax, sizeof D.ax);
  std::memcpy(D.kx, A.kx, sizeof D.kx);
  std::memcpy(D.ay, A.ay, sizeof D.ay);
  std::memcpy(D.ky, A.ky, sizeof D.ky);
  for (int side = 0; side < 2; ++side) {  // the batch's rows are shorter (2D sets only)
    std::memcpy(D.wS[side], A.wS[side], sizeof D.wS[side]);
    std::memcpy(D.wSdev[side], A.wSdev[side], sizeof D.wSdev[side]);
  }
  std::memcpy(D.wA, A.wA, sizeof D.wA);
  std::memcpy(D.wB, A.wB, sizeof D.wB);
  if (!b->lat_ready[cls]) {
    LatTables &lt = b->lat[cls];
    std::memcpy(lt.c, A.c, sizeof lt.c);
    std::memcpy(lt.he, A.he, sizeof lt.he);
    std::memcpy(lt.hw, A.hw, sizeof lt.hw);
    std::memcpy(lt.wq, A.wq, sizeof lt.wq);  // (the 2D sets: the first kMaxQ entries)
    std::memcpy(lt.iwq, A.iwq, sizeof lt.iwq);
    b->lat_ready[cls] = true;
    drop_graph(b);
  }
  *slot_out = slot;
  return 0;
}

// Wait for the copy of a pinned h_init before returning (a pageable one is
// staged before cudaMemcpyAsync returns).
cudaError_t settle_host_copy(const double *h_init, cudaStream_t s) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaSuccess;
  if (cudaPointerGetAttributes(&at, h_init) == cudaSuccess && at.type == cudaMemoryTypeHost)
    e = cudaStreamSynchronize(s);
  cudaGetLastError();
  return e;
}

void release_slot(lesbgk_batch *b, int slot) {
  auto &sl = b->slots[slot];
  b->pool.release(sl.off, sl.bytes);
  sl = lesbgk_batch::Slot();
}

}  // namespace

extern "C" int lesbgk_batch_add(lesbgk_batch *b, const lesbgk_params *p, const double *h_init, void *stream,
                                int32_t *slot_out) {
  lesbgk_internal::Range range_("lesbgk_batch_add");
  if (!b || !slot_out) return fail(LESBGK_EINVAL, "NULL argument");
  int slot = -1;
  if (int rc = prepare_slot(b, p, h_init, &slot)) return rc;
  auto &sl = b->slots[slot];
  const InstDesc &D = sl.desc;
  const size_t cells = (size_t)p->nx * p->ny;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(b->d_desc + slot, &D, sizeof D, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_nstep + 2 * slot + b->par, 0, sizeof(long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(guard_of(b, sl), kGuardByte, kGuardBytes, s);
  if (e == cudaSuccess && D.heat)  // (pageable host copy: staged before the call returns)
    e = cudaMemcpyAsync(const_cast<HeatPoly *>(D.heat), sl.heat.data(), sizeof(HeatPoly), cudaMemcpyHostToDevice, s);
  const double *dfields = nullptr;
  if (e == cudaSuccess && h_init) {
    e = cudaMemcpyAsync(D.f[b->par ^ 1], h_init, 4 * cells * sizeof(double), cudaMemcpyHostToDevice, s);
    dfields = reinterpret_cast<const double *>(D.f[b->par ^ 1]);
  }
  if (e == cudaSuccess)
    e = lesbgk_internal::launch_init(sl.args, sl.nr, sl.order, p->storage, p->dim, dfields, D.f[b->par], b->sm_count,
                                     s);
  if (e == cudaSuccess && h_init) e = settle_host_copy(h_init, s);
  if (e != cudaSuccess) {
    release_slot(b, slot);
    return cuda_fail(e, "slot initialisation");
  }
  sl.used = true;
  b->items_dirty = true;  // the work list is rebuilt before the next step
  *slot_out = slot;
  return 0;
}

extern "C" int lesbgk_batch_add_many(lesbgk_batch *b, int32_t n, const lesbgk_params *ps,
                                     const double *const *h_inits, void *stream, int32_t *slots_out) {
  lesbgk_internal::Range range_("lesbgk_batch_add_many");
  if (!b || n < 0 || (n && (!ps || !slots_out))) return fail(LESBGK_EINVAL, "NULL argument");
  std::vector<int> taken;
  taken.reserve(n);
  int rc = 0;
  for (int i = 0; i < n && !rc; ++i) {
    int slot = -1;
    rc = prepare_slot(b, &ps[i], h_inits ? h_inits[i] : nullptr, &slot);
    if (!rc) {
      b->slots[slot].used = true;  // taken for the rest of this call
      taken.push_back(slot);
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!rc && n) {
    // the descriptors of the touched range in one copy, the fields one by one,
    // then one init launch per lattice class over the new slots
    const int lo = *std::min_element(taken.begin(), taken.end());
    const int hi = *std::max_element(taken.begin(), taken.end());
    std::vector<InstDesc> desc(hi - lo + 1);
    for (int i = lo; i <= hi; ++i)
      if (b->slots[i].used) desc[i - lo] = b->slots[i].desc;
    // (slots in the range not taken here keep their device descriptors: copy
    // them back unchanged from the host mirror, which is the same data)
    e = cudaMemcpyAsync(b->d_desc + lo, desc.data(), sizeof(InstDesc) * desc.size(), cudaMemcpyHostToDevice, s);
    std::vector<int> list[kNumClasses];
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      const auto &sl = b->slots[taken[i]];
      e = cudaMemsetAsync(guard_of(b, sl), kGuardByte, kGuardBytes, s);
      if (e == cudaSuccess && sl.desc.heat)
        e = cudaMemcpyAsync(const_cast<HeatPoly *>(sl.desc.heat), sl.heat.data(), sizeof(HeatPoly),
                            cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) break;
      const double *hi_init = h_inits ? h_inits[i] : nullptr;
      if (hi_init)
        e = cudaMemcpyAsync(sl.desc.f[b->par ^ 1], hi_init, 4 * (size_t)sl.p.nx * sl.p.ny * sizeof(double),
                            cudaMemcpyHostToDevice, s);
      list[sl.cls].push_back(taken[i] | (hi_init ? (1 << 30) : 0));
    }
    int at = 0;
    for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls) {
      const int m = (int)list[cls].size();
      if (!m) continue;
      e = cudaMemcpyAsync(b->d_list + at, list[cls].data(), sizeof(int) * m, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) break;
      BatchArgs a = make_args(b, cls);
      const int *lst = b->d_list + at;
      with_class(cls, [&](auto r, auto nn, auto st, auto, auto z) {
        k_batch_init<decltype(r)::value, decltype(nn)::value, decltype(st), decltype(z)::value>
            <<<m, kBBlock, 0, s>>>(a, lst, m, b->par);
      });
      e = cudaGetLastError();
      at += m;
    }
    // host arrays above are pageable (staged at once); pinned fields are waited for
    for (int i = 0; i < n && e == cudaSuccess && h_inits; ++i)
      if (h_inits[i]) e = settle_host_copy(h_inits[i], s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the list and descriptor staging buffers
  }
  if (rc || e != cudaSuccess) {
    for (int slot : taken) release_slot(b, slot);
    return rc ? rc : cuda_fail(e, "batched slot initialisation");
  }
  for (int i = 0; i < n; ++i) slots_out[i] = taken[i];
  b->items_dirty = true;
  return 0;
}

extern "C" int lesbgk_batch_remove(lesbgk_batch *b, int32_t slot, void *stream) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return fail(LESBGK_EINVAL, "no such slot");
  auto &sl = b->slots[slot];
  // the slot's buffers may still be read by queued steps: order the release
  // after them on the stream, then rebuild the work list
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "slot removal");
  sl.used = false;
  b->items_dirty = true;
  b->pool.release(sl.off, sl.bytes);
  return 0;
}

extern "C" int lesbgk_batch_step(lesbgk_batch *b, int64_t nsteps, void *stream) {
  lesbgk_internal::Range range_("lesbgk_batch_step");
  if (!b) return fail(LESBGK_EINVAL, "batch is NULL");
  if (nsteps < 0) return fail(LESBGK_EINVAL, "nsteps < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = ensure_items(b, s)) return rc;
  cudaError_t e = cudaSuccess;
  auto direct_step = [&]() {
    for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls)
      if (b->range[cls][1]) e = launch_one_step(b, cls, b->par, step_grid(b, b->range[cls][1]), s);
    if (e == cudaSuccess) e = launch_resident(b, 1, b->par, b->par ^ 1, s);
    if (e == cudaSuccess) {
      b->par ^= 1;  // the slots' current buffers are desc.f[par]
      for (auto &sl : b->slots)
        if (sl.used) sl.steps += 1;
    }
  };
  if (nsteps >= kGraphSteps) {
    if (b->par == 1) {  // the graph's steps run parity 0, 1, 0, ...
      direct_step();
      --nsteps;
    }
    if (e == cudaSuccess && (b->graph_dirty || !b->graph))
      if (int rc = build_graph(b)) return rc;
  }
  while (nsteps >= kGraphSteps && e == cudaSuccess) {
    e = cudaGraphLaunch(b->graph, s);
    nsteps -= kGraphSteps;
    for (auto &sl : b->slots)
      if (sl.used) sl.steps += kGraphSteps;
  }
  for (; nsteps > 0 && e == cudaSuccess; --nsteps) direct_step();
  if (e != cudaSuccess) return cuda_fail(e, "batch step");
  return 0;
}

extern "C" int lesbgk_batch_residuals(lesbgk_batch *b, double *h_res, double *h_mass, void *stream) {
  lesbgk_internal::Range range_("lesbgk_batch_residuals");
  if (!b || !h_res) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = ensure_items(b, s)) return rc;
  cudaError_t e = cudaMemsetAsync(b->d_res, 0, sizeof(unsigned) * b->capacity, s);
  for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls) {
    const int n = b->range_all[cls][1];
    if (!n) continue;
    BatchArgs a = make_args_all(b, cls);
    with_class(cls, [&](auto r, auto, auto st, auto, auto z) {
      k_batch_residual<decltype(r)::value, decltype(st), decltype(z)::value>
          <<<n, kBBlock, 0, s>>>(a, b->par, b->d_res, b->d_mass);
    });
    e = cudaGetLastError();
  }
  std::vector<unsigned> bits(b->capacity);
  std::vector<double> part(h_mass ? b->items.size() : 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bits.data(), b->d_res, sizeof(unsigned) * b->capacity, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !part.empty())
    e = cudaMemcpyAsync(part.data(), b->d_mass, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "batch residuals");
  for (int i = 0; i < b->capacity; ++i) {
    auto &sl = b->slots[i];
    h_res[i] = NAN;
    if (h_mass) h_mass[i] = NAN;
    if (!sl.used) continue;
    float r;
    std::memcpy(&r, &bits[i], sizeof r);
    if (sl.snap_step >= 0 && sl.steps > sl.snap_step) h_res[i] = r / ((double)(sl.steps - sl.snap_step) * sl.dt);
    else if (sl.snap_step >= 0) h_res[i] = 0.0;
    sl.snap_step = sl.steps;
    if (h_mass) h_mass[i] = (double)sl.p.nx * sl.p.ny;
  }
  if (h_mass)  // the items' partials in work-list order: reproducible
    for (size_t k = 0; k < part.size(); ++k) h_mass[b->items[k].inst] += part[k];
  return 0;
}

extern "C" int lesbgk_batch_moments(lesbgk_batch *b, int32_t slot, float *d_out, double *h_sums, void *stream) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return fail(LESBGK_EINVAL, "no such slot");
  auto &sl = b->slots[slot];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = lesbgk_internal::launch_moments(sl.args, sl.nr, sl.order, sl.p.storage, sl.p.dim, sl.desc.f[b->par],
                                                  d_out, b->d_partial, b->d_sums, s);
  if (e == cudaSuccess && h_sums) {
    e = cudaMemcpyAsync(h_sums, b->d_sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch moments");
  if (h_sums)
    for (int k = 0; k < 4; ++k)
      if (!std::isfinite(h_sums[k])) return fail(LESBGK_EDIVERGED, "slot %d diverged", slot);
  return 0;
}

extern "C" int lesbgk_batch_moments_many(lesbgk_batch *b, int32_t n, const int32_t *slots, float *const *d_outs,
                                         void *stream) {
  lesbgk_internal::Range range_("lesbgk_batch_moments_many");
  if (!b || n < 0 || (n && (!slots || !d_outs))) return fail(LESBGK_EINVAL, "NULL argument");
  std::vector<float *> outs(b->capacity, nullptr);
  for (int i = 0; i < n; ++i) {
    const int sl = slots[i];
    if (sl < 0 || sl >= b->capacity || !b->slots[sl].used) return fail(LESBGK_EINVAL, "no such slot %d", sl);
    if (!d_outs[i]) return fail(LESBGK_EINVAL, "output %d is NULL", i);
    outs[sl] = d_outs[i];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = ensure_items(b, s)) return rc;
  cudaError_t e = cudaMemcpyAsync(b->d_outs, outs.data(), sizeof(float *) * outs.size(), cudaMemcpyHostToDevice, s);
  for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls) {
    const int m = b->range_all[cls][1];
    if (!m) continue;
    BatchArgs a = make_args_all(b, cls);
    with_class(cls, [&](auto r, auto, auto st, auto, auto z) {
      k_batch_moments<decltype(r)::value, decltype(st), decltype(z)::value><<<m, kBBlock, 0, s>>>(a, b->par, b->d_outs);
    });
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "batched moments");
  return 0;
}

extern "C" int lesbgk_batch_get_populations(lesbgk_batch *b, int32_t slot, float *d_out, void *stream) {
  if (!b || !d_out || slot < 0 || slot >= b->capacity || !b->slots[slot].used)
    return fail(LESBGK_EINVAL, "no such slot");
  auto &sl = b->slots[slot];
  cudaError_t e = lesbgk_internal::launch_ungroup(sl.args, sl.nr, sl.order, sl.p.storage, sl.p.dim, sl.desc.f[b->par],
                                                  d_out,
                                                  (long long)sl.p.nx * sl.p.ny, b->sm_count,
                                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : cuda_fail(e, "batch populations");
}

namespace {

size_t raw_bytes(const lesbgk_batch::Slot &sl) {
  return (size_t)sl.p.nx * sl.p.ny * stored_values(sl.p) * elem_bytes(sl.p.storage);
}

}  // namespace

extern "C" int lesbgk_batch_raw_bytes(const lesbgk_batch *b, int32_t slot, size_t *bytes) {
  if (!b || !bytes || slot < 0 || slot >= b->capacity || !b->slots[slot].used)
    return fail(LESBGK_EINVAL, "no such slot");
  *bytes = raw_bytes(b->slots[slot]);
  return 0;
}

extern "C" int lesbgk_batch_get_raw(lesbgk_batch *b, int32_t slot, void *d_out, void *stream) {
  if (!b || !d_out || slot < 0 || slot >= b->capacity || !b->slots[slot].used)
    return fail(LESBGK_EINVAL, "no such slot");
  const auto &sl = b->slots[slot];
  cudaError_t e = cudaMemcpyAsync(d_out, sl.desc.f[b->par], raw_bytes(sl), cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : cuda_fail(e, "batch raw populations");
}

extern "C" int lesbgk_batch_set_raw(lesbgk_batch *b, int32_t slot, const void *d_in, int64_t steps_done,
                                   void *stream) {
  if (!b || !d_in || slot < 0 || slot >= b->capacity || !b->slots[slot].used)
    return fail(LESBGK_EINVAL, "no such slot");
  if (steps_done < 0) return fail(LESBGK_EINVAL, "steps_done < 0");
  auto &sl = b->slots[slot];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = steps_done;
  cudaError_t e = cudaMemcpyAsync(sl.desc.f[b->par], d_in, raw_bytes(sl), cudaMemcpyDeviceToDevice, s);
  // the slot's clock (heated walls, 16-bit rounding keys) resumes at steps_done
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_nstep + 2 * slot + b->par, &n, sizeof n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // (n is on this stack frame)
  if (e != cudaSuccess) return cuda_fail(e, "batch raw populations");
  sl.steps = steps_done;
  sl.snap_step = -1;  // the residual snapshot is of the state replaced
  return 0;
}

extern "C" int lesbgk_batch_get_info(const lesbgk_batch *b, int32_t slot, lesbgk_info *out) {
  if (!b || !out || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return fail(LESBGK_EINVAL, "no such slot");
  const auto &sl = b->slots[slot];
  out->dt = sl.dt;
  out->dx = sl.dx;
  out->dy = sl.dy;
  out->c_max = sl.cmax;
  out->cfl = sl.cmax * sl.dt / std::fmin(sl.dx, sl.dy);
  out->tau_ref = sl.tau_ref;
  out->steps_done = sl.steps;
  out->q = (int)stored_values(sl.p);
  out->order = sl.order;
  out->cells_per_thread = 1;
  out->rows_per_segment = b->rows;
  return 0;
}

extern "C" int lesbgk_batch_set_rows(lesbgk_batch *b, int32_t rows, void *stream) {
  if (!b || rows < 1 || rows > 4096) return fail(LESBGK_EINVAL, "rows must be in [1, 4096]");
  for (auto &sl : b->slots)
    if (sl.used && (long long)(sl.p.ny + rows - 1) / rows > (long long)kItemsPerSlot)
      return fail(LESBGK_EINVAL, "rows %d too short for ny %d", rows, sl.p.ny);
  b->rows = rows;
  drop_graph(b);
  return rebuild_items(b, static_cast<cudaStream_t>(stream));
}

extern "C" int lesbgk_batch_set_resident(lesbgk_batch *b, int32_t on, int32_t steps_per_launch, int32_t max_ny,
                                         void *stream) {
  if (!b) return fail(LESBGK_EINVAL, "batch is NULL");
  if (max_ny < 0) return fail(LESBGK_EINVAL, "max_ny must be >= 0");
  if (max_ny) b->resident_limit = max_ny;
  if (steps_per_launch && (steps_per_launch < 2 || steps_per_launch > kGraphSteps || (steps_per_launch & 1) ||
                           kGraphSteps % steps_per_launch))
    return fail(LESBGK_EINVAL, "steps per resident launch must be an even divisor of %d", kGraphSteps);
  b->resident = on != 0;
  if (steps_per_launch) b->resident_k = steps_per_launch;
  drop_graph(b);
  return rebuild_items(b, static_cast<cudaStream_t>(stream));
}

extern "C" int lesbgk_batch_get_launch(const lesbgk_batch *b, int32_t *rows, int32_t *resident,
                                       int32_t *steps_per_launch, int32_t *resident_max_ny) {
  if (!b) return fail(LESBGK_EINVAL, "batch is NULL");
  if (rows) *rows = b->rows;
  if (resident) *resident = b->resident ? 1 : 0;
  if (steps_per_launch) *steps_per_launch = b->resident_k;
  if (resident_max_ny) *resident_max_ny = std::min(b->resident_ny, b->resident_limit);
  return 0;
}

extern "C" int lesbgk_batch_autotune(lesbgk_batch *b, const int32_t *candidates, int32_t n, int32_t *chosen,
                                     void *stream) {
  lesbgk_internal::Range range_("lesbgk_batch_autotune");
  if (!b || !candidates || n < 1) return fail(LESBGK_EINVAL, "bad autotune arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStream_t s2 = nullptr;
  cudaEvent_t t0, t1, fork, join;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "autotune set-up");
  // candidates: rows per work item x {per-step kernel for all, resident
  // kernel with 16 or 64 steps per launch}; each timed as a 64-step chunk,
  // the resident launches on a second stream beside the per-step chain (as in
  // the graph), every launch reading the current buffers and writing the
  // spare ones, so the state is left untouched
  struct Cand { int rows, res, k, limit; };
  std::vector<Cand> cands;
  for (int c = 0; c < n; ++c) {
    cands.push_back({candidates[c], 0, b->resident_k, b->resident_limit});
    for (int lim : {64, 128, 256, 1 << 30})
      for (int k : {16, 64}) cands.push_back({candidates[c], 1, k, lim});
  }
  Cand best{b->rows, b->resident ? 1 : 0, b->resident_k, b->resident_limit};
  float best_ms = 1e30f;
  int rc = 0;
  for (const Cand &cd : cands) {
    b->resident = cd.res != 0;
    b->resident_k = cd.k;
    b->resident_limit = cd.limit;
    if ((rc = lesbgk_batch_set_rows(b, cd.rows, stream))) break;
    float ms = 0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(t0, s);
      if (e == cudaSuccess) e = cudaEventRecord(fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, fork, 0);
      for (int c = 0; c < kGraphSteps / cd.k && e == cudaSuccess; ++c) e = launch_resident(b, cd.k, b->par, b->par ^ 1, s2);
      if (e == cudaSuccess) e = cudaEventRecord(join, s2);
      for (int st = 0; st < kGraphSteps && e == cudaSuccess; ++st)
        for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls)
          if (b->range[cls][1]) e = launch_one_step(b, cls, b->par, step_grid(b, b->range[cls][1]), s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join, 0);
      if (e == cudaSuccess) e = cudaEventRecord(t1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    }
    if (e != cudaSuccess) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = cd;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaEventDestroy(fork);
  cudaEventDestroy(join);
  cudaStreamDestroy(s2);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  b->resident = best.res != 0;
  b->resident_k = best.k;
  b->resident_limit = best.limit;
  if (chosen) *chosen = best.rows;
  return lesbgk_batch_set_rows(b, best.rows, stream);
}

extern "C" int lesbgk_batch_check_guards(lesbgk_batch *b, int32_t *h_bad, void *stream) {
  if (!b || !h_bad) return fail(LESBGK_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const unsigned *> guards;
  std::vector<int> list;
  for (int i = 0; i < b->capacity; ++i)
    if (b->slots[i].used) {
      guards.push_back(reinterpret_cast<const unsigned *>(guard_of(b, b->slots[i])));
      list.push_back(i);
    }
  std::vector<unsigned> bad(b->capacity, 0u);
  cudaError_t e = cudaMemsetAsync(b->d_res, 0, sizeof(unsigned) * b->capacity, s);
  if (e == cudaSuccess && !list.empty()) {
    // (the pointer and slot lists go through the moment-output and admission
    // scratch of the workspace; pageable sources are staged at once)
    e = cudaMemcpyAsync(b->d_outs, guards.data(), sizeof(void *) * guards.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_batch_guards<<<(unsigned)list.size(), 64, 0, s>>>(reinterpret_cast<const unsigned *const *>(b->d_outs),
                                                          b->d_list, (int)list.size(), b->d_res);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad.data(), b->d_res, sizeof(unsigned) * b->capacity, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "guard check");
  for (int i = 0; i < b->capacity; ++i) h_bad[i] = (int32_t)bad[i];
  return 0;
}

extern "C" int lesbgk_batch_debug_poison(lesbgk_batch *b, int32_t slot, void *stream) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return fail(LESBGK_EINVAL, "no such slot");
  cudaError_t e = cudaMemsetAsync(guard_of(b, b->slots[slot]) + kGuardBytes / 2, 0, 4, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : cuda_fail(e, "guard poison");
}

extern "C" int lesbgk_batch_pool_free(const lesbgk_batch *b, size_t *largest, size_t *total) {
  if (!b) return fail(LESBGK_EINVAL, "batch is NULL");
  if (largest) *largest = b->pool.largest_free();
  if (total) *total = b->pool.total_free();
  return 0;
}

extern "C" int lesbgk_batch_destroy(lesbgk_batch *b) {
  if (!b) return 0;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
  return 0;
}
