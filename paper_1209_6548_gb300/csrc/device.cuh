// Device code shared by the lattice ES-BGK kernels (single domain and
// batched): limiter, row mapping, the grouped population layout, the
// per-node Hermite collision (Sec. 2.2) and the diffuse wall (Sec. 3.2).
//
// Velocity sets: the D = 2 tensor-product sets (Q = NR^2, population
// alpha = ix*NR + iy) and the D = 3 set with NR^3 velocities on the same
// two-dimensional grid, stored by its z-even half: nothing varies in z and
// the walls and forces have no z component, so a state even in c_z stays
// even; populations (ix, iy, +c_z) and (ix, iy, -c_z) are equal and one value
// (alpha = iz*NR^2 + ix*NR + iy, c_z = c[NR/2 + iz] > 0) stands for both.
// NZ = the number of stored z-levels (1 for D = 2, NR/2 for D = 3).
//
// Functions take their tables through template "accessor" types:
//   TT: lattice tables  c[i], he[i][m] = He_m(c_i), hw[i][m] = w_i He_m(c_i)/m!
//   TP: per-solve scalars c_omega, visc_pow, vmode, b, beta, has_force, dtgx, dtgy
//   TW: wall tables wS[2][Q], wSdev[2][Q], wA[2], wB[2] (walls normal to y);
//       wSx[2][Q], wSxdev[2][Q], wAx[2], wBx[2], wAc[4], wBc[4] (walls normal
//       to x and the corners); wspec (specular share)
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

namespace lesbgk_dev {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float minmod(float a, float b) {
  // signed smaller magnitude when a and b agree in sign, else 0; equals
  // [f_{i+1}-f_i] Psi(Theta) of Sec. 3.1 with the minmod limiter.
  // min.xorsign.abs gives min(|a|,|b|) signed by sign(a) XOR sign(b); clamping
  // at 0 keeps it only when the signs agree; a's sign is then put back
  // (three instructions instead of the four of median(a, b, 0)).
  float t;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(t) : "f"(a), "f"(b));
  t = fmaxf(t, 0.0f);
  return __uint_as_float(__float_as_uint(t) | (__float_as_uint(a) & 0x80000000u));
}

// Packed FP32 pairs (sm_100 family): one instruction, two independently
// rounded results, each bitwise equal to the scalar operation.  The pair
// travels as one 64-bit register; the subtraction has no intrinsic.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n.reg .b64 ra, rb, rr;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\n"
      "sub.rn.f32x2 rr, ra, rb;\nmov.b64 {%0, %1}, rr;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

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

// ---------------------------------------------------------------------------
// Second-order TVD advection with the minmod limiter (Sec. 3.1), per
// population, in units of the Courant number: the update is
// f -= (c dt/dh) diff with diff = F_{i+1/2} - F_{i-1/2} divided by c, where
// F_{i+1/2} = f_i + k sigma_i for c > 0 and f_{i+1} - k sigma_{i+1} for c < 0,
// k = (1 - |c| dt/dh)/2 and sigma_i = minmod(f_i - f_{i-1}, f_{i+1} - f_i).
//
// The y-sweep marches up the rows and carries a stencil per population:
//   c_y > 0: s0 = f_j - f_{j-1}, s1 = sigma_{j-1}, fc = f_j
//   c_y < 0: s0 = f_{j+1},       s1 = sigma_j,     fc = f_j
// ld holds the row entering the stencil: f_{j+1} (c_y > 0) or f_{j+2}
// (c_y < 0).  yflux returns diff at row j, sets f0 = f_j and moves the
// stencil on by one row.  The packed forms treat populations a and a+1 (the
// same ix, neighbouring iy, so c_y of one sign when the caller pairs them) as
// one f32x2 pair; each of their operations is the scalar one, term for term.
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ float yflux(bool up, int a, float (&fc)[Q], float (&s0)[Q], float (&s1)[Q],
                                       const float (&ld)[Q], float ky, float &f0) {
  f0 = fc[a];
  float diff;
  if (up) {  // c_y > 0
    const float dn = ld[a] - f0;
    const float sg = minmod(s0[a], dn);
    diff = fmaf(ky, sg - s1[a], s0[a]);
    s0[a] = dn;
    s1[a] = sg;
    fc[a] = ld[a];
  } else {  // c_y < 0
    const float d1 = s0[a] - f0;
    const float sg = minmod(d1, ld[a] - s0[a]);
    diff = fmaf(-ky, sg - s1[a], d1);
    s1[a] = sg;
    fc[a] = s0[a];
    s0[a] = ld[a];
  }
  return diff;
}

template <int Q>
__device__ __forceinline__ float2 yflux2(bool up, int a, float (&fc)[Q], float (&s0)[Q], float (&s1)[Q],
                                         const float (&ld)[Q], float2 ky, float2 &f0) {
  f0 = make_float2(fc[a], fc[a + 1]);
  const float2 l2 = make_float2(ld[a], ld[a + 1]);
  const float2 S0 = make_float2(s0[a], s0[a + 1]);
  const float2 S1 = make_float2(s1[a], s1[a + 1]);
  float2 diff, sg;
  if (up) {
    const float2 dn = sub2(l2, f0);
    sg = make_float2(minmod(S0.x, dn.x), minmod(S0.y, dn.y));
    diff = fma2(ky, sub2(sg, S1), S0);
    s0[a] = dn.x;
    s0[a + 1] = dn.y;
    fc[a] = l2.x;
    fc[a + 1] = l2.y;
  } else {
    const float2 d1 = sub2(S0, f0);
    const float2 dr = sub2(l2, S0);
    sg = make_float2(minmod(d1.x, dr.x), minmod(d1.y, dr.y));
    diff = fma2(ky, sub2(S1, sg), d1);  // (-k)(sg - s1) = k (s1 - sg), exactly
    fc[a] = S0.x;
    fc[a + 1] = S0.y;
    s0[a] = l2.x;
    s0[a + 1] = l2.y;
  }
  s1[a] = sg.x;
  s1[a + 1] = sg.y;
  return diff;
}

// x-sweep of f_i (xflux) or of a pair x2 = (f_i of population a, of a+1)
// with c_x of one sign (right: c_x > 0).  The neighbours f_{i-1}, f_{i+1}
// and the slopes of the adjacent nodes come from the adjacent lanes:
// nb.left(v) / nb.right(v) return v of the lane holding node i-1 / i+1.
template <class NB>
__device__ __forceinline__ float2 xflux2(bool right, float2 x2, float2 kx, const NB &nb) {
  const float2 dl = sub2(x2, make_float2(nb.left(x2.x), nb.left(x2.y)));  // f_i - f_{i-1}
  const float2 dr = make_float2(nb.right(dl.x), nb.right(dl.y));           // f_{i+1} - f_i
  const float2 sg = make_float2(minmod(dl.x, dr.x), minmod(dl.y, dr.y));   // sigma_i
  if (right) {
    const float2 sp = make_float2(nb.left(sg.x), nb.left(sg.y));
    return fma2(kx, sub2(sg, sp), dl);
  }
  const float2 sn = make_float2(nb.right(sg.x), nb.right(sg.y));
  return fma2(kx, sub2(sg, sn), dr);  // (-k)(sigma_{i+1} - sigma_i) = k (sigma_i - sigma_{i+1})
}

template <class NB>
__device__ __forceinline__ float xflux(bool right, float x, float kx, const NB &nb) {
  const float dl = x - nb.left(x);
  const float dr = nb.right(dl);
  const float sg = minmod(dl, dr);
  if (right) return fmaf(kx, sg - nb.left(sg), dl);
  return fmaf(-kx, nb.right(sg) - sg, dr);
}

// neighbour lanes of a warp-wide strip
struct StripLanes {
  __device__ __forceinline__ float left(float v) const { return __shfl_up_sync(kFull, v, 1); }
  __device__ __forceinline__ float right(float v) const { return __shfl_down_sync(kFull, v, 1); }
};

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
template <int NR, int KM, class TT>
__device__ __forceinline__ void hermite_moments(const float (&F)[NR * NR], float (&a)[KM + 1][KM + 1],
                                                const TT &A) {
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
template <int NR, int N, class TT>
__device__ __forceinline__ void hermite_evaluate(const float (&d)[N + 1][N + 1], float (&S)[NR * NR],
                                                 const TT &A) {
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
template <int NR, int N, class TT, class TP>
__device__ __forceinline__ void collide(const float (&F)[NR * NR], float (&S)[NR * NR], float &omw,
                                        const TT &Lt, const TP &P, float *om_out = nullptr) {
  constexpr int KM = (N - 1 > 2) ? N - 1 : 2;
  float a[KM + 1][KM + 1];
  hermite_moments<NR, KM>(F, a, Lt);
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
  if (P.vmode == 1) Tp = fast_sqrt(T);
  else if (P.vmode == 2) Tp = 1.0f;
  else Tp = exp2f(P.visc_pow * __log2f(T));
  const float om = P.c_omega * rho * Tp;  // dt/tau, tau = (Kn/Pr) T^varpi / (rho T)
  omw = 1.0f - om;
  if (om_out) *om_out = om;
  // rho (lambda - I) = (1-b) rho (T-1) I + b M,  lambda = (1-b) T I + b P/rho
  const float RLxx = fmaf(P.beta, trM, P.b * Mxx);
  const float RLxy = P.b * Mxy;
  const float RLyy = fmaf(P.beta, trM, P.b * Myy);
  float e[N + 1][N + 1];
  gaussian_coeffs<N>(rho, a[1][0], a[0][1], ux, uy, RLxx * ir, RLxy * ir, RLyy * ir, RLxx, RLxy, RLyy, e);
  float d[N + 1][N + 1];
#pragma unroll
  for (int m = 0; m <= N; ++m)
#pragma unroll
    for (int k = 0; m + k <= N; ++k) d[m][k] = om * e[m][k];
  d[0][0] = om * a[0][0];
  if (P.has_force) {
    // projected body force: coefficient m g_x a_{m-1,k} + k g_y a_{m,k-1} (a_00 = rho)
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
      for (int k = 0; m + k <= N; ++k) {
        if (m + k == 0) continue;
        float v = d[m][k];
        if (m >= 1) v = fmaf((float)m * P.dtgx, (m - 1 + k == 0) ? rho : a[m - 1][k], v);
        if (k >= 1) v = fmaf((float)k * P.dtgy, (m + k - 1 == 0) ? rho : a[m][k - 1], v);
        d[m][k] = v;
      }
  }
  hermite_evaluate<NR, N>(d, S, Lt);
}

// ---------------------------------------------------------------------------
// D = 3 set, z-even storage (NZ = NR/2 stored z-levels).  Hermite
// coefficients carry a third index l (He_l(c_z)); odd l vanish by the
// symmetry, so each node holds the in-plane arrays for l = 0, 2, 4.
// ---------------------------------------------------------------------------

// Moments b[l/2][m][k] = sum over all NR^3 velocities of df He_m(c_x) He_k(c_y)
// He_l(c_z), l even, m + k <= KM - l: per stored level the in-plane sums,
// weighted by 2 He_l(c_z) (the stored value stands for c_z and -c_z).
template <int NR, int KM, int Q, class TT>
__device__ __forceinline__ void hermite_moments3(const float (&F)[Q], float (&b)[3][KM + 1][KM + 1], const TT &A) {
  constexpr int H = NR / 2, Q2 = NR * NR, NZ = Q / Q2;
  static_assert(NZ == H, "the D = 3 set stores NR/2 z-levels");
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int m = 0; m <= KM; ++m)
#pragma unroll
      for (int k = 0; k <= KM; ++k) b[l][m][k] = 0.0f;
#pragma unroll
  for (int iz = 0; iz < NZ; ++iz) {
    float Fs[Q2];
#pragma unroll
    for (int a = 0; a < Q2; ++a) Fs[a] = F[iz * Q2 + a];
    float a2[KM + 1][KM + 1];
    hermite_moments<NR, KM>(Fs, a2, A);
#pragma unroll
    for (int l = 0; l <= 4 && l <= KM; l += 2) {
      const float hz = 2.0f * A.he[H + iz][l];
#pragma unroll
      for (int m = 0; m + l <= KM; ++m)
#pragma unroll
        for (int k = 0; m + k + l <= KM; ++k) b[l / 2][m][k] = fmaf(hz, a2[m][k], b[l / 2][m][k]);
    }
  }
}

// S_a = w_a sum_{m+k+l<=N, l even} d[l/2][m][k] He_m He_k He_l(c_z)/(m! k! l!)
// over the stored populations: per level the in-plane evaluation of
// d'_mk = sum_l d[l/2][m][k] w_z He_l(c_z)/l!.
template <int NR, int N, int Q, class TT>
__device__ __forceinline__ void hermite_evaluate3(const float (&d)[3][N + 1][N + 1], float (&S)[Q], const TT &A) {
  constexpr int H = NR / 2, Q2 = NR * NR, NZ = Q / Q2;
#pragma unroll
  for (int iz = 0; iz < NZ; ++iz) {
    float dz[N + 1][N + 1];
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
      for (int k = 0; m + k <= N; ++k) {
        float v = d[0][m][k] * A.hw[H + iz][0];
        if (m + k + 2 <= N) v = fmaf(d[1][m][k], A.hw[H + iz][2], v);
        if (m + k + 4 <= N) v = fmaf(d[2][m][k], A.hw[H + iz][4], v);
        dz[m][k] = v;
      }
    float Ss[Q2];
    hermite_evaluate<NR, N>(dz, Ss, A);
#pragma unroll
    for (int a = 0; a < Q2; ++a) S[iz * Q2 + a] = Ss[a];
  }
}

// In-plane Gaussian coefficients e (from gaussian_coeffs) times the z-factor
// E[He_l(Z)], Z ~ N(0, 1 + Lzz): 1, Lzz, 3 Lzz^2 for l = 0, 2, 4 (lambda has no
// xz or yz part and u_z = 0, so the generating function factorises).
template <int N>
__device__ __forceinline__ void z_factor(const float (&e)[N + 1][N + 1], float Lzz, float scale,
                                         float (&d)[3][N + 1][N + 1]) {
  const float z2 = Lzz * scale, z4 = 3.0f * Lzz * Lzz * scale;
#pragma unroll
  for (int m = 0; m <= N; ++m)
#pragma unroll
    for (int k = 0; m + k <= N; ++k) {
      d[0][m][k] = scale * e[m][k];
      d[1][m][k] = (m + k + 2 <= N) ? z2 * e[m][k] : 0.0f;
      d[2][m][k] = (m + k + 4 <= N) ? z4 * e[m][k] : 0.0f;
    }
}

// Coefficients d[l/2][m][k] of the D = 3 collision + force source from the
// moments b of hermite_moments3 (T = tr P/(3 rho), lambda 3x3 with
// lambda_zz = (1-b) T + b P_zz/rho), and omw = 1 - dt/tau.
template <int NR, int N, int KM, class TP>
__device__ __forceinline__ void es_coefficients3(const float (&b)[3][KM + 1][KM + 1], float (&d)[3][N + 1][N + 1],
                                                 float &omw, const TP &P, float *om_out = nullptr) {
  const float rho = 1.0f + b[0][0][0];
  const float ir = fast_rcp(rho);
  const float ux = b[0][1][0] * ir, uy = b[0][0][1] * ir;
  const float Mxx = fmaf(-b[0][1][0], ux, b[0][2][0]);
  const float Mxy = fmaf(-b[0][1][0], uy, b[0][1][1]);
  const float Myy = fmaf(-b[0][0][1], uy, b[0][0][2]);
  const float Mzz = b[1][0][0];  // sum df He_2(c_z); u_z = 0
  const float trM = Mxx + Myy + Mzz;
  const float T = fmaf((1.0f / 3.0f) * trM, ir, 1.0f);  // T = tr P / (D rho), D = 3
  float Tp;
  if (P.vmode == 1) Tp = fast_sqrt(T);
  else if (P.vmode == 2) Tp = 1.0f;
  else Tp = exp2f(P.visc_pow * __log2f(T));
  const float om = P.c_omega * rho * Tp;
  omw = 1.0f - om;
  if (om_out) *om_out = om;
  // rho (lambda - I) = (1-b) rho (T-1) I + b M, with beta = (1-b)/3
  const float RLxx = fmaf(P.beta, trM, P.b * Mxx);
  const float RLxy = P.b * Mxy;
  const float RLyy = fmaf(P.beta, trM, P.b * Myy);
  const float RLzz = fmaf(P.beta, trM, P.b * Mzz);
  float e[N + 1][N + 1];
  gaussian_coeffs<N>(rho, b[0][1][0], b[0][0][1], ux, uy, RLxx * ir, RLxy * ir, RLyy * ir, RLxx, RLxy, RLyy, e);
  z_factor<N>(e, RLzz * ir, om, d);
  d[0][0][0] = om * b[0][0][0];
  if (P.has_force) {
    // m g_x a_{m-1,k,l} + k g_y a_{m,k-1,l} (a_000 = rho; g_z = 0)
#pragma unroll
    for (int l = 0; l <= 2 && l <= N; l += 2)
#pragma unroll
      for (int m = 0; m + l <= N; ++m)
#pragma unroll
        for (int k = 0; m + k + l <= N; ++k) {
          if (m + k == 0) continue;
          float v = d[l / 2][m][k];
          if (m >= 1) v = fmaf((float)m * P.dtgx, (m - 1 + k + l == 0) ? rho : b[l / 2][m - 1][k], v);
          if (k >= 1) v = fmaf((float)k * P.dtgy, (m + k - 1 + l == 0) ? rho : b[l / 2][m][k - 1], v);
          d[l / 2][m][k] = v;
        }
  }
}

// The collision + force source of collide() for the D = 3 set, all stored
// levels in one thread.
template <int NR, int N, int Q, class TT, class TP>
__device__ __forceinline__ void collide3(const float (&F)[Q], float (&S)[Q], float &omw, const TT &Lt,
                                         const TP &P, float *om_out = nullptr) {
  constexpr int KM = (N - 1 > 2) ? N - 1 : 2;
  float b[3][KM + 1][KM + 1];
  hermite_moments3<NR, KM>(F, b, Lt);
  float d[3][N + 1][N + 1];
  es_coefficients3<NR, N, KM>(b, d, omw, P, om_out);
  hermite_evaluate3<NR, N>(d, S, Lt);
}

// One node's source for either kind of set: collide() for D = 2, collide3() for D = 3.
template <int NR, int N, int Q, class TT, class TP>
__device__ __forceinline__ void collide_any(const float (&F)[Q], float (&S)[Q], float &omw, const TT &Lt,
                                            const TP &P) {
  if constexpr (Q == NR * NR) collide<NR, N>(F, S, omw, Lt, P);
  else collide3<NR, N>(F, S, omw, Lt, P);
}

// The same, returning dt/tau itself (om) rather than 1 - dt/tau: the
// compensated update adds -om f to the remainder, where 1 - (1 - om) would
// carry the rounding of 1 - om (2^-24 absolute, a 1e-4 relative error of om
// at dt/tau ~ 1e-3).
template <int NR, int N, int Q, class TT, class TP>
__device__ __forceinline__ void collide_om(const float (&F)[Q], float (&S)[Q], float &om, const TT &Lt,
                                           const TP &P) {
  float omw;
  if constexpr (Q == NR * NR) collide<NR, N>(F, S, omw, Lt, P, &om);
  else collide3<NR, N>(F, S, omw, Lt, P, &om);
}

// ---------------------------------------------------------------------------
// Moments of Eq. (mac) of one node from its deviations F = f - w, written to
// out[k * cells + c] (k = rho, u_x, u_y, T, sigma_xx, sigma_xy, sigma_yy, q_x,
// q_y) when out is set; returns in d the node's deviations of the conserved
// sums sum_a df_a {1, c_x, c_y, c^2}: with the Hermite moments m_pql =
// sum df He_p(c_x) He_q(c_y) He_l(c_z) these are m000, m100, m010 and
// m200 + m020 (+ m002) + D m000.  D = 2 for the 2D sets; D = 3 (Q = NR^3/2
// stored, z-even) adds the c_z terms: T = tr P/(3 rho), sigma trace-free in
// 3D (sigma_zz = -sigma_xx - sigma_yy is not written), q with c_z^2 in C^2.
// ---------------------------------------------------------------------------
template <int NR, int Q, class TT>
__device__ __forceinline__ void node_moments(const float (&F)[Q], float *__restrict__ out, long long cells,
                                             long long c, const TT &A, float (&d)[4]) {
  constexpr bool D3 = Q != NR * NR;
  float m[4][4];
  float mzz = 0.0f, mzx = 0.0f, mzy = 0.0f;  // m002, m102, m012 (D = 3)
  if constexpr (!D3) {
    hermite_moments<NR, 3>(F, m, A);
  } else {
    float b[3][4][4];
    hermite_moments3<NR, 3>(F, b, A);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; p + q < 4; ++q) m[p][q] = b[0][p][q];
    mzz = b[1][0][0];
    mzx = b[1][1][0];
    mzy = b[1][0][1];
  }
  const float rho = 1.0f + m[0][0];
  const float ir = __frcp_rn(rho);
  const float ux = m[1][0] * ir, uy = m[0][1] * ir;
  const float Mxx = fmaf(-m[1][0], ux, m[2][0]);
  const float Mxy = fmaf(-m[1][0], uy, m[1][1]);
  const float Myy = fmaf(-m[0][1], uy, m[0][2]);
  const float trM = Mxx + Myy + mzz;  // M_zz = m002 (u_z = 0)
  const float T = fmaf((D3 ? 1.0f / 3.0f : 0.5f) * trM, ir, 1.0f);
  const float u2 = ux * ux + uy * uy;
  // sum f C_i C^2 = sum df c_i (c^2 - D - 2) - 2 M_ij u_j - u_i tr M - rho u_i u^2
  const float hx = m[3][0] + m[1][2] + mzx, hy = m[0][3] + m[2][1] + mzy;
  const float qx = 0.5f * (hx - 2.0f * (Mxx * ux + Mxy * uy) - ux * trM - rho * ux * u2);
  const float qy = 0.5f * (hy - 2.0f * (Mxy * ux + Myy * uy) - uy * trM - rho * uy * u2);
  if (out) {
    out[c] = rho;
    out[cells + c] = ux;
    out[2 * cells + c] = uy;
    out[3 * cells + c] = T;
    if constexpr (!D3) {
      out[4 * cells + c] = 0.5f * (Mxx - Myy);
      out[6 * cells + c] = 0.5f * (Myy - Mxx);
    } else {
      out[4 * cells + c] = fmaf(-1.0f / 3.0f, trM, Mxx);
      out[6 * cells + c] = fmaf(-1.0f / 3.0f, trM, Myy);
    }
    out[5 * cells + c] = Mxy;
    out[7 * cells + c] = qx;
    out[8 * cells + c] = qy;
  }
  d[0] = m[0][0];
  d[1] = m[1][0];
  d[2] = m[0][1];
  d[3] = fmaf(D3 ? 3.0f : 2.0f, m[0][0], m[2][0] + m[0][2] + mzz);
}

// Wall rule of Sec. 3.2 on one node's updated deviations: rho_W from the
// incoming half (zero net normal mass flux through the wall), outgoing half =
// rho_W S_a(T_w, u_w), the fully diffuse wall; with SPEC (Maxwell model,
// accommodation gamma = 1 - W.wspec) the outgoing half is instead
// gamma rho_W S_a + (1 - gamma) f_a', a' the incoming mirror image (c_y -> -c_y).
// side 0: bottom (outgoing c_y > 0), side 1: top (outgoing c_y < 0).  The
// S tables are built on the host in FP64 for the wall temperature of the time
// the launch writes (a varying one for the heated walls of Sec. 4.2).
template <int NR, bool SPEC, int Q, class TT, class TW>
__device__ __forceinline__ void wall_fix(float (&O)[Q], int side, const TT &T, const TW &W) {
  constexpr int H = NR / 2;
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int iy = a % NR;
    const bool incoming = side == 0 ? (iy < H) : (iy >= H);
    if (incoming) s = fmaf(fabsf(T.c[iy]), O[a], s);
  }
  const float rw1 = (s - W.wA[side]) * W.wB[side];  // rho_W - 1
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int iy = a % NR;
    const bool outgoing = side == 0 ? (iy >= H) : (iy < H);
    if (outgoing) {
      const float diffuse = fmaf(rw1, W.wS[side][a], W.wSdev[side][a]);
      if constexpr (SPEC) O[a] = fmaf(W.wspec, O[a + (NR - 1 - 2 * iy)] - diffuse, diffuse);
      else O[a] = diffuse;
    }
  }
}

// Diffuse wall at rest normal to x (columns i = 0 and nx-1; side 0 = left,
// inward normal +x): the rule of wall_fix with c_x in place of c_y, tables
// wSx, wSxdev, wAx, wBx of S(T_wx, u = 0).
template <int NR, int Q, class TT, class TW>
__device__ __forceinline__ void wall_fix_x(float (&O)[Q], int side, const TT &T, const TW &W) {
  constexpr int H = NR / 2;
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ix = (a / NR) % NR;
    const bool incoming = side == 0 ? (ix < H) : (ix >= H);
    if (incoming) s = fmaf(fabsf(T.c[ix]), O[a], s);
  }
  const float rw1 = (s - W.wAx[side]) * W.wBx[side];  // rho_W - 1
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ix = (a / NR) % NR;
    const bool outgoing = side == 0 ? (ix >= H) : (ix < H);
    if (outgoing) O[a] = fmaf(rw1, W.wSx[side][a], W.wSxdev[side][a]);
  }
}

// Corner node on the x-wall xside and the y-wall yside (a reading: the paper
// has no corners).  Kept: the populations arriving towards both walls
// (c.n_x < 0 and c.n_y < 0, inward normals); all others are re-emitted as
// rho_W S(T_wx, u = 0) of the side wall, with rho_W from zero net mass flux
// along n = n_x + n_y: rho_W - 1 = (sum_kept |c.n| df - wAc) wBc.
template <int NR, int Q, class TT, class TW>
__device__ __forceinline__ void wall_corner(float (&O)[Q], int xside, int yside, const TT &T, const TW &W) {
  constexpr int H = NR / 2;
  const int k = yside * 2 + xside;
  const float nx = xside == 0 ? 1.0f : -1.0f, ny = yside == 0 ? 1.0f : -1.0f;
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ix = (a / NR) % NR, iy = a % NR;
    const bool kept = (xside == 0 ? ix < H : ix >= H) && (yside == 0 ? iy < H : iy >= H);
    if (kept) s = fmaf(fabsf(fmaf(T.c[ix], nx, T.c[iy] * ny)), O[a], s);
  }
  const float rw1 = (s - W.wAc[k]) * W.wBc[k];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ix = (a / NR) % NR, iy = a % NR;
    const bool kept = (xside == 0 ? ix < H : ix >= H) && (yside == 0 ? iy < H : iy >= H);
    if (!kept) O[a] = fmaf(rw1, W.wSx[xside][a], W.wSxdev[xside][a]);
  }
}

// The walls of one node.  WM = 0: y-walls (fully diffuse) if any; 1: y-walls
// with a specular share; 2: walls in x as well (cavity; y-walls diffuse).
template <int NR, int WM, int Q, class TA>
__device__ __forceinline__ void apply_walls_node(float (&O)[Q], int i, int j, const TA &A) {
  const bool yw = A.walls && (j == 0 || j == A.ny - 1);
  if constexpr (WM == 2) {
    const bool xw = i == 0 || i == A.nx - 1;
    if (xw && yw) wall_corner<NR>(O, i == 0 ? 0 : 1, j == 0 ? 0 : 1, A, A);
    else if (xw) wall_fix_x<NR>(O, i == 0 ? 0 : 1, A, A);
    else if (yw) wall_fix<NR, false>(O, j == 0 ? 0 : 1, A, A);
  } else {
    if (yw) wall_fix<NR, WM == 1>(O, j == 0 ? 0 : 1, A, A);
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
// Storage of one population: FP32 holds df itself; the 16-bit types hold the
// relative deviation s = df / w_a (rounded to nearest), which gives every
// population the same relative precision whatever its weight.
template <class S>
struct Store;
template <>
struct Store<float> {
  static constexpr bool kScaled = false;
  __device__ static float get(float v, float) { return v; }
  __device__ static float put(float x, float) { return x; }
};
template <>
struct Store<__half> {
  static constexpr bool kScaled = true;
  // a rounded product (__fmul_rn is never contracted into the subtraction
  // that follows): a loaded value is then one number whether a segment's
  // prologue or the ring brought it, so results do not depend on the launch shape
  __device__ static float get(__half v, float w) { return __fmul_rn(__half2float(v), w); }
  __device__ static __half put(float x, float iw) { return __float2half_rn(x * iw); }
  // two values packed (x0 low, x1 high), stochastically rounded by the
  // hardware (cvt.rs): rbits supplies the random bits of both
  __device__ static unsigned put_sr2(float x0, float x1, unsigned rbits) {
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(x1), "f"(x0), "r"(rbits));
    return d;
  }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr bool kScaled = true;
  __device__ static float get(__nv_bfloat16 v, float w) { return __fmul_rn(__bfloat162float(v), w); }
  __device__ static __nv_bfloat16 put(float x, float iw) { return __float2bfloat16_rn(x * iw); }
  __device__ static unsigned put_sr2(float x0, float x1, unsigned rbits) {
    unsigned d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(x1), "f"(x0), "r"(rbits));
    return d;
  }
};

// 32-bit integer mixer (the "lowbias32" finaliser published by C. Wellons):
// a bijection with good avalanche, used as a counter-based random generator.
__device__ __forceinline__ unsigned mix32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__host__ __device__ constexpr int pick_vector(int half, int bytes) {
  return (half % 8 == 0 && 8 * bytes <= 16) ? 8 : (half % 4 == 0 && 4 * bytes <= 16) ? 4 : (half % 2 == 0) ? 2 : 1;
}

template <int NR, class S = float, int NZ = 1>
struct Layout {
  static constexpr int Q = NZ * NR * NR;
  static constexpr int H = NR / 2;
  static constexpr int HALF = Q / 2;
  static constexpr int V = pick_vector(HALF, (int)sizeof(S));  // populations per vector
  static constexpr int G = Q / V;                               // vectors (groups) per node
  static constexpr int VB = V * (int)sizeof(S);                 // bytes per vector
  // slot s -> population alpha = iz*NR^2 + ix*NR + iy: the first half of the
  // slots holds c_y < 0 (iy < H), the second c_y > 0, each in (iz, ix, iy) order
  __host__ __device__ static constexpr int alpha(int s) {
    return (s % HALF) / (NR * H) * NR * NR + (s % HALF) % (NR * H) / H * NR + ((s / HALF) ? H : 0) +
           (s % HALF) % H;
  }
};

template <int NR, class S, int Q>
using LayoutQ = Layout<NR, S, Q / (NR * NR)>;

template <int V>
struct VecT;
template <>
struct VecT<2> { using T = float2; };
template <>
struct VecT<4> { using T = float4; };

template <int B>
struct Raw;
template <>
struct Raw<16> { using T = uint4; };
template <>
struct Raw<8> { using T = uint2; };
template <>
struct Raw<4> { using T = unsigned; };

// Load group g of one node (p points at the node's row, group 0) into F[alpha].
template <int NR, int Q>
__device__ __forceinline__ void ld_group(const float *p, long long gstride, int g, float (&F)[Q]) {
  using L = LayoutQ<NR, float, Q>;
  using T = typename VecT<L::V>::T;
  const T v = __ldg(reinterpret_cast<const T *>(p + g * gstride));
  const float *e = reinterpret_cast<const float *>(&v);
#pragma unroll
  for (int k = 0; k < L::V; ++k) F[L::alpha(g * L::V + k)] = e[k];
}

template <int NR, int Q>
__device__ __forceinline__ void st_group(float *p, long long gstride, int g, const float (&F)[Q]) {
  using L = LayoutQ<NR, float, Q>;
  using T = typename VecT<L::V>::T;
  T v;
  float *e = reinterpret_cast<float *>(&v);
#pragma unroll
  for (int k = 0; k < L::V; ++k) e[k] = F[L::alpha(g * L::V + k)];
  *reinterpret_cast<T *>(p + g * gstride) = v;
}

// The same for any storage type S: one raw vector per group, converted to
// FP32 deviations (TT provides wq[a] = w_a and iwq[a] = 1/w_a).
template <int NR, class S, int Q, class TT>
__device__ __forceinline__ void unpack_group(const typename Raw<LayoutQ<NR, S, Q>::VB>::T &raw, int g,
                                             float (&F)[Q], const TT &Tt) {
  using L = LayoutQ<NR, S, Q>;
  const S *e = reinterpret_cast<const S *>(&raw);
#pragma unroll
  for (int k = 0; k < L::V; ++k) {
    const int a = L::alpha(g * L::V + k);
    F[a] = Store<S>::get(e[k], Store<S>::kScaled ? Tt.wq[a] : 1.0f);
  }
}

template <int NR, class S, int Q, class TT>
__device__ __forceinline__ void ld_group_s(const S *p, long long gstride, int g, float (&F)[Q], const TT &Tt) {
  using R = typename Raw<LayoutQ<NR, S, Q>::VB>::T;
  const R raw = __ldg(reinterpret_cast<const R *>(p + g * gstride));
  unpack_group<NR, S>(raw, g, F, Tt);
}

template <int NR, class S, int Q, class TT>
__device__ __forceinline__ void st_group_s(S *p, long long gstride, int g, const float (&F)[Q],
                                           const TT &Tt) {
  using L = LayoutQ<NR, S, Q>;
  using R = typename Raw<L::VB>::T;
  R raw;
  S *e = reinterpret_cast<S *>(&raw);
#pragma unroll
  for (int k = 0; k < L::V; ++k) {
    const int a = L::alpha(g * L::V + k);
    e[k] = Store<S>::put(F[a], Store<S>::kScaled ? Tt.iwq[a] : 1.0f);
  }
  *reinterpret_cast<R *>(p + g * gstride) = raw;
}

// Store with stochastic rounding for the 16-bit types (FP32 stores as is):
// pairs of values go through the hardware's stochastic rounding (cvt.rs,
// unbiased for both halves), fed one 32-bit random word per pair: the first
// is mix32(key ^ g * 0x9e3779b9), each next one a multiply-add of the last
// (each word is a bijection of a uniform seed, hence uniform).  Results depend
// only on the key and the population, never on the launch shape.
template <int NR, class S, int Q, class TT>
__device__ __forceinline__ void st_group_sr(S *p, long long gstride, int g, const float (&F)[Q],
                                            const TT &Tt, unsigned key) {
  if constexpr (!Store<S>::kScaled) {
    st_group_s<NR, S>(p, gstride, g, F, Tt);
  } else {
    using L = LayoutQ<NR, S, Q>;
    static_assert(L::V % 2 == 0, "16-bit groups hold pairs");
    using R = typename Raw<L::VB>::T;
    R raw;
    unsigned *w = reinterpret_cast<unsigned *>(&raw);
    unsigned bits = mix32(key ^ ((unsigned)g * 0x9e3779b9u));
#pragma unroll
    for (int k = 0; k < L::V; k += 2) {
      const int a0 = L::alpha(g * L::V + k), a1 = L::alpha(g * L::V + k + 1);
      w[k / 2] = Store<S>::put_sr2(F[a0] * Tt.iwq[a0], F[a1] * Tt.iwq[a1], bits);
      bits = bits * 0x9e3779b5u + 0x7f4a7c15u;
    }
    *reinterpret_cast<R *>(p + g * gstride) = raw;
  }
}

// ---------------------------------------------------------------------------
// Compensated FP32 storage (tag Comp): each stored deviation is hi + lo, hi an
// FP32 value in the grouped layout above and lo its rounding remainder, held
// in FP16 as lo * 2^24 / w_a (TT's wq[a] = w_a 2^-24 converts back) in a
// second plane of the same 16-byte vectors right after the hi plane (its
// groups hold twice as many values, so a row of either plane is nx 16-byte
// vectors per group and one byte offset serves both).  Built for the sets
// whose hi vectors hold 4 values (D2Q16, D3Q64).
// ---------------------------------------------------------------------------
struct Comp {};

template <class S>
struct Elem { using T = S; };
template <>
struct Elem<Comp> { using T = float; };

template <class S>
constexpr bool kIsComp = false;
template <>
constexpr bool kIsComp<Comp> = true;

// The lo plane of the populations whose hi plane starts at f (or at a row of
// it: the byte offset is the same in both planes); plane = nx ny of the grid.
template <int Q>
__device__ __forceinline__ const __half *lo_plane(const float *f, long long plane) {
  return reinterpret_cast<const __half *>(reinterpret_cast<const char *>(f) + (size_t)Q * plane * sizeof(float));
}
template <int Q>
__device__ __forceinline__ __half *lo_plane(float *f, long long plane) {
  return reinterpret_cast<__half *>(reinterpret_cast<char *>(f) + (size_t)Q * plane * sizeof(float));
}

// All stored values of node c as FP32 deviations (for Comp, hi + lo rounded
// once); f at the grid's (or a row's) start, plane = nx ny.
template <int NR, class S, int NZ, class TT>
__device__ __forceinline__ void ld_node(const typename Elem<S>::T *f, long long c, long long plane,
                                        float (&F)[NZ * NR * NR], const TT &Tt) {
  if constexpr (kIsComp<S>) {
    using LH = Layout<NR, float, NZ>;
    using LL = Layout<NR, __half, NZ>;
    static_assert(LL::V == 2 * LH::V, "hi and lo vectors of 16 bytes");
#pragma unroll
    for (int g = 0; g < LH::G; ++g) ld_group<NR>(f + c * LH::V, (long long)LH::V * plane, g, F);
    const __half *lo = lo_plane<LH::Q>(f, plane) + c * LL::V;
#pragma unroll
    for (int g = 0; g < LL::G; ++g) {
      const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(lo + (long long)g * LL::V * plane));
      const __half *e = reinterpret_cast<const __half *>(&raw);
#pragma unroll
      for (int k = 0; k < LL::V; ++k) {
        const int a = LL::alpha(g * LL::V + k);
        F[a] = fmaf(__half2float(e[k]), Tt.wq[a], F[a]);
      }
    }
  } else if constexpr (std::is_same<S, float>::value) {  // (no scale tables needed)
    using L = Layout<NR, float, NZ>;
#pragma unroll
    for (int g = 0; g < L::G; ++g) ld_group<NR>(f + c * L::V, (long long)L::V * plane, g, F);
  } else {
    using L = Layout<NR, S, NZ>;
#pragma unroll
    for (int g = 0; g < L::G; ++g) ld_group_s<NR, S>(f + c * L::V, (long long)L::V * plane, g, F, Tt);
  }
}

// Store node c's values F (round to nearest; for Comp, hi = F and lo = 0).
template <int NR, class S, int NZ, class TT>
__device__ __forceinline__ void st_node(typename Elem<S>::T *f, long long c, long long plane,
                                        const float (&F)[NZ * NR * NR], const TT &Tt) {
  if constexpr (kIsComp<S>) {
    using LH = Layout<NR, float, NZ>;
    using LL = Layout<NR, __half, NZ>;
#pragma unroll
    for (int g = 0; g < LH::G; ++g) st_group<NR>(f + c * LH::V, (long long)LH::V * plane, g, F);
    __half *lo = lo_plane<LH::Q>(f, plane) + c * LL::V;
#pragma unroll
    for (int g = 0; g < LL::G; ++g)
      *reinterpret_cast<uint4 *>(lo + (long long)g * LL::V * plane) = make_uint4(0u, 0u, 0u, 0u);
  } else if constexpr (std::is_same<S, float>::value) {
    using L = Layout<NR, float, NZ>;
#pragma unroll
    for (int g = 0; g < L::G; ++g) st_group<NR>(f + c * L::V, (long long)L::V * plane, g, F);
  } else {
    using L = Layout<NR, S, NZ>;
#pragma unroll
    for (int g = 0; g < L::G; ++g) st_group_s<NR, S>(f + c * L::V, (long long)L::V * plane, g, F, Tt);
  }
}

// Asynchronous global->shared copy of B bytes (cp.async; 16-byte copies bypass L1).
template <int B>
__device__ __forceinline__ void cp_async_raw(void *smem_dst, const void *gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  if constexpr (B == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else if constexpr (B == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
  }
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


}  // namespace lesbgk_dev
