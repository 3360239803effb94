// pflb_model.cuh -- per-cell arithmetic of the conservative Allen-Cahn
// phase-field lattice Boltzmann step (D3Q19), device side.
//
// Sources (arXiv 2512.01032):
//   Eq. 1     h_i relaxation with tau_phi = M/T + 1/2
//   Eqs. 2-3  h equilibrium phi*Gamma_i + theta*w_i*(c_i . n), Gamma_i
//   Eq. 4     local mobility correction delta-theta
//   Eqs. 5-6  hydrodynamic equilibrium and force K_i
//   Eq. 7     chemical potential
//   Eq. 8     tau_mix; optimised F(phi) of Sec. III A
//   Eqs. 9-11 filtered collision (Hermite second-order filter)
//   text after Eq. 11: P and rho*u recovery
//   Eq. 13    central-difference gradient and Laplacian
//   Eqs. 12-15 wettability ghosts; Sec. III A blend and free-slip band
//
// Populations: h = phase field, g = hydrodynamic (the paper's g-bar).
#pragma once
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace pflb {

constexpr int Q = 19;

// D3Q19: rest, +-x, +-y, +-z, then twelve edge directions in opposite pairs.
__host__ __device__ constexpr int cx_of(int i) {
  constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[i];
}
__host__ __device__ constexpr int cy_of(int i) {
  constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz_of(int i) {
  constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[i];
}
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double w_of(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// Direction index of a velocity vector (-1 if not in the set).
__host__ __device__ constexpr int dir_of(int x, int y, int z) {
  for (int i = 0; i < Q; ++i)
    if (cx_of(i) == x && cy_of(i) == y && cz_of(i) == z) return i;
  return -1;
}

// Specular-reflection data of edge link i (two nonzero components on axes
// a < b).  fa/fb: face directions along c_ia e_a and c_ib e_b.  If the face
// neighbour fa is solid and fb fluid, the wall lies across axis a: the
// tangential partner is x + e(fb) and the reflected direction is ra.
// Symmetrically for fb solid / fa fluid with rb.
struct EdgeInfo { int fa, fb, ra, rb; };
__host__ __device__ constexpr EdgeInfo edge_info(int i) {
  int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
  int a = -1, b = -1;
  for (int k = 0; k < 3; ++k)
    if (c[k] != 0) { if (a < 0) a = k; else b = k; }
  if (b < 0) return EdgeInfo{-1, -1, -1, -1};
  int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
  ea[a] = c[a];
  eb[b] = c[b];
  int fa = dir_of(ea[0], ea[1], ea[2]);
  int fb = dir_of(eb[0], eb[1], eb[2]);
  int r1[3] = {c[0], c[1], c[2]};
  r1[a] = -r1[a];
  int r2[3] = {c[0], c[1], c[2]};
  r2[b] = -r2[b];
  return EdgeInfo{fa, fb, dir_of(r1[0], r1[1], r1[2]), dir_of(r2[0], r2[1], r2[2])};
}

// Diagnostic accumulator slots (double, device).
// Slots before D_UMAX are sums; D_UMAX, D_FRONT and D_REAR are maxima of
// non-negative values (the interface crossings are stored shifted so that
// 0 means "none": x + 1 for the front, nx - x for the rear).
enum {
  D_MASS = 0, D_NHEAVY, D_PH, D_NPH, D_PL, D_NPL, D_REGION, D_CLN, D_CLX, D_CLY, D_CLZ,
  D_CLXX, D_CLYY, D_CLZZ, D_KIN, D_NONFINITE, D_UMAX, D_FRONT, D_REAR, D_COUNT
};

// Cell flags.
constexpr uint8_t F_SOLID = 1;
constexpr uint8_t F_WALL = 2;
constexpr uint8_t F_BC = 4;  // fluid cell of an open x boundary plane (reading R22)
constexpr uint8_t F_NEAR = 8;  // fluid cell whose phi a wall node reads (the node or a neighbour)

// Model parameters in the compute precision R (derived constants included).
template <class R>
struct Model {
  R sigma, W, M, rho_L, rho_dif;
  R tau_H, tau_L;
  R Fx, Fy, Fz;
  R gamma, phi_M, phi_m, inv_D, eps, blend, band_lo, band_hi, F_tilde, inv_F_width;
  R inv_tau_phi;       // 1 / (M/T + 1/2)
  R theta_coef;        // M / (T W)
  R mu_a, mu_b;        // 48 sigma / W, 3 sigma W / 2
  R two_over_W;        // 2 / W
  int F_mode, mobility_corr, free_slip;
};

// ------------------------------------------------------------ storage
// Population storage types: the collision always runs in R.
template <class S> struct Store;
template <> struct Store<double> {
  static __device__ __forceinline__ double ld(const double *p) { return *p; }
  static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Store<float> {
  static __device__ __forceinline__ float ld(const float *p) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
// Loads of data that no thread writes during the launch (the h buffer being
// read): may go through the read-only data path.  In-place arrays (g) must
// not, since the compiler may then move such loads past aliasing stores.
template <class S> __device__ __forceinline__ S ld_ro(const S *p) { return __ldg(p); }

// ------------------------------------------------------------ codecs
// Populations are stored in S and computed in R.  FP64 and FP32 store the
// value itself.  The two 16-bit formats ("narrow") make the h set
// mass-conserving: the rest population never moves, so each cell adds the
// rounding error of the 18 moving h populations it writes to its own rest
// population, which is kept as a pair of 16-bit values (a high part and the
// remainder, about 22 significant bits at FP16, 16 at BF16).  The sum of all
// stored h then equals the sum of the computed ones up to FP32 rounding, so
// total phi does not drift.
// FP16 ("scaled") stores each population divided by the lattice weight of
// its direction: values of order phi in [0, 1] for h and of order P/T for g
// (the rest value of g being w_i P / T), which keeps them above FP16's
// normal range limit of 6.1e-5 down to phi or P/T of that size.  BF16 has
// FP32's exponent range, so its relative spacing is the same at any
// magnitude and it stores the value itself: dividing by w_i would change no
// rounding, only add a multiply to every encode and decode.  i is a
// compile-time constant at every call, so the scale folds into one multiply.
template <class S> struct Codec {
  template <class R> static __device__ __forceinline__ R to(S v) { return (R)v; }
  template <class R> static __device__ __forceinline__ S from(R v) { return (S)v; }
  static constexpr bool scaled = false, narrow = false;
};
template <> struct Codec<__half> {
  template <class R> static __device__ __forceinline__ R to(__half v) { return (R)__half2float(v); }
  template <class R> static __device__ __forceinline__ __half from(R v) {
    return __float2half_rn((float)v);
  }
  static constexpr bool scaled = true, narrow = true;
};
template <> struct Codec<__nv_bfloat16> {
  template <class R> static __device__ __forceinline__ R to(__nv_bfloat16 v) {
    return (R)__bfloat162float(v);
  }
  template <class R> static __device__ __forceinline__ __nv_bfloat16 from(R v) {
    return __float2bfloat16_rn((float)v);
  }
  static constexpr bool scaled = false, narrow = true;
};

// Number of h slots per cell: 19, plus the remainder of the rest population
// for the 16-bit formats (slot 19).
template <class S> __host__ __device__ constexpr int h_slots() { return Codec<S>::narrow ? Q + 1 : Q; }

__host__ __device__ constexpr double inv_w_of(int i) { return i == 0 ? 3.0 : (i <= 6 ? 18.0 : 36.0); }

template <class S, class R>
__device__ __forceinline__ R dec_pop(S v, int i) {
  if constexpr (Codec<S>::scaled)
    return Codec<S>::template to<R>(v) * R(w_of(i));
  else
    return Codec<S>::template to<R>(v);
}
template <class S, class R>
__device__ __forceinline__ S enc_pop(R v, int i) {
  if constexpr (Codec<S>::scaled)
    return Codec<S>::template from<R>(v * R(inv_w_of(i)));
  else
    return Codec<S>::template from<R>(v);
}
// Two populations encoded together: the 16-bit formats round both with one
// packed conversion (round to nearest even, as the single conversions).
template <class S, class R>
__device__ __forceinline__ void enc_pop2(R a, int i, R b, int j, S &ea, S &eb) {
  if constexpr (Codec<S>::narrow && sizeof(S) == 2 && !Codec<S>::scaled) {
    const __nv_bfloat162 p = __floats2bfloat162_rn((float)a, (float)b);
    ea = __low2bfloat16(p);
    eb = __high2bfloat16(p);
  } else if constexpr (Codec<S>::narrow) {
    const __half2 p =
        __floats2half2_rn((float)(a * R(inv_w_of(i))), (float)(b * R(inv_w_of(j))));
    ea = __low2half(p);
    eb = __high2half(p);
  } else {
    ea = (S)a;
    eb = (S)b;
  }
}
// The 19 g of a cell encoded for storage (pairs share a conversion).
template <class S, class R>
__device__ __forceinline__ void enc_g_cell(const R g[Q], S ge[Q]) {
  ge[0] = enc_pop<S, R>(g[0], 0);
#pragma unroll
  for (int i = 1; i < Q; i += 2) enc_pop2<S, R>(g[i], i, g[i + 1], i + 1, ge[i], ge[i + 1]);
}
template <class S, class R> __device__ __forceinline__ R ld_g(const S *p, int i) {
  return dec_pop<S, R>(*p, i);
}
template <class S, class R> __device__ __forceinline__ void st_g(S *p, int i, R v) {
  *p = enc_pop<S, R>(v, i);
}
// Loads all 19 h of cell c from direction bases hb (read-only path); the
// rest population of the 16-bit formats is high part + remainder.
template <class S, class R>
__device__ __forceinline__ void ld_h_cell(const S *const *hb, int c, R h[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) h[i] = dec_pop<S, R>(ld_ro<S>(hb[i] + c), i);
  if constexpr (Codec<S>::narrow) h[0] += dec_pop<S, R>(ld_ro<S>(hb[Q] + c), 0);
}
// Encodes the 19 post-collision h of a cell; for the 16-bit formats the
// rounding error of directions 1..18 is moved into the rest population,
// whose high part goes to enc[0] and remainder to *rest_lo.
template <class S, class R>
__device__ __forceinline__ void enc_h_cell(const R h[Q], S enc[Q], S *rest_lo) {
  if constexpr (Codec<S>::narrow) {
    R err = R(0);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      enc_pop2<S, R>(h[i], i, h[i + 1], i + 1, enc[i], enc[i + 1]);
      err += (dec_pop<S, R>(enc[i], i) - h[i]) + (dec_pop<S, R>(enc[i + 1], i + 1) - h[i + 1]);
    }
    const R h0 = h[0] - err;
    enc[0] = enc_pop<S, R>(h0, 0);
    *rest_lo = enc_pop<S, R>(h0 - dec_pop<S, R>(enc[0], 0), 0);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) enc[i] = (S)h[i];
    (void)rest_lo;
  }
}

// Square root, reciprocal, quotient and tanh: IEEE versions in FP64 (the
// parity path); in FP32, short hardware-approximation forms (a few ulp,
// well inside the FP32 tolerance of the step) that cost a handful of
// instructions instead of the correctly rounded sequences.
template <class R> __device__ __forceinline__ R sqrt_(R x);
template <> __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_(float x) {
  return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}
template <class R> __device__ __forceinline__ R div_(R a, R b);
template <> __device__ __forceinline__ double div_(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
template <class R> __device__ __forceinline__ R tanh_(R x);
template <> __device__ __forceinline__ double tanh_(double x) { return tanh(x); }
template <> __device__ __forceinline__ float tanh_(float x) {
  // tanh x = 1 - 2 / (e^{2x} + 1); saturates correctly at +-inf
  return 1.0f - __fdividef(2.0f, __expf(2.0f * x) + 1.0f);
}
template <class R> __device__ __forceinline__ R abs_(R x);
template <> __device__ __forceinline__ double abs_(double x) { return fabs(x); }
template <> __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
template <class R> __device__ __forceinline__ R clamp01_(R x) {
  return x < R(0) ? R(0) : (x > R(1) ? R(1) : x);
}
template <class R> __device__ __forceinline__ R fminf_(R a, R b) { return a < b ? a : b; }

// ------------------------------------------------------------ stencil
// Eq. 13 written with both halves of each opposite pair merged:
// grad = (1/T) sum_i w_i c_i v_i,  lap = (2/T) sum_i w_i (v_i - v_0).
template <class R>
__device__ __forceinline__ void cd_stencil(const R v[Q], R &gx, R &gy, R &gz, R &lap) {
  const R a = R(1.0 / 18.0) * R(3.0), b = R(1.0 / 36.0) * R(3.0);
  gx = a * (v[1] - v[2]) + b * ((v[7] - v[8]) + (v[9] - v[10]) + (v[11] - v[12]) + (v[13] - v[14]));
  gy = a * (v[3] - v[4]) + b * ((v[7] - v[8]) - (v[9] - v[10]) + (v[15] - v[16]) + (v[17] - v[18]));
  gz = a * (v[5] - v[6]) + b * ((v[11] - v[12]) - (v[13] - v[14]) + (v[15] - v[16]) - (v[17] - v[18]));
  R sf = (v[1] + v[2]) + (v[3] + v[4]) + (v[5] + v[6]);
  R se = ((v[7] + v[8]) + (v[9] + v[10])) + ((v[11] + v[12]) + (v[13] + v[14])) +
         ((v[15] + v[16]) + (v[17] + v[18]));
  lap = R(6.0) * (R(1.0 / 18.0) * sf + R(1.0 / 36.0) * se - R(2.0 / 3.0) * v[0]);
}

// ------------------------------------------------------------ wetting
// Ghost values of Eqs. 14-15 with the hysteresis blend of Sec. III A.
// The tanh of a sum is evaluated through tanh(a + b) = (s + tb)/(1 + s tb)
// with s = tanh(a) = 2 phi_smpl - 1 (clamped to [-1, 1]) and
// tb = tanh(2 d_i/W), which is algebraically identical to the artanh form
// and needs no artanh.  WallDir holds what a node's links share: w (n_w
// rotated by pi - theta about n_w x grad) and s.
template <class R>
struct WallDir {
  R wx, wy, wz, s;
};
template <class R>
__device__ __forceinline__ WallDir<R> wall_dir(R phi_smpl, R gx, R gy, R gz, R nwx, R nwy,
                                               R nwz, R cth, R sth) {
  R gn = gx * nwx + gy * nwy + gz * nwz;
  R tx = gx - gn * nwx, ty = gy - gn * nwy, tz = gz - gn * nwz;
  R tn2 = tx * tx + ty * ty + tz * tz;
  R inv = tn2 >= R(1e-20) ? div_(R(1), sqrt_(tn2)) : R(0);
  tx *= inv; ty *= inv; tz *= inv;
  WallDir<R> d;
  d.wx = -cth * nwx + sth * tx;
  d.wy = -cth * nwy + sth * ty;
  d.wz = -cth * nwz + sth * tz;
  R s = R(2) * phi_smpl - R(1);
  d.s = s > R(1) ? R(1) : (s < R(-1) ? R(-1) : s);
  return d;
}
// The unblended ghost phi_{s,i} of link i (Eq. 15 with d_i = w . c_i).
template <class R>
__device__ __forceinline__ R fresh_ghost(const Model<R> &m, const WallDir<R> &w, int i) {
  R d = w.wx * R(cx_of(i)) + w.wy * R(cy_of(i)) + w.wz * R(cz_of(i));
  R tb = tanh_(m.two_over_W * d);
  return R(0.5) * (R(1) + div_(w.s + tb, R(1) + w.s * tb));
}
// ------------------------------------------------------------ macros
template <class R>
struct Macro {
  R rho, P, ux, uy, uz, mu;
};

// Chemical potential (Eq. 7), rho, velocity and pressure recovery.
template <class R>
__device__ __forceinline__ Macro<R> macros(const Model<R> &m, const R g[Q], R phi, R gx, R gy,
                                           R gz, R lap) {
  Macro<R> r;
  r.rho = m.rho_L + phi * m.rho_dif;
  r.mu = m.mu_a * phi * (phi - R(1)) * (phi - R(0.5)) - m.mu_b * lap;
  R s = R(0), jx, jy, jz;
#pragma unroll
  for (int i = 0; i < Q; ++i) s += g[i];
  jx = (g[1] - g[2]) + ((g[7] - g[8]) + (g[9] - g[10])) + ((g[11] - g[12]) + (g[13] - g[14]));
  jy = (g[3] - g[4]) + ((g[7] - g[8]) - (g[9] - g[10])) + ((g[15] - g[16]) + (g[17] - g[18]));
  jz = (g[5] - g[6]) + ((g[11] - g[12]) - (g[13] - g[14])) + ((g[15] - g[16]) - (g[17] - g[18]));
  R irho = div_(R(1), r.rho);
  r.ux = (jx + R(0.5) * (r.mu * gx + m.Fx)) * irho;
  r.uy = (jy + R(0.5) * (r.mu * gy + m.Fy)) * irho;
  r.uz = (jz + R(0.5) * (r.mu * gz + m.Fz)) * irho;
  R ug = r.ux * gx + r.uy * gy + r.uz * gz;
  r.P = R(1.0 / 3.0) * s + R(0.5 / 3.0) * m.rho_dif * ug;
  return r;
}

template <class R>
__device__ __forceinline__ R tau_mix(const Model<R> &m, R phi) {
  R F = phi;
  if (m.F_mode == 1) F = R(0.5) * (tanh_((phi - m.F_tilde) * m.inv_F_width) + R(1));
  return (R(1) - F) * m.tau_L + F * m.tau_H;
}

// Local mobility correction (Eq. 4).
template <class R>
__device__ __forceinline__ R delta_theta(const Model<R> &m, R phi, R gnorm, R lap) {
  R Y1 = fminf_(clamp01_((phi - m.phi_M) * m.inv_D), clamp01_((R(1) - phi) * m.inv_D));
  R Y2 = fminf_(clamp01_(phi * m.inv_D), clamp01_((m.phi_m - phi) * m.inv_D));
  R s = div_(lap, abs_(lap) + m.eps);  // reading R4: the sign of lap, regularised
  return m.gamma * m.theta_coef * gnorm * ((R(1) + s) * Y1 + (R(1) - s) * Y2);
}

// Both collisions of one cell, in place on h[] and g[] (Eqs. 1-11):
//   h: theta + delta-theta, h_eq = phi Gamma_i + theta w_i (c_i . n), BGK
//      with 1/tau_phi; the rest population is closed as phi - sum_{i>0} h*_i
//      (Eq. 1 conserves sum_i h_i = phi exactly; the closure keeps the
//      stored sum free of the rounding bias of sum_i Gamma_i - 1).
//   g: K_i (Eq. 6), E_i = w_i P/T + rho (Gamma_i - w_i), reading R2 of the
//      filtered collision: g* = E + K/2 + (1 - 1/tau) Phi_i : Pi with
//      Pi = sum c c (g - E + K/2).  Gamma_i - w_i is evaluated directly so
//      that the heavy phase (rho = 1) does not cancel the pressure part.
// Gamma_i is shared by the two sets.
template <class R>
__device__ __forceinline__ void collide(const Model<R> &m, R h[Q], R g[Q], const Macro<R> &mc,
                                        R phi, R gx, R gy, R gz, R lap) {
  const R ux = mc.ux, uy = mc.uy, uz = mc.uz;
  // interface normal and theta (Eqs. 2-4)
  const R gn2 = gx * gx + gy * gy + gz * gz;
  const R gnorm = sqrt_(gn2);
  const R inv = div_(R(1), gnorm + m.eps);
  R th = m.theta_coef * (R(1) - R(4) * (phi - R(0.5)) * (phi - R(0.5)));
  if (m.mobility_corr) th += delta_theta(m, phi, gnorm, lap);
  const R thn = th * inv;  // theta * n = thn * grad
  const R om = m.inv_tau_phi;
  const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  const R ug = ux * gx + uy * gy + uz * gz;
  const R uF = ux * m.Fx + uy * m.Fy + uz * m.Fz;
  const R muT = R(3) * mc.mu;  // mu / T
  const R P3 = R(3) * mc.P;    // P / T
  R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
  R rest = phi;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
    const R wi = R(w_of(i));
    const R cu = R(c0) * ux + R(c1) * uy + R(c2) * uz;
    const R Gd = wi * (cu * (R(3) + R(4.5) * cu) - uu15);  // Gamma_i - w_i
    const R G = wi + Gd;
    // h
    if (i != 0) {
      const R cgr = R(c0) * gx + R(c1) * gy + R(c2) * gz;  // c . grad phi
      const R heq = phi * G + (thn * wi) * cgr;
      h[i] = h[i] + om * (heq - h[i]);
      rest -= h[i];
    }
    // g
    const R cg = R(c0) * gx + R(c1) * gy + R(c2) * gz - ug;        // (c - u) . grad phi
    const R cF = R(c0) * m.Fx + R(c1) * m.Fy + R(c2) * m.Fz - uF;  // (c - u) . F
    const R K = (Gd * m.rho_dif + G * muT) * cg + R(3) * G * cF;
    const R E = wi * P3 + mc.rho * Gd;
    const R bse = E + R(0.5) * K;
    const R neq = g[i] - bse + K;  // g - (E - K/2)
    g[i] = bse;
    if (c0) pxx += neq;
    if (c1) pyy += neq;
    if (c2) pzz += neq;
    if (c0 * c1 > 0) pxy += neq;
    if (c0 * c1 < 0) pxy -= neq;
    if (c0 * c2 > 0) pxz += neq;
    if (c0 * c2 < 0) pxz -= neq;
    if (c1 * c2 > 0) pyz += neq;
    if (c1 * c2 < 0) pyz -= neq;
  }
  h[0] = rest;
  // Phi_i : Pi = w_i / (2 T^2) (c_i c_i : Pi - T tr Pi)
  const R tau = tau_mix(m, phi);
  const R f = (R(1) - div_(R(1), tau)) * R(4.5);
  const R tr3 = (pxx + pyy + pzz) * R(1.0 / 3.0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
    R cc = -tr3;
    if (c0) cc += pxx;
    if (c1) cc += pyy;
    if (c2) cc += pzz;
    if (c0 * c1) cc += R(2 * c0 * c1) * pxy;
    if (c0 * c2) cc += R(2 * c0 * c2) * pxz;
    if (c1 * c2) cc += R(2 * c1 * c2) * pyz;
    g[i] = g[i] + (f * R(w_of(i))) * cc;
  }
}

// collide() in pair form (same results up to rounding).  Directions i and
// opp(i) have c_opp = -c_i and equal weights, so with a = c_i . u and
// s = 1 + m, m = 9a^2/2 - 3u^2/2 (Gamma_i = w_i (s + 3a), Gamma_opp =
// w_i (s - 3a)) every per-direction term of Eqs. 2, 5 and 6 splits into a
// part even in c_i and a part odd in c_i, each evaluated once per pair:
//   h_eq   = w_i phi s               +- w_i (3 phi a + theta n . c_i)
//   K_i    = w_i (C c.grad - B u.grad - 3 s u.F + 9 a c.F)
//         +- w_i (B c.grad - C u.grad + 3 s c.F - 9 a u.F)
//            with B = m (rho_dif + mu/T) + mu/T, C = 3 a (rho_dif + mu/T)
//   E_i    = w_i (P/T + rho m)        +- 3 w_i rho a
// and the pair's non-equilibrium sum (g_i - g_eq,i) + (g_opp - g_eq,opp)
// feeds Pi with the pair's common c_i c_i.  The filtered correction of
// Eqs. 9-11 is even.  m is carried instead of s so that, as in collide(),
// the heavy phase (rho = 1) does not cancel the pressure part of E_i.
// About two thirds of collide()'s arithmetic.
template <class R>
__device__ __forceinline__ void collide_pairs(const Model<R> &m, R h[Q], R g[Q],
                                              const Macro<R> &mc, R phi, R gx, R gy, R gz,
                                              R lap) {
  const R ux = mc.ux, uy = mc.uy, uz = mc.uz;
  const R gn2 = gx * gx + gy * gy + gz * gz;
  const R gnorm = sqrt_(gn2);
  const R inv = div_(R(1), gnorm + m.eps);
  R th = m.theta_coef * (R(1) - R(4) * (phi - R(0.5)) * (phi - R(0.5)));
  if (m.mobility_corr) th += delta_theta(m, phi, gnorm, lap);
  const R thn = th * inv;  // theta n = thn grad phi
  const R om = m.inv_tau_phi;
  const R m0 = R(-1.5) * (ux * ux + uy * uy + uz * uz);  // s - 1 of the rest direction
  const R ug = ux * gx + uy * gy + uz * gz;
  const R uF = ux * m.Fx + uy * m.Fy + uz * m.Fz;
  const R rho = mc.rho;
  const R muT = R(3) * mc.mu;             // mu / T
  const R al = m.rho_dif + muT;           // rho_dif + mu / T
  const R P3 = R(3) * mc.P;               // P / T
  const R phi3 = R(3) * phi, rho3 = R(3) * rho, uF3 = R(3) * uF;
  R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
  R rest = phi;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1;  // opp(i)
    const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
    const R wi = R(w_of(i));
    const R a = R(c0) * ux + R(c1) * uy + R(c2) * uz;
    const R cgr = R(c0) * gx + R(c1) * gy + R(c2) * gz;
    const R cF = R(c0) * m.Fx + R(c1) * m.Fy + R(c2) * m.Fz;
    const R mm = m0 + R(4.5) * a * a;  // s - 1
    const R s = R(1) + mm;
    // h (Eqs. 1-2)
    const R HS = wi * (phi + phi * mm), HA = wi * (phi3 * a + thn * cgr);
    h[i] = h[i] + om * ((HS + HA) - h[i]);
    h[j] = h[j] + om * ((HS - HA) - h[j]);
    rest -= h[i] + h[j];
    // g (Eqs. 5-6 and reading R2 of Eqs. 9-11)
    const R B = mm * al + muT, C = R(3) * a * al;
    const R KS = wi * (C * cgr - B * ug - s * uF3 + R(9) * a * cF);
    const R KA = wi * (B * cgr - C * ug + R(3) * s * cF - R(9) * a * uF);
    const R ES = wi * (P3 + rho * mm), EA = wi * rho3 * a;
    const R BS = ES + R(0.5) * KS, BA = EA + R(0.5) * KA;
    const R nsum = (g[i] + g[j]) - (R(2) * ES - KS);
    g[i] = BS + BA;
    g[j] = BS - BA;
    if (c0) pxx += nsum;
    if (c1) pyy += nsum;
    if (c2) pzz += nsum;
    if (c0 * c1 > 0) pxy += nsum;
    if (c0 * c1 < 0) pxy -= nsum;
    if (c0 * c2 > 0) pxz += nsum;
    if (c0 * c2 < 0) pxz -= nsum;
    if (c1 * c2 > 0) pyz += nsum;
    if (c1 * c2 < 0) pyz -= nsum;
  }
  h[0] = rest;
  {  // rest direction: a = c . grad = c . F = 0
    const R w0 = R(w_of(0));
    const R B = m0 * al + muT;
    const R K0 = w0 * (-B * ug - (R(1) + m0) * uF3);
    g[0] = w0 * (P3 + rho * m0) + R(0.5) * K0;
  }
  const R tau = tau_mix(m, phi);
  const R f = (R(1) - div_(R(1), tau)) * R(4.5);
  const R tr3 = (pxx + pyy + pzz) * R(1.0 / 3.0);
  g[0] = g[0] - (f * R(w_of(0))) * tr3;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
    R cc = -tr3;
    if (c0) cc += pxx;
    if (c1) cc += pyy;
    if (c2) cc += pzz;
    if (c0 * c1) cc += R(2 * c0 * c1) * pxy;
    if (c0 * c2) cc += R(2 * c0 * c2) * pxz;
    if (c1 * c2) cc += R(2 * c1 * c2) * pyz;
    const R d = (f * R(w_of(i))) * cc;
    g[i] += d;
    g[i + 1] += d;
  }
}

// ------------------------------------------------------------ packed FP32
// Blackwell issues two FP32 operations on a float2 register pair as one
// instruction (add / sub / mul / fma .f32x2, each lane rounded exactly as
// its scalar form).  collide_pairs_x2 is collide_pairs with two opposite
// pairs in the two lanes: (+x, +y), (+x+y, +x-y), (+x+z, +x-z),
// (+y+z, +y-z); the +z pair stays scalar.  Within a lane the operations
// are collide_pairs' with the weight w_i factored out of K_i, E_i and the
// blends until the populations are formed, so the results agree with
// collide_pairs to rounding.  The step is issue-bound (instruction issue,
// not DRAM, limits it), so halving the issued arithmetic instructions is
// what pays.  FORCE = false drops the terms of the body force; the host
// chooses it only when F_ex = 0, where those terms vanish identically.
__device__ __forceinline__ float2 f2_(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 bc_(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2_(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2_(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2_(float2 a, float2 b) {
  unsigned long long A, B, D;
  memcpy(&A, &a, 8);
  memcpy(&B, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
  float2 d;
  memcpy(&d, &D, 8);
  return d;
}

// Dot product of c_i with (x, y, z) for a compile-time direction i.
template <int I>
__device__ __forceinline__ float cdot_(float x, float y, float z) {
  float r = 0.0f;
  bool any = false;
  if (cx_of(I) != 0) { r = cx_of(I) > 0 ? x : -x; any = true; }
  if (cy_of(I) != 0) { r = any ? (cy_of(I) > 0 ? r + y : r - y) : (cy_of(I) > 0 ? y : -y); any = true; }
  if (cz_of(I) != 0) { r = any ? (cz_of(I) > 0 ? r + z : r - z) : (cz_of(I) > 0 ? z : -z); }
  return r;
}

// Shared per-cell terms of the packed collision, as lane pairs.
struct X2Cell {
  float2 M0, AL, AL3, MUT, NUG, P3, RHO, RHO3, OM, HALF;
  float2 NUF3, NUF9;  // -3 u.F, -9 u.F (FORCE)
};

// Eq. 13 (cd_stencil) with the opposite pairs' differences and sums of the
// (+x, +y), (+x+y, +x-y), (+x+z, +x-z), (+y+z, +y-z) pairs in packed lanes.
__device__ __forceinline__ void cd_stencil_x2(const float v[Q], float &gx, float &gy, float &gz,
                                              float &lap) {
  const float a = 1.0f / 6.0f, b = 1.0f / 12.0f;
  const float2 iA = f2_(v[1], v[3]), jA = f2_(v[2], v[4]), iB = f2_(v[7], v[9]),
               jB = f2_(v[8], v[10]), iC = f2_(v[11], v[13]), jC = f2_(v[12], v[14]),
               iD = f2_(v[15], v[17]), jD = f2_(v[16], v[18]);
  const float2 dA = sub2_(iA, jA), dB = sub2_(iB, jB), dC = sub2_(iC, jC), dD = sub2_(iD, jD);
  gx = a * dA.x + b * ((dB.x + dB.y) + (dC.x + dC.y));
  gy = a * dA.y + b * ((dB.x - dB.y) + (dD.x + dD.y));
  gz = a * (v[5] - v[6]) + b * ((dC.x - dC.y) + (dD.x - dD.y));
  const float2 sA = add2_(iA, jA);
  const float2 sE = add2_(add2_(add2_(iB, jB), add2_(iC, jC)), add2_(iD, jD));
  const float sf = (sA.x + sA.y) + (v[5] + v[6]), se = sE.x + sE.y;
  lap = 6.0f * ((1.0f / 18.0f) * sf + (1.0f / 36.0f) * se - (2.0f / 3.0f) * v[0]);
}

// macros() with the moment sums of g taken over packed opposite pairs.
__device__ __forceinline__ Macro<float> macros_x2(const Model<float> &m, const float g[Q],
                                                  float phi, float gx, float gy, float gz,
                                                  float lap) {
  Macro<float> r;
  r.rho = m.rho_L + phi * m.rho_dif;
  r.mu = m.mu_a * phi * (phi - 1.0f) * (phi - 0.5f) - m.mu_b * lap;
  const float2 iA = f2_(g[1], g[3]), jA = f2_(g[2], g[4]), iB = f2_(g[7], g[9]),
               jB = f2_(g[8], g[10]), iC = f2_(g[11], g[13]), jC = f2_(g[12], g[14]),
               iD = f2_(g[15], g[17]), jD = f2_(g[16], g[18]);
  const float2 dA = sub2_(iA, jA), dB = sub2_(iB, jB), dC = sub2_(iC, jC), dD = sub2_(iD, jD);
  const float2 s2 = add2_(add2_(add2_(iA, jA), add2_(iB, jB)), add2_(add2_(iC, jC), add2_(iD, jD)));
  const float s = (s2.x + s2.y) + (g[0] + (g[5] + g[6]));
  const float jx = dA.x + ((dB.x + dB.y) + (dC.x + dC.y));
  const float jy = dA.y + ((dB.x - dB.y) + (dD.x + dD.y));
  const float jz = (g[5] - g[6]) + ((dC.x - dC.y) + (dD.x - dD.y));
  const float irho = div_(1.0f, r.rho);
  r.ux = (jx + 0.5f * (r.mu * gx + m.Fx)) * irho;
  r.uy = (jy + 0.5f * (r.mu * gy + m.Fy)) * irho;
  r.uz = (jz + 0.5f * (r.mu * gz + m.Fz)) * irho;
  const float ug = r.ux * gx + r.uy * gy + r.uz * gz;
  r.P = (1.0f / 3.0f) * s + (0.5f / 3.0f) * m.rho_dif * ug;
  return r;
}

// One packed group: lanes I and K (odd directions), opposites I + 1, K + 1,
// weight w (the same for both lanes).  Returns the pair's non-equilibrium
// sums (lane I, lane K) for Pi; h[] and g[] are updated in place and the
// moved h are subtracted from rest.
template <int I, int K, bool FORCE>
__device__ __forceinline__ float2 x2_group(const X2Cell &c, const Model<float> &m, float h[Q],
                                           float g[Q], float ux, float uy, float uz, float gx,
                                           float gy, float gz, float2 WPHI, float2 W3PHI,
                                           float2 WTHN, float2 W, float2 NW, float2 &rest) {
  const float2 a = f2_(cdot_<I>(ux, uy, uz), cdot_<K>(ux, uy, uz));
  const float2 cg = f2_(cdot_<I>(gx, gy, gz), cdot_<K>(gx, gy, gz));
  const float2 mm = fma2_(mul2_(a, bc_(4.5f)), a, c.M0);  // s - 1
  // h (Eqs. 1-2): h_eq = w phi s +- w (3 phi a + theta n . c)
  const float2 HS = fma2_(mm, WPHI, WPHI);
  const float2 HA = fma2_(a, W3PHI, mul2_(cg, WTHN));
  float2 hi = f2_(h[I], h[K]), hj = f2_(h[I + 1], h[K + 1]);
  hi = fma2_(c.OM, sub2_(add2_(HS, HA), hi), hi);
  hj = fma2_(c.OM, sub2_(sub2_(HS, HA), hj), hj);
  rest = sub2_(rest, add2_(hi, hj));
  h[I] = hi.x; h[K] = hi.y; h[I + 1] = hj.x; h[K + 1] = hj.y;
  // g (Eqs. 5-6, reading R2 of Eqs. 9-11), all divided by w
  const float2 B = fma2_(mm, c.AL, c.MUT);
  const float2 C = mul2_(a, c.AL3);
  float2 KS = fma2_(C, cg, mul2_(B, c.NUG));
  float2 KA = fma2_(B, cg, mul2_(C, c.NUG));
  if constexpr (FORCE) {
    const float2 cF = f2_(cdot_<I>(m.Fx, m.Fy, m.Fz), cdot_<K>(m.Fx, m.Fy, m.Fz));
    const float2 s = add2_(mm, bc_(1.0f));
    KS = fma2_(s, c.NUF3, fma2_(mul2_(a, bc_(9.0f)), cF, KS));
    KA = fma2_(a, c.NUF9, fma2_(mul2_(s, bc_(3.0f)), cF, KA));
  }
  const float2 ES = fma2_(c.RHO, mm, c.P3), EA = mul2_(c.RHO3, a);
  const float2 BS = fma2_(c.HALF, KS, ES), BA = fma2_(c.HALF, KA, EA);
  const float2 gi = f2_(g[I], g[K]), gj = f2_(g[I + 1], g[K + 1]);
  // non-equilibrium sum: (g_i + g_opp) - w (2 E_S - K_S)
  const float2 nsum = fma2_(NW, sub2_(add2_(ES, ES), KS), add2_(gi, gj));
  const float2 gni = mul2_(W, add2_(BS, BA)), gnj = mul2_(W, sub2_(BS, BA));
  g[I] = gni.x; g[K] = gni.y; g[I + 1] = gnj.x; g[K + 1] = gnj.y;
  return nsum;
}

// Filtered correction of a packed group: g_i and g_opp += f w_i cc_i.
template <int I, int K>
__device__ __forceinline__ void x2_filter(float g[Q], float2 cc, float2 FW) {
  const float2 d = mul2_(FW, cc);
  const float2 gi = add2_(f2_(g[I], g[K]), d), gj = add2_(f2_(g[I + 1], g[K + 1]), d);
  g[I] = gi.x; g[K] = gi.y; g[I + 1] = gj.x; g[K + 1] = gj.y;
}

template <bool FORCE>
__device__ __forceinline__ void collide_pairs_x2(const Model<float> &m, float h[Q], float g[Q],
                                                 const Macro<float> &mc, float phi, float gx,
                                                 float gy, float gz, float lap) {
  const float ux = mc.ux, uy = mc.uy, uz = mc.uz;
  const float gnorm = sqrt_(gx * gx + gy * gy + gz * gz);
  const float inv = div_(1.0f, gnorm + m.eps);
  float th = m.theta_coef * (1.0f - 4.0f * (phi - 0.5f) * (phi - 0.5f));
  if (m.mobility_corr) th += delta_theta(m, phi, gnorm, lap);
  const float thn = th * inv;  // theta n = thn grad phi
  const float m0 = -1.5f * (ux * ux + uy * uy + uz * uz);
  const float ug = ux * gx + uy * gy + uz * gz;
  const float uF = FORCE ? ux * m.Fx + uy * m.Fy + uz * m.Fz : 0.0f;
  const float muT = 3.0f * mc.mu, al = m.rho_dif + muT, P3 = 3.0f * mc.P, rho = mc.rho;
  X2Cell c;
  c.M0 = bc_(m0); c.AL = bc_(al); c.AL3 = bc_(3.0f * al); c.MUT = bc_(muT); c.NUG = bc_(-ug);
  c.P3 = bc_(P3); c.RHO = bc_(rho); c.RHO3 = bc_(3.0f * rho); c.OM = bc_(m.inv_tau_phi);
  c.HALF = bc_(0.5f);
  if (FORCE) { c.NUF3 = bc_(-3.0f * uF); c.NUF9 = bc_(-9.0f * uF); }
  constexpr float wf = 1.0f / 18.0f, we = 1.0f / 36.0f;
  float2 rest = f2_(phi, 0.0f);
  // faces (+x, +y)
  const float2 nA = x2_group<1, 3, FORCE>(c, m, h, g, ux, uy, uz, gx, gy, gz, bc_(wf * phi),
                                          bc_(3.0f * wf * phi), bc_(wf * thn), bc_(wf),
                                          bc_(-wf), rest);
  // edges
  const float2 WPHI = bc_(we * phi), W3PHI = bc_(3.0f * we * phi), WTHN = bc_(we * thn);
  const float2 W = bc_(we), NW = bc_(-we);
  const float2 nB = x2_group<7, 9, FORCE>(c, m, h, g, ux, uy, uz, gx, gy, gz, WPHI, W3PHI, WTHN,
                                          W, NW, rest);
  const float2 nC = x2_group<11, 13, FORCE>(c, m, h, g, ux, uy, uz, gx, gy, gz, WPHI, W3PHI,
                                            WTHN, W, NW, rest);
  const float2 nD = x2_group<15, 17, FORCE>(c, m, h, g, ux, uy, uz, gx, gy, gz, WPHI, W3PHI,
                                            WTHN, W, NW, rest);
  // +z pair, scalar (collide_pairs' arithmetic)
  float n5;
  float rs = rest.x + rest.y;
  {
    const float a = uz, cgr = gz, mm = m0 + 4.5f * a * a;
    const float HS = wf * (phi + phi * mm), HA = wf * (3.0f * phi * a + thn * cgr);
    h[5] = h[5] + m.inv_tau_phi * ((HS + HA) - h[5]);
    h[6] = h[6] + m.inv_tau_phi * ((HS - HA) - h[6]);
    rs -= h[5] + h[6];
    const float B = mm * al + muT, C = 3.0f * a * al;
    float KS = C * cgr - B * ug, KA = B * cgr - C * ug;
    if (FORCE) {
      const float s = 1.0f + mm, cF = m.Fz;
      KS += -s * 3.0f * uF + 9.0f * a * cF;
      KA += 3.0f * s * cF - 9.0f * a * uF;
    }
    const float ES = P3 + rho * mm, EA = 3.0f * rho * a;
    const float BS = ES + 0.5f * KS, BA = EA + 0.5f * KA;
    n5 = (g[5] + g[6]) - wf * (2.0f * ES - KS);
    g[5] = wf * (BS + BA);
    g[6] = wf * (BS - BA);
  }
  h[0] = rs;
  {  // rest direction: a = c . grad = c . F = 0
    constexpr float w0 = 1.0f / 3.0f;
    const float B = m0 * al + muT;
    const float K0 = w0 * (-B * ug - (1.0f + m0) * 3.0f * uF);
    g[0] = w0 * (P3 + rho * m0) + 0.5f * K0;
  }
  // Pi from the pairs' sums: (+x,+y) | (+x+y,+x-y) | (+x+z,+x-z) | (+y+z,+y-z) | +z
  const float tB = nB.x + nB.y, tC = nC.x + nC.y, tD = nD.x + nD.y;
  const float pxx = nA.x + tB + tC, pyy = nA.y + tB + tD, pzz = n5 + tC + tD;
  const float pxy = nB.x - nB.y, pxz = nC.x - nC.y, pyz = nD.x - nD.y;
  const float tau = tau_mix(m, phi);
  const float f = (1.0f - div_(1.0f, tau)) * 4.5f;
  const float tr3 = (pxx + pyy + pzz) * (1.0f / 3.0f);
  g[0] = g[0] - (f * (1.0f / 3.0f)) * tr3;
  const float2 FWf = bc_(f * wf), FWe = bc_(f * we);
  x2_filter<1, 3>(g, f2_(pxx - tr3, pyy - tr3), FWf);
  const float bxy = pxx + pyy - tr3, bxz = pxx + pzz - tr3, byz = pyy + pzz - tr3;
  x2_filter<7, 9>(g, f2_(bxy + 2.0f * pxy, bxy - 2.0f * pxy), FWe);
  x2_filter<11, 13>(g, f2_(bxz + 2.0f * pxz, bxz - 2.0f * pxz), FWe);
  x2_filter<15, 17>(g, f2_(byz + 2.0f * pyz, byz - 2.0f * pyz), FWe);
  const float d5 = (f * wf) * (pzz - tr3);
  g[5] += d5;
  g[6] += d5;
}

// h_eq (Eqs. 2-4) for initialisation.
template <class R>
__device__ __forceinline__ void h_equilibrium(const Model<R> &m, R h[Q], R phi, R gx, R gy, R gz,
                                              R lap) {
  const R gnorm = sqrt_(gx * gx + gy * gy + gz * gz);
  R th = m.theta_coef * (R(1) - R(4) * (phi - R(0.5)) * (phi - R(0.5)));
  if (m.mobility_corr) th += delta_theta(m, phi, gnorm, lap);
  const R thn = div_(th, gnorm + m.eps);
  R rest = phi;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const R cgr = R(cx_of(i)) * gx + R(cy_of(i)) * gy + R(cz_of(i)) * gz;
    h[i] = phi * R(w_of(i)) + (thn * R(w_of(i))) * cgr;
    rest -= h[i];
  }
  h[0] = rest;
}

}  // namespace pflb
