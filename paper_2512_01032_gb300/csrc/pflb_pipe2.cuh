// pflb_pipe2.cuh -- the pipelined step with two cells per thread and packed
// FP32 arithmetic (FP32 storage, periodic x, nx a multiple of 4).
//
// Same step, same staging and the same shared-memory buffers as k_pipe
// (arXiv 2512.01032, Sec. II and Sec. III A; see pflb_pipe.cuh), but each
// of the 64 threads of a block owns the two neighbouring cells x0 + 2t and
// x0 + 2t + 1 of a 32 x 4 tile row.  The per-cell arithmetic of the bulk
// cells (Eq. 13 stencils, the macroscopic recovery, both collisions of
// Eqs. 1-11 in pair form, the diagnostics) runs once for the pair on
// float2 values with the sm_100 packed instructions (__ffma2_rn,
// __fadd2_rn, __fmul2_rn: two FP32 results per issued instruction), and the
// pair's populations move as 8-byte words where both cells' slots are
// adjacent: shared-memory reads of h, of g on even steps and of the
// stencil's phi values, and global stores of the directions without an x
// component.  The step is issue-bound, so halving the instructions of the
// arithmetic is what lifts it; the price is two warps per block instead of
// four.  Wall nodes are left to k_wall, as with k_pipe.
#pragma once
#include "pflb_pipe.cuh"

namespace pflb {
namespace p2 {

using f2 = float2;
__device__ __forceinline__ f2 sp(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return __ffma2_rn(b, sp(-1.0f), a); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 ld2(const float *p) { return *reinterpret_cast<const f2 *>(p); }
__device__ __forceinline__ void st2(float *p, f2 v) { *reinterpret_cast<f2 *>(p) = v; }

// c_i . (vx, vy, vz) for the D3Q19 direction i (components 0 or +-1).
__device__ __forceinline__ f2 cdot(int i, f2 vx, f2 vy, f2 vz) {
  const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
  f2 r = sp(0.0f);
  bool any = false;
  auto acc = [&](int c, f2 v) {
    if (c == 0) return;
    if (!any) {
      r = c > 0 ? v : v * sp(-1.0f);
      any = true;
    } else {
      r = c > 0 ? r + v : r - v;
    }
  };
  acc(c0, vx);
  acc(c1, vy);
  acc(c2, vz);
  return r;
}

}  // namespace p2

constexpr int P2_NT = 64;              // threads per block: 16 pairs x 4 rows
constexpr int P2_PW = PP_BX + 4;       // phi ring row: x0 - 2 .. x0 + 33
constexpr int P2_PS = P2_PW * PP_ROWS;

struct Pipe2Smem {
  static constexpr int V = 4, W = PP_BX + 2 * V, NCH = W / V;
  float h[2][Q][PP_ROWS][W];       // h of planes z + 1 and z + 2, slot = plane & 1
  float g[Q][PP_BY][W];            // g arriving at the cells of the next plane
  float phi[4][P2_PS];             // phi ring, slot = plane & 3; column = x - x0 + 2
  uint32_t fl[4][PP_ROWS][PP_FW];  // flag words, x0 - 4 .. x0 + 36, slot = plane & 3
};

// Update of the two bulk cells (xa, y, z), (xa + 1, y, z): h, g the
// streamed populations, phi and val[1..18] their phi and their neighbours'.
// oka / okb: which of the two is a bulk fluid cell to store.
template <bool ODD, bool DIAG>
__device__ __forceinline__ void bulk_pair(const Args<float, float> &a, int xa, int y, int z,
                                          int ca, bool oka, bool okb, const Nbr &nb,
                                          p2::f2 h[Q], p2::f2 g[Q], p2::f2 phi,
                                          const p2::f2 val[Q], DiagAcc<float> &acc) {
  using namespace p2;
  const Model<float> &m = a.m;
  // ---- Eq. 13, both halves of each opposite pair merged (as cd_stencil)
  const f2 d1 = val[1] - val[2], d3 = val[3] - val[4], d5 = val[5] - val[6];
  const f2 d7 = val[7] - val[8], d9 = val[9] - val[10], d11 = val[11] - val[12];
  const f2 d13 = val[13] - val[14], d15 = val[15] - val[16], d17 = val[17] - val[18];
  const f2 A = sp(1.0f / 6.0f), B = sp(1.0f / 12.0f);
  const f2 gx = fma2(A, d1, B * ((d7 + d9) + (d11 + d13)));
  const f2 gy = fma2(A, d3, B * ((d7 - d9) + (d15 + d17)));
  const f2 gz = fma2(A, d5, B * ((d11 - d13) + (d15 - d17)));
  const f2 sf = (val[1] + val[2]) + (val[3] + val[4]) + (val[5] + val[6]);
  const f2 se = ((val[7] + val[8]) + (val[9] + val[10])) + ((val[11] + val[12]) + (val[13] + val[14])) +
                ((val[15] + val[16]) + (val[17] + val[18]));
  const f2 lap = fma2(sp(1.0f / 3.0f), sf, fma2(sp(1.0f / 6.0f), se, phi * sp(-4.0f)));

  // ---- macroscopic fields (Eq. 7 and the recovery after Eq. 11)
  const f2 rho = fma2(phi, sp(m.rho_dif), sp(m.rho_L));
  const f2 mu = fma2(sp(m.mu_a), phi * (phi - sp(1.0f)) * (phi - sp(0.5f)), lap * sp(-m.mu_b));
  const f2 s = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) +
               (((g[8] + g[9]) + (g[10] + g[11])) + ((g[12] + g[13]) + (g[14] + g[15]))) +
               ((g[16] + g[17]) + g[18]);
  const f2 e1 = g[1] - g[2], e3 = g[3] - g[4], e5 = g[5] - g[6], e7 = g[7] - g[8];
  const f2 e9 = g[9] - g[10], e11 = g[11] - g[12], e13 = g[13] - g[14];
  const f2 e15 = g[15] - g[16], e17 = g[17] - g[18];
  const f2 jx = e1 + ((e7 + e9) + (e11 + e13));
  const f2 jy = e3 + ((e7 - e9) + (e15 + e17));
  const f2 jz = e5 + ((e11 - e13) + (e15 - e17));
  const f2 irho = make_float2(div_(1.0f, rho.x), div_(1.0f, rho.y));
  const f2 ux = fma2(sp(0.5f), fma2(mu, gx, sp(m.Fx)), jx) * irho;
  const f2 uy = fma2(sp(0.5f), fma2(mu, gy, sp(m.Fy)), jy) * irho;
  const f2 uz = fma2(sp(0.5f), fma2(mu, gz, sp(m.Fz)), jz) * irho;
  const f2 ug = fma2(ux, gx, fma2(uy, gy, uz * gz));
  const f2 P = fma2(sp(1.0f / 3.0f), s, sp(m.rho_dif * (0.5f / 3.0f)) * ug);

  if (DIAG) {
    const f2 u2 = fma2(ux, ux, fma2(uy, uy, uz * uz));
    const f2 kin = sp(0.5f) * rho * u2;
    const float ph[2] = {phi.x, phi.y}, pr[2] = {P.x, P.y}, uu[2] = {u2.x, u2.y};
    const float kk[2] = {kin.x, kin.y}, pn[2] = {val[1].x, val[1].y};
    const bool ok[2] = {oka, okb};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      if (!ok[l]) continue;
      const int x = xa + l;
      const float p = ph[l];
      acc.v[D_MASS] += p;
      if (p >= 0.5f) acc.v[D_NHEAVY] += 1.0f;
      if (p > 0.95f) { acc.v[D_PH] += pr[l]; acc.v[D_NPH] += 1.0f; }
      if (p < 0.05f) { acc.v[D_PL] += pr[l]; acc.v[D_NPL] += 1.0f; }
      if (z >= a.reg[4] && z < a.reg[5] && x >= a.reg[0] && x < a.reg[1] && y >= a.reg[2] &&
          y < a.reg[3]) {
        acc.v[D_REGION] += p;
        const float q = pn[l];  // phi of the +x neighbour, a fluid cell
        if (p >= 0.5f && q < 0.5f) {
          const float xc = (float)x + div_(p - 0.5f, p - q);
          acc.front = xc + 1.0f > acc.front ? xc + 1.0f : acc.front;
        } else if (p < 0.5f && q >= 0.5f) {
          const float xc = (float)x + div_(0.5f - p, q - p);
          acc.rear = (float)a.nx - xc > acc.rear ? (float)a.nx - xc : acc.rear;
        }
      }
      acc.v[D_KIN] += kk[l];
      if (!finite_(p + pr[l] + uu[l])) acc.v[D_NONFINITE] += 1.0f;
      acc.umax = uu[l] > acc.umax ? uu[l] : acc.umax;
    }
  }

  // ---- both collisions in pair form (collide_pairs, Eqs. 1-11)
  const f2 gn2 = fma2(gx, gx, fma2(gy, gy, gz * gz));
  const f2 gnorm = make_float2(sqrt_(gn2.x), sqrt_(gn2.y));
  const f2 inv = make_float2(div_(1.0f, gnorm.x + m.eps), div_(1.0f, gnorm.y + m.eps));
  const f2 hp = phi - sp(0.5f);
  f2 th = sp(m.theta_coef) * fma2(sp(-4.0f), hp * hp, sp(1.0f));
  if (m.mobility_corr)
    th = th + make_float2(delta_theta(m, phi.x, gnorm.x, lap.x),
                          delta_theta(m, phi.y, gnorm.y, lap.y));
  const f2 thn = th * inv;
  const f2 om = sp(m.inv_tau_phi);
  const f2 m0 = sp(-1.5f) * fma2(ux, ux, fma2(uy, uy, uz * uz));
  const f2 uF = fma2(ux, sp(m.Fx), fma2(uy, sp(m.Fy), uz * sp(m.Fz)));
  const f2 muT = sp(3.0f) * mu;
  const f2 al = sp(m.rho_dif) + muT;
  const f2 P3 = sp(3.0f) * P;
  const f2 phi3 = sp(3.0f) * phi, rho3 = sp(3.0f) * rho, uF3 = sp(3.0f) * uF;
  f2 pxx = sp(0.0f), pyy = pxx, pzz = pxx, pxy = pxx, pxz = pxx, pyz = pxx;
  f2 rest = phi;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1;
    const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
    const float wi = (float)w_of(i);
    const f2 au = cdot(i, ux, uy, uz);
    const f2 cgr = cdot(i, gx, gy, gz);
    const float cF = (float)c0 * m.Fx + (float)c1 * m.Fy + (float)c2 * m.Fz;
    const f2 mm = fma2(sp(4.5f), au * au, m0);
    const f2 sv = mm + sp(1.0f);
    const f2 HS = sp(wi) * fma2(phi, mm, phi);
    const f2 HA = sp(wi) * fma2(phi3, au, thn * cgr);
    h[i] = fma2(om, (HS + HA) - h[i], h[i]);
    h[j] = fma2(om, (HS - HA) - h[j], h[j]);
    rest = rest - (h[i] + h[j]);
    const f2 Bv = fma2(mm, al, muT), Cv = sp(3.0f) * au * al;
    const f2 KS = sp(wi) * (fma2(Cv, cgr, fma2(sp(9.0f * cF), au, sp(0.0f))) - fma2(Bv, ug, sv * uF3));
    const f2 KA = sp(wi) * (fma2(Bv, cgr, sp(3.0f * cF) * sv) - fma2(Cv, ug, sp(9.0f) * au * uF));
    const f2 ES = sp(wi) * fma2(rho, mm, P3), EA = sp(wi) * (rho3 * au);
    const f2 BS = fma2(sp(0.5f), KS, ES), BA = fma2(sp(0.5f), KA, EA);
    const f2 nsum = (g[i] + g[j]) - fma2(sp(2.0f), ES, sp(0.0f) - KS);
    g[i] = BS + BA;
    g[j] = BS - BA;
    if (c0) pxx = pxx + nsum;
    if (c1) pyy = pyy + nsum;
    if (c2) pzz = pzz + nsum;
    if (c0 * c1 > 0) pxy = pxy + nsum;
    if (c0 * c1 < 0) pxy = pxy - nsum;
    if (c0 * c2 > 0) pxz = pxz + nsum;
    if (c0 * c2 < 0) pxz = pxz - nsum;
    if (c1 * c2 > 0) pyz = pyz + nsum;
    if (c1 * c2 < 0) pyz = pyz - nsum;
  }
  h[0] = rest;
  {
    const float w0 = (float)w_of(0);
    const f2 Bv = fma2(m0, al, muT);
    const f2 K0 = sp(w0) * (sp(0.0f) - fma2(Bv, ug, (m0 + sp(1.0f)) * uF3));
    g[0] = fma2(sp(w0), fma2(rho, m0, P3), sp(0.5f) * K0);
  }
  const f2 tau = make_float2(tau_mix(m, phi.x), tau_mix(m, phi.y));
  const f2 fr = make_float2((1.0f - div_(1.0f, tau.x)) * 4.5f, (1.0f - div_(1.0f, tau.y)) * 4.5f);
  const f2 tr3 = ((pxx + pyy) + pzz) * sp(1.0f / 3.0f);
  g[0] = g[0] - (fr * sp((float)w_of(0))) * tr3;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int c0 = cx_of(i), c1 = cy_of(i), c2 = cz_of(i);
    f2 cc = sp(0.0f) - tr3;
    if (c0) cc = cc + pxx;
    if (c1) cc = cc + pyy;
    if (c2) cc = cc + pzz;
    if (c0 * c1) cc = fma2(sp((float)(2 * c0 * c1)), pxy, cc);
    if (c0 * c2) cc = fma2(sp((float)(2 * c0 * c2)), pxz, cc);
    if (c1 * c2) cc = fma2(sp((float)(2 * c1 * c2)), pyz, cc);
    const f2 d = (fr * sp((float)w_of(i))) * cc;
    g[i] = g[i] + d;
    g[i + 1] = g[i + 1] + d;
  }

  // ---- streaming: h pushed, g A-A.  Cells xa and xa + 1 (xa even, nx a
  // multiple of 4, so ca is even and their slots form an aligned 8-byte
  // word in every direction without an x component).
  const int xm_a = xa == 0 ? a.nx - 1 : -1;        // x - 1 of cell a
  const int xp_b = xa + 1 == a.nx - 1 ? 1 - a.nx : 1;  // x + 1 of cell b
  const bool both = oka && okb;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i);
    int yz = 0;
    if (cy_of(i) > 0) yz += nb.yp;
    if (cy_of(i) < 0) yz += nb.ym;
    if (cz_of(i) > 0) yz += nb.zp;
    if (cz_of(i) < 0) yz += nb.zm;
    if (cx == 0) {
      float *p = a.hout[i] + (ca + yz);
      if (both) st2(p, h[i]);
      else if (oka) p[0] = h[i].x;
      else if (okb) p[1] = h[i].y;
    } else {
      const int oa = yz + (cx > 0 ? 1 : xm_a), ob = yz + (cx > 0 ? xp_b : -1);
      if (oka) a.hout[i][ca + oa] = h[i].x;
      if (okb) a.hout[i][ca + 1 + ob] = h[i].y;
    }
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i);
    if (!ODD) {
      float *p = a.g[opp_of(i)] + ca;
      if (both) st2(p, g[i]);
      else if (oka) p[0] = g[i].x;
      else if (okb) p[1] = g[i].y;
    } else {
      int yz = 0;
      if (cy_of(i) > 0) yz += nb.yp;
      if (cy_of(i) < 0) yz += nb.ym;
      if (cz_of(i) > 0) yz += nb.zp;
      if (cz_of(i) < 0) yz += nb.zm;
      if (cx == 0) {
        float *p = a.g[i] + (ca + yz);
        if (both) st2(p, g[i]);
        else if (oka) p[0] = g[i].x;
        else if (okb) p[1] = g[i].y;
      } else {
        const int oa = yz + (cx > 0 ? 1 : xm_a), ob = yz + (cx > 0 ? xp_b : -1);
        if (oka) a.g[i][ca + oa] = g[i].x;
        if (okb) a.g[i][ca + 1 + ob] = g[i].y;
      }
    }
  }
}

// One tile column (x0, y0) over planes [zb, ze): k_pipe's march with 64
// threads, each owning cells x0 + 2 tx and x0 + 2 tx + 1 of row y0 + ty.
template <bool ODD, bool DIAG>
__device__ __forceinline__ void pipe2_march(const Args<float, float> &a, int x0, int y0, int zb,
                                            int ze, Pipe2Smem &sm, float (*wacc)[32]) {
  using namespace p2;
  using SM = Pipe2Smem;
  constexpr int V = SM::V, NCH = SM::NCH, NT = P2_NT;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int nx = a.nx, ny = a.ny, nz = a.nz, sz = nx * ny;
  const int xa = x0 + 2 * tx;            // even; xa + 1 < nx whenever xa < nx
  const bool valid = xa < nx && (y0 + ty) < ny;
  const int cxa = xa % nx, cy0 = (y0 + ty) % ny;
  const int col = cxa + nx * cy0;
  // ring cells (x0 - 1 .. x0 + 32 on rows y0 - 1 and y0 + 4, x0 - 1 and
  // x0 + 32 on the tile rows): 76 jobs over 64 threads
  constexpr int NR = PP_NR;
  int rx[2] = {0, 0}, ry[2] = {0, 0};
  bool ring[2] = {false, false};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int rj = tid + k * NT;
    if (rj < NR) {
      ring[k] = true;
      if (rj < PP_PW) {
        rx[k] = rj; ry[k] = 0;
      } else if (rj < 2 * PP_PW) {
        rx[k] = rj - PP_PW; ry[k] = PP_BY + 1;
      } else {
        const int q = rj - 2 * PP_PW;
        rx[k] = (q & 1) ? PP_BX + 1 : 0;
        ry[k] = 1 + (q >> 1);
      }
    }
  }  // rx: x - x0 + 1 in [0, 34)
  auto wrapz = [nz](int zu) {
    while (zu < 0) zu += nz;
    while (zu >= nz) zu -= nz;
    return zu;
  };
  auto wrap = [](int v, int n) { return ((v % n) + n) % n; };

  constexpr int HU = 2 * PP_ROWS * NCH, GU = 2 * PP_BY * NCH;
  constexpr int HPT = (HU + NT - 1) / NT, GPT = (GU + NT - 1) / NT;
  int h_rc[HPT], h_off[HPT];
  int g_rc[GPT], g_off[GPT][3];
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int u = tid + k * NT;
    h_rc[k] = -1;
    h_off[k] = 0;
    if (u < HU) {
      const int half = u >= HU / 2, v = u - half * (HU / 2);
      const int r = v / NCH, ch = v - r * NCH;
      h_rc[k] = half << 16 | r << 8 | ch;
      h_off[k] = wrap(x0 - V + ch * V, nx) + nx * wrap(y0 - 1 + r, ny);
    }
  }
#pragma unroll
  for (int k = 0; k < GPT; ++k) {
    const int u = tid + k * NT;
    g_rc[k] = -1;
    g_off[k][0] = g_off[k][1] = g_off[k][2] = 0;
    if (u < GU) {
      const int half = u >= GU / 2, v = u - half * (GU / 2);
      const int r = v / NCH, ch = v - r * NCH;
      g_rc[k] = half << 16 | r << 8 | ch;
      const int xs = wrap(x0 - V + ch * V, nx);
#pragma unroll
      for (int d = 0; d < 3; ++d) g_off[k][d] = xs + nx * wrap(y0 + r - 1 + d, ny);
    }
  }
  const int fj = tid < PP_ROWS * PP_FW ? tid : -1;
  int fl_off = -1;
  if (fj >= 0) fl_off = wrap(x0 - 4 + 4 * (fj % PP_FW), nx) + nx * wrap(y0 - 1 + fj / PP_FW, ny);

  auto stage_flags = [&](int zu) {
    if (fl_off >= 0)
      cp_async_4(&sm.fl[zu & 3][fj / PP_FW][fj % PP_FW], a.flags + (fl_off + sz * wrapz(zu)));
  };
  auto stage_h = [&](int zu, bool skip_solid) {
    const int zoff = sz * wrapz(zu);
    const uint32_t (*fl)[PP_FW] = sm.fl[zu & 3];
    float(*dst)[PP_ROWS][SM::W] = sm.h[zu & 1];
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
      if (h_rc[k] < 0) continue;
      const int half = h_rc[k] >> 16, r = (h_rc[k] >> 8) & 0xff, ch = h_rc[k] & 0xff;
      if (skip_solid && chunk_solid<V>(fl[r], ch)) continue;
      const int cell = h_off[k] + zoff;
      if (!half) {
#pragma unroll
        for (int i = 0; i < 10; ++i) cp_async_16(&dst[i][r][ch * V], a.hin[i] + cell);
      } else {
#pragma unroll
        for (int i = 10; i < Q; ++i) cp_async_16(&dst[i][r][ch * V], a.hin[i] + cell);
      }
    }
  };
  auto stage_g = [&](int zu) {
    const int z = wrapz(zu);
    const uint32_t (*fl)[PP_FW] = sm.fl[zu & 3];
#pragma unroll
    for (int u = 0; u < GPT; ++u) {
      if (g_rc[u] < 0) continue;
      const int half = g_rc[u] >> 16, r = (g_rc[u] >> 8) & 0xff, ch = g_rc[u] & 0xff;
      const int k0 = half ? 10 : 0, k1 = half ? Q : 10;
      if constexpr (!ODD) {
        if (ch == 0 || ch == NCH - 1) continue;
        if (chunk_solid<V>(fl[r + 1], ch)) continue;
        const int cell = g_off[u][1] + sz * z;
#pragma unroll
        for (int k = 0; k < Q; ++k)
          if (k >= k0 && k < k1) cp_async_16(&sm.g[k][r][ch * V], a.g[k] + cell);
      } else {
        const int zo[3] = {sz * wrapz(zu - 1), sz * z, sz * wrapz(zu + 1)};
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          if (k < k0 || k >= k1) continue;
          const int cxk = cx_of(k), cyk = cy_of(k), czk = cz_of(k);
          const int lo = (V - (cxk > 0 ? cxk : 0)) / V;
          const int hi = (V + PP_BX - 1 - (cxk < 0 ? cxk : 0)) / V;
          if (ch < lo || ch > hi) continue;
          cp_async_16(&sm.g[k][r][ch * V], a.g[opp_of(k)] + (g_off[u][1 - cyk] + zo[1 - czk]));
        }
      }
    }
  };
  auto staged_phi = [&](const float (*st)[PP_ROWS][SM::W], int row, int idx) {
    float v = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) v += st[i][row][idx];
    return v;
  };
  auto phi_plane = [&](int zu) {
    const float(*st)[PP_ROWS][SM::W] = sm.h[zu & 1];
    const uint32_t (*fl)[PP_FW] = sm.fl[zu & 3];
    float *dst = sm.phi[zu & 3];
    const int ia = V + 2 * tx;  // staged column of cell a
    const uint8_t fa = flag_byte(fl, ty + 1, 2 * tx), fb = flag_byte(fl, ty + 1, 2 * tx + 1);
    // the two cells' h as 8-byte words, summed in the order cell_phi uses
    f2 sum = p2::sp(0.0f);
#pragma unroll
    for (int i = 0; i < Q; ++i) sum = sum + p2::ld2(&st[i][ty + 1][ia]);
    const float va = (fa & F_SOLID) ? 0.0f : sum.x, vb = (fb & F_SOLID) ? 0.0f : sum.y;
    p2::st2(&dst[(ty + 1) * P2_PW + 2 + 2 * tx], make_float2(va, vb));
    if (valid && zu >= zb && zu < ze) {
      if (fa & F_NEAR) a.phi_w[col + sz * zu] = va;
      if (fb & F_NEAR) a.phi_w[col + 1 + sz * zu] = vb;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (ring[k])
        dst[ry[k] * P2_PW + rx[k] + 1] =
            (flag_byte(fl, ry[k], rx[k] - 1) & F_SOLID) ? 0.0f : staged_phi(st, ry[k], V - 1 + rx[k]);
  };

  DiagAcc<float> tot;
  tot.zero();
  if (DIAG) diag_block_zero(wacc);

  for (int zu = zb - 1; zu <= zb + 2; ++zu) stage_flags(zu);
  stage_h(zb - 1, false);
  stage_h(zb, false);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  phi_plane(zb - 1);
  phi_plane(zb);
  __syncthreads();
  stage_h(zb + 1, true);
  stage_g(zb);
  cp_async_commit();

  const int o = (ty + 1) * P2_PW + 2 + 2 * tx;  // ring index of cell a
  for (int z = zb; z < ze; ++z) {
    cp_async_wait_all();
    __syncthreads();
    phi_plane(z + 1);
    const int c = col + sz * z;
    const uint8_t fa = flag_byte(sm.fl[z & 3], ty + 1, 2 * tx);
    const uint8_t fb = flag_byte(sm.fl[z & 3], ty + 1, 2 * tx + 1);
    const bool oka = valid && !(fa & (F_SOLID | F_WALL));
    const bool okb = valid && !(fb & (F_SOLID | F_WALL));
    f2 h[Q], g[Q];
    if (oka || okb) {
      const int ia = V + 2 * tx;
#pragma unroll
      for (int i = 0; i < Q; ++i) h[i] = p2::ld2(&sm.h[z & 1][i][ty + 1][ia]);
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        if (!ODD || cx_of(k) == 0) {
          g[k] = p2::ld2(&sm.g[k][ty][ia]);
        } else {
          const float *p = &sm.g[k][ty][ia - cx_of(k)];
          g[k] = make_float2(p[0], p[1]);
        }
      }
    }
    __syncthreads();
    if (z + 2 <= ze) stage_h(z + 2, true);
    if (z + 1 < ze) stage_g(z + 1);
    if (z + 3 <= ze) stage_flags(z + 3);
    cp_async_commit();
    if (oka || okb) {
      Nbr nb;
      nb.init(cxa, cy0, z, nx, ny, nz);
      const float *p0 = sm.phi[z & 3], *pm = sm.phi[(z - 1) & 3], *pp = sm.phi[(z + 1) & 3];
      // the phi values of the pair's neighbours, rows (dy, dz) read as the
      // aligned words at x - 2, x, x + 2 (x = cell a)
      f2 val[Q];
      const f2 ctr = p2::ld2(p0 + o);
      val[0] = ctr;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const float *pl = cz_of(i) == 0 ? p0 : (cz_of(i) > 0 ? pp : pm);
        const int r = o + cy_of(i) * P2_PW;
        if (cx_of(i) == 0) {
          val[i] = p2::ld2(pl + r);
        } else if (cx_of(i) > 0) {
          const f2 mid = p2::ld2(pl + r), right = p2::ld2(pl + r + 2);
          val[i] = make_float2(mid.y, right.x);
        } else {
          const f2 left = p2::ld2(pl + r - 2), mid = p2::ld2(pl + r);
          val[i] = make_float2(left.y, mid.x);
        }
      }
      DiagAcc<float> acc;
      acc.zero();
      bulk_pair<ODD, DIAG>(a, cxa, cy0, z, c, oka, okb, nb, h, g, ctr, val, acc);
      if (DIAG) {
#pragma unroll
        for (int k = 0; k < D_UMAX; ++k) tot.v[k] += acc.v[k];
        tot.umax = tot.umax > acc.umax ? tot.umax : acc.umax;
        tot.front = tot.front > acc.front ? tot.front : acc.front;
        tot.rear = tot.rear > acc.rear ? tot.rear : acc.rear;
      }
    }
  }
  cp_async_wait_all();
  if (DIAG) {
    diag_warp_add(wacc[tid >> 5], tot);
    diag_block_flush(a.diag, wacc);
  }
}

template <bool ODD, bool DIAG>
__global__ void __launch_bounds__(P2_NT, 4) k_pipe2(const __grid_constant__ Args<float, float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float wacc[DIAG_MAX_WARPS][32];
  zero_next_diag(a);
  const int zb = blockIdx.z * a.lz;
  pipe2_march<ODD, DIAG>(a, blockIdx.x * PP_BX, blockIdx.y * PP_BY, zb, min(zb + a.lz, a.nz),
                         *reinterpret_cast<Pipe2Smem *>(smem_raw), wacc);
}

}  // namespace pflb
