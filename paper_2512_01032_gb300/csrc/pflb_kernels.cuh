// pflb_kernels.cuh -- CUDA kernels of one time step of the phase-field LB
// method (arXiv 2512.01032, Sec. II and Sec. III A) on a periodic D3Q19
// lattice with voxel walls.
//
// Memory layout (SoA, x fastest, cell = x + nx*(y + ny*z), N < 2^31):
//   h  : two buffers [19][N]; push streaming from h[t&1] into h[(t+1)&1].
//        Two buffers because the fused kernel recomputes phi = sum_i h_i in
//        a one-cell halo around its tile; in place, a neighbouring block
//        could overwrite those populations mid-step.
//   g  : one buffer [19][N], in-place A-A streaming.  Even steps read and
//        write the cell's own slots (writing slot opp(i)); odd steps gather
//        slot opp(k) of x - c_k and scatter into slot i of x + c_i.
//   wp : per wall node, g populations crossing a solid link, double buffered
//        [2][18][nwall].  Step t reads wp[t&1] and writes wp[(t+1)&1]; this
//        lets the free-slip (specular) rule hand a population to the
//        tangential neighbour without two threads touching one A-A slot.
//   ghost : per wall node, wetting ghosts phi_{s,i} [18][nwall] (compute type).
//   flags : uint8 per cell (bit0 solid, bit1 wall node); widx: wall index.
// The 19 per-direction base pointers of each population array travel in the
// kernel parameters (constant bank), so an access costs one multiply-add.
#pragma once
#include "pflb_internal.h"
#include "pflb_model.cuh"

namespace pflb {

enum { MODE_STEP = 0, MODE_MACRO = 1 };
// Collision forms: per direction (collide), per opposite pair
// (collide_pairs), pairs in packed FP32 lanes with and without the body
// force terms (collide_pairs_x2; FP32 arithmetic only, else collide_pairs).
enum { COLL_PLAIN = 0, COLL_PAIRS = 1, COLL_X2 = 2, COLL_X2_NOF = 3 };

// Blocks of 256 threads per SM the batch kernel is compiled for (sets its
// register cap: 128).
#ifndef PFLB_MIN_BLOCKS
#define PFLB_MIN_BLOCKS 2
#endif

// Register cap of the plain fused kernel.  At 96 registers five 128-thread
// blocks fit on an SM (20 warps instead of the 16 that 128 registers allow);
// the FP32 and 16-bit instantiations then spill 36-52 bytes per thread, and
// the extra warps hide more of the DRAM latency that bounds the kernel.
#ifndef PFLB_FUSED_MAXNREG
#define PFLB_FUSED_MAXNREG 96
#endif

template <class S, class R>
struct Args {
  int nx, ny, nz, lz;
  int N;
  int nw;
  const S *hin[Q + 1];   // direction bases of the h buffer being read (+ rest remainder)
  S *hout[Q + 1];        // direction bases of the h buffer being written
  S *g[Q];           // direction bases of the g buffer (in place)
  const uint8_t *flags;
  const int *widx;
  const uint32_t *wmask;
  const int *wcell;  // [nw] cell of each wall node
  const R *wgeo;     // [5][nw]: n_w (x,y,z), cos theta, sin theta
  const uint32_t *wcut; // [nw] links into cut cells (bits 1..18) | c_n << 24, or null
  const R *sfrac;    // [N] solid volume fraction (1 on solid cells), or null
  R *ghost;          // [18][nw]
  const S *wp_rd;    // [18][nw]
  S *wp_wr;          // [18][nw]
  const R *phi;      // [N] phi field (two-pass path and field reads)
  R *phi_w;          // the same field, written by the pipelined kernel for wall nodes' reads
  Model<R> m;
  double *diag;      // [D_COUNT] accumulator of this launch, or null
  double *diag_zero; // [32] accumulator of the next diagnostic launch, zeroed here
  int reg[6];        // diagnostic box [x0,x1) x [y0,y1) x [z0,z1)
  double *out;       // macro outputs [6][N] (phi, rho, P, ux, uy, uz) or null
  R *bcm;            // open x boundaries: states [5][nbc] (phi, P, ux, uy, uz), or null
  int nbc;           // 2 ny nz: plane x = 0, then plane x = nx-1
  // pipelined kernel: wall records grouped by the block whose march covers
  // them (block b owns wl[wl_start[b] .. wl_start[b + 1])), or null
  const int *wl;
  const int *wl_start;
};

// Index of the boundary state of a cell in plane x = 0 or x = nx-1.
template <class S, class R>
__device__ __forceinline__ int bc_index(const Args<S, R> &a, int x, int yz) {
  return yz + (x == 0 ? 0 : a.ny * a.nz);
}

template <class R>
struct DiagAcc {
  R v[D_UMAX];
  R umax;          // max |u|^2
  R front, rear;   // D_FRONT, D_REAR (maxima, 0 = no crossing)
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < D_UMAX; ++k) v[k] = R(0);
    umax = R(0);
    front = R(0);
    rear = R(0);
  }
};

// Periodic neighbour offsets of one cell from six per-axis deltas.
struct Nbr {
  int xm, xp, ym, yp, zm, zp;
  __device__ __forceinline__ void init(int x, int y, int z, int nx, int ny, int nz) {
    const int sy = nx, sz = nx * ny;
    xm = x == 0 ? nx - 1 : -1;
    xp = x == nx - 1 ? 1 - nx : 1;
    ym = (y == 0 ? ny - 1 : -1) * sy;
    yp = (y == ny - 1 ? 1 - ny : 1) * sy;
    zm = (z == 0 ? nz - 1 : -1) * sz;
    zp = (z == nz - 1 ? 1 - nz : 1) * sz;
  }
  // offset of x + c_i relative to x
  __device__ __forceinline__ int off(int i) const {
    int o = 0;
    if (cx_of(i) > 0) o += xp;
    if (cx_of(i) < 0) o += xm;
    if (cy_of(i) > 0) o += yp;
    if (cy_of(i) < 0) o += ym;
    if (cz_of(i) > 0) o += zp;
    if (cz_of(i) < 0) o += zm;
    return o;
  }
};

template <class R>
__device__ __forceinline__ bool finite_(R v) { return isfinite(v); }

// Gather the g populations arriving at cell c (A-A): solid sources come
// from the wall population buffer.
template <class S, class R, bool ODD>
__device__ __forceinline__ void gather_g(const Args<S, R> &a, int c, uint32_t lm, int rec,
                                         const Nbr &nb, R g[Q]) {
  if (lm == 0) {  // bulk cell: no solid link
#pragma unroll
    for (int k = 0; k < Q; ++k)
      g[k] = ODD ? ld_g<S, R>(a.g[opp_of(k)] + (c + nb.off(opp_of(k))), k)
                 : ld_g<S, R>(a.g[k] + c, k);
    return;
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    if (k != 0 && ((lm >> opp_of(k)) & 1u)) {
      g[k] = ld_g<S, R>(a.wp_rd + ((k - 1) * a.nw + rec), k);
    } else if (!ODD) {
      g[k] = ld_g<S, R>(a.g[k] + c, k);
    } else {
      g[k] = ld_g<S, R>(a.g[opp_of(k)] + (c + nb.off(opp_of(k))), k);
    }
  }
}

template <class S, class R, bool ODD>
__device__ __forceinline__ void store_cell(const Args<S, R> &a, int c, uint32_t lm, int rec,
                                           const Nbr &nb, R h[Q], R g[Q], const R val[Q],
                                           bool in_band);

// Open x boundary cell (reading R22): not collided; its post-collision
// populations are the equilibria at the boundary state formed before the
// step (k_xbc), h_i = phi_b Gamma_i(u_b), g_i = w_i P_b / T +
// rho_b (Gamma_i - w_i); no diagnostics, no ghost update, no free-slip band.
template <class S, class R, bool ODD, int MODE>
__device__ __forceinline__ void boundary_cell(const Args<S, R> &a, int x, int y, int z, int c,
                                              uint32_t lm, int rec, const Nbr &nb) {
  const int j = bc_index(a, x, y + a.ny * z), nb5 = a.nbc;
  const R phib = a.bcm[j], Pb = a.bcm[nb5 + j];
  const R ux = a.bcm[2 * nb5 + j], uy = a.bcm[3 * nb5 + j], uz = a.bcm[4 * nb5 + j];
  const R rho = a.m.rho_L + phib * a.m.rho_dif;
  if (MODE == MODE_MACRO) {
    if (a.out) {
      const long long N = a.N;
      a.out[c] = (double)phib;
      a.out[N + c] = (double)rho;
      a.out[2 * N + c] = (double)Pb;
      a.out[3 * N + c] = (double)ux;
      a.out[4 * N + c] = (double)uy;
      a.out[5 * N + c] = (double)uz;
    }
    return;
  }
  const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  R h[Q], g[Q], val[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R wi = R(w_of(i));
    const R cu = R(cx_of(i)) * ux + R(cy_of(i)) * uy + R(cz_of(i)) * uz;
    const R Gd = wi * (cu * (R(3) + R(4.5) * cu) - uu15);  // Gamma_i - w_i
    h[i] = phib * (wi + Gd);
    g[i] = wi * R(3) * Pb + rho * Gd;
    val[i] = R(0);
  }
  store_cell<S, R, ODD>(a, c, lm, rec, nb, h, g, val, false);
}

// Rest of the update (or macro evaluation) of one fluid cell c at (x, y, z)
// once its populations are gathered: h[] and g[] hold the streamed
// populations, phi = sum h, val[1..18] the phi of the 18 neighbours
// (anything for solid ones), lm/rec the wall data (0 for bulk cells).
template <class S, class R, bool ODD, int MODE, bool DIAG, bool XBC = false, int PAIRS = COLL_PLAIN>
__device__ __forceinline__ void finish_cell(const Args<S, R> &a, int x, int y, int z, int c,
                                            uint8_t f, uint32_t lm, int rec, const Nbr &nb,
                                            R h[Q], R g[Q], R phi, R val[Q], DiagAcc<R> &acc) {
  const Model<R> &m = a.m;
  if constexpr (XBC) {
    if (f & F_BC) {
      boundary_cell<S, R, ODD, MODE>(a, x, y, z, c, lm, rec, nb);
      return;
    }
  }
  val[0] = phi;
  R gx, gy, gz, lap;
  // Stencil corrections of the cut links (sub-voxel walls): a cut
  // neighbour y enters the CD stencils as s_y ghost + (1 - s_y) phi(y); val
  // keeps phi(y), which the free-slip band and the front probe read, and
  // s_y (ghost - phi(y)) is added through the stencil weights (3 w_i c_i
  // for the gradient, 6 w_i for the Laplacian).
  R cgx = R(0), cgy = R(0), cgz = R(0), clap = R(0);
  const bool wall = (f & F_WALL) != 0;
  if (wall) {
    const int nw = a.nw;
    // sub-voxel walls: links into cut cells and the sample direction c_n
    const uint32_t cw = a.wcut ? a.wcut[rec] : 0u;
    const uint32_t lc = cw & 0x7fffeu;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if ((lm >> i) & 1u) val[i] = a.ghost[(i - 1) * nw + rec];
    // phi_smpl: the node's phi, or for a cut node the average over the
    // parallelepiped on the wall, (1 - s_x) phi + s_x phi(x + c_n)
    R smpl = phi;
    if (cw >> 24) {
      const int cn = (int)(cw >> 24);
      R pn = phi;
#pragma unroll
      for (int i = 1; i <= 6; ++i)
        if (i == cn) pn = val[i];
      const R sx = a.sfrac[c];
      smpl = (R(1) - sx) * phi + sx * pn;
    }
    cd_stencil(val, gx, gy, gz, lap);  // grad phi with the previous ghosts
    if (lc) {
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if ((lc >> i) & 1u) {
          const R d = a.sfrac[c + nb.off(i)] * (a.ghost[(i - 1) * nw + rec] - val[i]) *
                      R(3.0 * w_of(i));
          gx += R(cx_of(i)) * d;
          gy += R(cy_of(i)) * d;
          gz += R(cz_of(i)) * d;
        }
    }
    const WallDir<R> wd = wall_dir(smpl, gx, gy, gz, a.wgeo[rec], a.wgeo[nw + rec],
                                   a.wgeo[2 * nw + rec], a.wgeo[3 * nw + rec],
                                   a.wgeo[4 * nw + rec]);
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if ((lm >> i) & 1u) {
        val[i] = m.blend * val[i] + (R(1) - m.blend) * fresh_ghost(m, wd, i);
        if (MODE == MODE_STEP) a.ghost[(i - 1) * nw + rec] = val[i];
      }
    if (lc) {
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if ((lc >> i) & 1u) {
          const R gnew = m.blend * a.ghost[(i - 1) * nw + rec] +
                         (R(1) - m.blend) * fresh_ghost(m, wd, i);
          if (MODE == MODE_STEP) a.ghost[(i - 1) * nw + rec] = gnew;
          const R d = a.sfrac[c + nb.off(i)] * (gnew - val[i]);
          cgx += R(3.0 * w_of(i) * cx_of(i)) * d;
          cgy += R(3.0 * w_of(i) * cy_of(i)) * d;
          cgz += R(3.0 * w_of(i) * cz_of(i)) * d;
          clap += R(6.0 * w_of(i)) * d;
        }
    }
  }
  if constexpr (PAIRS >= COLL_X2 && std::is_same<R, float>::value)
    cd_stencil_x2(val, gx, gy, gz, lap);
  else
    cd_stencil(val, gx, gy, gz, lap);
  if (wall) {
    gx += cgx;
    gy += cgy;
    gz += cgz;
    lap += clap;
  }
  Macro<R> mc;
  if constexpr (PAIRS >= COLL_X2 && std::is_same<R, float>::value)
    mc = macros_x2(m, g, phi, gx, gy, gz, lap);
  else
    mc = macros(m, g, phi, gx, gy, gz, lap);

  if (DIAG) {
    acc.v[D_MASS] += phi;
    if (phi >= R(0.5)) acc.v[D_NHEAVY] += R(1);
    if (phi > R(0.95)) { acc.v[D_PH] += mc.P; acc.v[D_NPH] += R(1); }
    if (phi < R(0.05)) { acc.v[D_PL] += mc.P; acc.v[D_NPL] += R(1); }
    if (z >= a.reg[4] && z < a.reg[5] && x >= a.reg[0] && x < a.reg[1] && y >= a.reg[2] &&
        y < a.reg[3]) {
      acc.v[D_REGION] += phi;
      // phi = 0.5 crossings towards the +x neighbour (a fluid cell): the
      // interface position of Sec. III C (front: phi falls through 0.5 along
      // +x; rear: phi rises through it), linearly interpolated
      if (!((lm >> 1) & 1u)) {
        const R pn = val[1];
        if (phi >= R(0.5) && pn < R(0.5)) {
          const R xc = R(x) + div_(phi - R(0.5), phi - pn);
          acc.front = xc + R(1) > acc.front ? xc + R(1) : acc.front;
        } else if (phi < R(0.5) && pn >= R(0.5)) {
          const R xc = R(x) + div_(R(0.5) - phi, pn - phi);
          acc.rear = R(a.nx) - xc > acc.rear ? R(a.nx) - xc : acc.rear;
        }
      }
    }
    if (wall && phi >= R(0.25) && phi <= R(0.75)) {
      acc.v[D_CLN] += R(1);
      acc.v[D_CLX] += R(x); acc.v[D_CLY] += R(y); acc.v[D_CLZ] += R(z);
      acc.v[D_CLXX] += R(x) * R(x); acc.v[D_CLYY] += R(y) * R(y); acc.v[D_CLZZ] += R(z) * R(z);
    }
    const R u2 = mc.ux * mc.ux + mc.uy * mc.uy + mc.uz * mc.uz;
    acc.v[D_KIN] += R(0.5) * mc.rho * u2;
    if (!finite_(phi + mc.P + u2)) acc.v[D_NONFINITE] += R(1);  // NaN/Inf propagate
    acc.umax = u2 > acc.umax ? u2 : acc.umax;  // squared; root taken at the flush
  }
  if (MODE == MODE_MACRO) {
    if (a.out) {
      const long long N = a.N;
      a.out[c] = (double)phi;
      a.out[N + c] = (double)mc.rho;
      a.out[2 * N + c] = (double)mc.P;
      a.out[3 * N + c] = (double)mc.ux;
      a.out[4 * N + c] = (double)mc.uy;
      a.out[5 * N + c] = (double)mc.uz;
    }
    return;
  }

  if constexpr (PAIRS >= COLL_X2 && std::is_same<R, float>::value)
    collide_pairs_x2<PAIRS == COLL_X2>(m, h, g, mc, phi, gx, gy, gz, lap);
  else if constexpr (PAIRS >= COLL_PAIRS)
    collide_pairs(m, h, g, mc, phi, gx, gy, gz, lap);
  else
    collide(m, h, g, mc, phi, gx, gy, gz, lap);
  store_cell<S, R, ODD>(a, c, lm, rec, nb, h, g, val,
                        m.free_slip && phi >= m.band_lo && phi <= m.band_hi);
}

// Streaming of one cell's post-collision populations: h pushed into the
// other buffer (halfway bounce-back at solid links), g written A-A; g on
// solid links goes to the wall population buffer, to this node
// (bounce-back) or, when in_band and the neighbour's phi (val) is in the
// band too, to the tangential neighbour (specular reflection, Sec. III A).
template <class S, class R, bool ODD>
__device__ __forceinline__ void store_cell(const Args<S, R> &a, int c, uint32_t lm, int rec,
                                           const Nbr &nb, R h[Q], R g[Q], const R val[Q],
                                           bool in_band) {
  const Model<R> &m = a.m;
  S he[Q], h_lo, ge[Q];
  enc_h_cell<S, R>(h, he, &h_lo);
  enc_g_cell<S, R>(g, ge);
  if constexpr (Codec<S>::narrow) a.hout[Q][c] = h_lo;  // rest population stays

  if (lm == 0) {  // bulk cell: plain streaming of both sets
#pragma unroll
    for (int i = 0; i < Q; ++i) a.hout[i][c + nb.off(i)] = he[i];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (!ODD)
        a.g[opp_of(i)][c] = ge[i];
      else
        a.g[i][c + nb.off(i)] = ge[i];
    }
    return;
  }
  // h: push into the other buffer, halfway bounce-back at solid links.
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i != 0 && ((lm >> i) & 1u))
      a.hout[opp_of(i)][c] = he[i];  // same weight class as i
    else
      a.hout[i][c + nb.off(i)] = he[i];
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i != 0 && ((lm >> i) & 1u)) {
      int drec = rec, ddir = opp_of(i);
      if (in_band) {
        const EdgeInfo e = edge_info(i);
        if (e.fa >= 0) {
          // Flat wall across axis a (face fa solid, fb fluid) or axis b.
          const bool sa = (lm >> e.fa) & 1u, sb = (lm >> e.fb) & 1u;
          const bool wa = sa && !sb, wb = sb && !sa;
          if (wa || wb) {
            const R py = wa ? val[e.fb] : val[e.fa];
            if (py >= m.band_lo && py <= m.band_hi) {
              drec = a.widx[c + (wa ? nb.off(e.fb) : nb.off(e.fa))];
              ddir = wa ? e.ra : e.rb;
            }
          }
        }
      }
      a.wp_wr[(ddir - 1) * a.nw + drec] = ge[i];
    } else if (!ODD) {
      a.g[opp_of(i)][c] = ge[i];
    } else {
      a.g[i][c + nb.off(i)] = ge[i];
    }
  }
}

// Full update (or macro evaluation) of one fluid cell: wall data, g
// gather, then finish_cell.
template <class S, class R, bool ODD, int MODE, bool DIAG, bool XBC = false, int PAIRS = COLL_PLAIN>
__device__ __forceinline__ void update_cell(const Args<S, R> &a, int x, int y, int z, int c,
                                            uint8_t f, R h[Q], R phi, R val[Q],
                                            DiagAcc<R> &acc) {
  Nbr nb;
  nb.init(x, y, z, a.nx, a.ny, a.nz);
  uint32_t lm = 0;
  int rec = 0;
  if (f & F_WALL) {
    rec = a.widx[c];
    lm = a.wmask[rec];
  }
  R g[Q];
  gather_g<S, R, ODD>(a, c, lm, rec, nb, g);
  finish_cell<S, R, ODD, MODE, DIAG, XBC, PAIRS>(a, x, y, z, c, f, lm, rec, nb, h, g, phi, val,
                                                 acc);
}

// Diagnostics are reduced in three levels: each cell's contributions (a
// DiagAcc zeroed per cell) are summed over the warp with shuffles once per
// plane into per-warp slots in shared memory (compute precision: FP32 work
// stays off the slow FP64 pipe); at the end of the block the slots are
// summed in FP64 and added to the device accumulator with FP64 atomics.
// Nothing is carried in registers across the z march.
constexpr int DIAG_MAX_WARPS = 8;

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R>
__device__ __forceinline__ void diag_warp_add(R *slot, const DiagAcc<R> &d) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < D_CLN; ++k) {
    const R t = warp_sum(d.v[k]);
    if (lane == 0) slot[k] += t;
  }
  if (__any_sync(0xffffffffu, d.v[D_CLN] != R(0))) {  // contact-line band cells (rare)
#pragma unroll
    for (int k = D_CLN; k <= D_CLZZ; ++k) {
      const R t = warp_sum(d.v[k]);
      if (lane == 0) slot[k] += t;
    }
  }
#pragma unroll
  for (int k = D_KIN; k < D_UMAX; ++k) {
    const R t = warp_sum(d.v[k]);
    if (lane == 0) slot[k] += t;
  }
  R um = d.umax, fr = d.front, re = d.rear;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
    fr = fmax(fr, __shfl_xor_sync(0xffffffffu, fr, o));
    re = fmax(re, __shfl_xor_sync(0xffffffffu, re, o));
  }
  if (lane == 0) {
    slot[D_UMAX] = slot[D_UMAX] > um ? slot[D_UMAX] : um;
    slot[D_FRONT] = slot[D_FRONT] > fr ? slot[D_FRONT] : fr;
    slot[D_REAR] = slot[D_REAR] > re ? slot[D_REAR] : re;
  }
}

template <class R>
__device__ __forceinline__ void diag_block_zero(R (*wacc)[32]) {
  for (int k = threadIdx.x; k < DIAG_MAX_WARPS * 32; k += blockDim.x) (&wacc[0][0])[k] = R(0);
}

template <class R>
__device__ __forceinline__ void diag_block_flush(double *diag, R (*wacc)[32]) {
  __syncthreads();
  const int nwarps = (blockDim.x + 31) >> 5;
  const int k = threadIdx.x;
  if (k < D_COUNT) {
    const bool is_max = k >= D_UMAX;
    double t = 0.0;
    for (int w = 0; w < nwarps; ++w)
      t = is_max ? fmax(t, (double)wacc[w][k]) : t + (double)wacc[w][k];
    if (is_max) {
      // non-negative doubles order like their bit patterns; D_UMAX holds
      // the squared speed until here
      if (k == D_UMAX) t = sqrt(t);
      if (t > 0.0)
        atomicMax((unsigned long long *)(diag + k), (unsigned long long)__double_as_longlong(t));
    } else if (t != 0.0) {
      atomicAdd(diag + k, t);
    }
  }
}

// Per-thread diagnostic slots in shared memory, laid out [quantity][thread]:
// each fluid cell adds its contributions to its own thread's slots (no
// cross-lane work per plane), and the block reduces the slots once, at the
// end of its tile column, through the per-warp slots above.
template <class R>
__host__ __device__ constexpr size_t diag_thread_bytes(int threads) {
  return (size_t)D_COUNT * threads * sizeof(R);
}

template <class R>
__device__ __forceinline__ void diag_thread_zero(R *tacc) {
  const int nt = blockDim.x, t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < D_COUNT; ++k) tacc[k * nt + t] = R(0);
}

template <class R>
__device__ __forceinline__ void diag_thread_add(R *tacc, const DiagAcc<R> &d) {
  const int nt = blockDim.x, t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < D_CLN; ++k) tacc[k * nt + t] += d.v[k];
  if (d.v[D_CLN] != R(0)) {  // contact-line band cells (rare)
#pragma unroll
    for (int k = D_CLN; k <= D_CLZZ; ++k) tacc[k * nt + t] += d.v[k];
  }
#pragma unroll
  for (int k = D_KIN; k < D_UMAX; ++k) tacc[k * nt + t] += d.v[k];
  R &um = tacc[D_UMAX * nt + t];
  um = um > d.umax ? um : d.umax;
  R &fr = tacc[D_FRONT * nt + t];
  fr = fr > d.front ? fr : d.front;
  R &re = tacc[D_REAR * nt + t];
  re = re > d.rear ? re : d.rear;
}

// Block reduction of the per-thread slots into the device accumulator
// (called by every thread of the block, after the last diag_thread_add).
template <class R>
__device__ __forceinline__ void diag_thread_flush(double *diag, const R *tacc,
                                                  R (*wacc)[32]) {
  const int nt = blockDim.x, t = threadIdx.x;
  diag_block_zero(wacc);
  __syncthreads();
  DiagAcc<R> d;
#pragma unroll
  for (int k = 0; k < D_UMAX; ++k) d.v[k] = tacc[k * nt + t];
  d.umax = tacc[D_UMAX * nt + t];
  d.front = tacc[D_FRONT * nt + t];
  d.rear = tacc[D_REAR * nt + t];
  diag_warp_add(wacc[t >> 5], d);
  diag_block_flush(diag, wacc);
}

// phi of one cell from the h buffer being read (0 for solid cells).
template <class S, class R, bool XBC = false>
__device__ __forceinline__ R cell_phi(const Args<S, R> &a, int c) {
  const uint8_t f = a.flags[c];
  if (f & F_SOLID) return R(0);
  if constexpr (XBC) {
    if (f & F_BC) return a.bcm[bc_index(a, c % a.nx, c / a.nx)];  // phi_b
  }
  R h[Q];
  ld_h_cell<S, R>(a.hin, c, h);
  R s = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) s += h[i];
  return s;
}

template <class S, class R>
__device__ __forceinline__ void zero_next_diag(const Args<S, R> &a) {
  if (a.diag_zero && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < 32)
    a.diag_zero[threadIdx.x] = 0.0;
}

// --------------------------------------------------------- two-pass path
// Pass 1: phi field.
template <class S, class R, bool XBC = false>
__global__ void k_phi(const __grid_constant__ Args<S, R> a, R *phi_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.N) return;
  phi_out[c] = cell_phi<S, R, XBC>(a, c);
}

// Pass 2: one thread per cell, neighbour phi from the field.
template <class S, class R, bool ODD, int MODE, bool DIAG, bool XBC = false>
__global__ void __launch_bounds__(256) k_cell(const __grid_constant__ Args<S, R> a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  zero_next_diag(a);
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  if (DIAG) {
    diag_block_zero(wacc);
    __syncthreads();
  }
  DiagAcc<R> acc;
  acc.zero();
  if (c < a.N) {
    const uint8_t f = a.flags[c];
    if (MODE == MODE_MACRO && (f & F_SOLID) && a.out) {
      // fields are defined as zero on solid cells
#pragma unroll
      for (int k = 0; k < 6; ++k) a.out[(long long)k * a.N + c] = 0.0;
    }
    if (!(f & F_SOLID)) {
      const int x = c % a.nx;
      const int y = (c / a.nx) % a.ny;
      const int z = c / (a.nx * a.ny);
      Nbr nb;
      nb.init(x, y, z, a.nx, a.ny, a.nz);
      R h[Q], val[Q];
      R phi = R(0);
      ld_h_cell<S, R>(a.hin, c, h);
#pragma unroll
      for (int i = 0; i < Q; ++i) phi += h[i];
#pragma unroll
      for (int i = 1; i < Q; ++i) val[i] = a.phi[c + nb.off(i)];
      update_cell<S, R, ODD, MODE, DIAG, XBC>(a, x, y, z, c, f, h, phi, val, acc);
    }
  }
  if (DIAG) {
    diag_warp_add(wacc[threadIdx.x >> 5], acc);
    diag_block_flush(a.diag, wacc);
  }
}

// ------------------------------------------------------------ fused path
// One thread per (x, y) column of a BX x BY tile, marching z over a chunk
// of planes.  phi of three consecutive planes over the tile plus a
// one-cell ring is kept in shared memory; each plane's phi is recomputed
// from the h populations (own cells and ring cells), so no phi field is
// stored in HBM.  march_tile does one tile column [zb, ze) of lattice a;
// sphi holds 3 (BX+2)(BY+2) values, tacc the per-thread diagnostic slots
// (zeroed by the caller, each thread its own).
template <class S, class R, bool ODD, bool DIAG, bool XBC = false>
__device__ __forceinline__ void march_tile(const Args<S, R> &a, int x0, int y0, int zb, int ze,
                                           int BX, int BY, R *sphi, R *tacc) {
  const int PW = BX + 2, PS = (BX + 2) * (BY + 2);
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int sz = nx * ny;
  const bool active = ty < BY;
  const bool valid = active && (x0 + tx) < nx && (y0 + ty) < ny;
  const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
  const int col = gx + nx * gy;
  // ring cell of this thread (smem coords), if any
  const int nring = 2 * PW + 2 * BY;
  int rx = -1, ry = -1;
  if (tid < nring) {
    if (tid < PW) { rx = tid; ry = 0; }
    else if (tid < 2 * PW) { rx = tid - PW; ry = BY + 1; }
    else { int k = tid - 2 * PW; rx = (k & 1) ? BX + 1 : 0; ry = 1 + (k >> 1); }
  }
  const int rcol = ((x0 + rx - 1) % nx + nx) % nx + nx * (((y0 + ry - 1) % ny + ny) % ny);

  auto plane = [&](int zu) {  // fill phi of (unwrapped) plane zu into its ring slot
    const int zw = ((zu % nz) + nz) % nz;
    R *dst = sphi + (((zu % 3) + 3) % 3) * PS;
    if (active) dst[(ty + 1) * PW + tx + 1] = cell_phi<S, R, XBC>(a, col + sz * zw);
    if (rx >= 0) dst[ry * PW + rx] = cell_phi<S, R, XBC>(a, rcol + sz * zw);
  };

  plane(zb - 1);
  plane(zb);
  for (int z = zb; z < ze; ++z) {
    plane(z + 1);
    __syncthreads();
    DiagAcc<R> acc;
    acc.zero();
    if (valid) {
      const int c = col + sz * z;
      const uint8_t f = a.flags[c];
      if (!(f & F_SOLID)) {
        R h[Q], val[Q];
        ld_h_cell<S, R>(a.hin, c, h);
        const R *p0 = sphi + (((z % 3) + 3) % 3) * PS;
        const R *pm = sphi + ((((z - 1) % 3) + 3) % 3) * PS;
        const R *pp = sphi + ((((z + 1) % 3) + 3) % 3) * PS;
        const int o = (ty + 1) * PW + tx + 1;
        const R phi = p0[o];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const R *pl = cz_of(i) == 0 ? p0 : (cz_of(i) > 0 ? pp : pm);
          val[i] = pl[o + cy_of(i) * PW + cx_of(i)];
        }
        update_cell<S, R, ODD, MODE_STEP, DIAG, XBC>(a, gx, gy, z, c, f, h, phi, val, acc);
        if (DIAG) diag_thread_add(tacc, acc);
      }
    }
    __syncthreads();
  }
}

// Dynamic shared memory of the fused kernel: the 3-plane phi ring, then
// (with diagnostics) the per-thread diagnostic slots.
template <class R>
__host__ __device__ constexpr size_t fused_phi_bytes(int BX, int BY) {
  return (3 * (size_t)(BX + 2) * (BY + 2) * sizeof(R) + 15) & ~size_t(15);
}
template <class R>
__host__ __device__ constexpr size_t fused_smem_bytes(int BX, int BY, bool diag) {
  return fused_phi_bytes<R>(BX, BY) + (diag ? diag_thread_bytes<R>(BX * BY) : 0);
}

template <class S, class R, bool ODD, bool DIAG, bool XBC = false>
__global__ void __maxnreg__(PFLB_FUSED_MAXNREG)
    k_fused(const __grid_constant__ Args<S, R> a, int BX, int BY) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sphi = reinterpret_cast<R *>(smem_raw);
  R *tacc = reinterpret_cast<R *>(smem_raw + fused_phi_bytes<R>(BX, BY));
  zero_next_diag(a);
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  if (DIAG) diag_thread_zero(tacc);
  const int zb = blockIdx.z * a.lz;
  march_tile<S, R, ODD, DIAG, XBC>(a, blockIdx.x * BX, blockIdx.y * BY, zb, min(zb + a.lz, a.nz), BX,
                              BY, sphi, tacc);
  if (DIAG) diag_thread_flush(a.diag, tacc, wacc);
}

// ------------------------------------------------------ open boundaries
// Boundary states of the open x planes (reading R22), formed before each
// step from the state the step will read: given values, and for the
// Neumann quantities the adjacent interior cell's bulk moments (phi = sum h,
// P = T sum g, rho u = sum c g + F/2), its g gathered exactly as that cell
// will gather it.  One thread per cell of the two planes; no other kernel
// runs meanwhile, so the reads cannot race the step's writes.
// XbcSpec (types and given values of the two planes) is in pflb_internal.h.

template <class S, class R, bool ODD>
__device__ __forceinline__ void xbc_cell(const Args<S, R> &a, const XbcSpec &sp, R *bcm, int j,
                                         long long t) {
  const int plane = a.ny * a.nz;
  const int side = j >= plane, yz = j - side * plane;
  const int y = yz % a.ny, z = yz / a.ny;
  const int xa = side ? a.nx - 2 : 1;
  const int ca = xa + a.nx * yz;
  const uint8_t fa = a.flags[ca];
  R phia = R(0), Pa = R(0), ua[3] = {R(0), R(0), R(0)};
  if (!(fa & F_SOLID)) {
    R h[Q], g[Q];
    ld_h_cell<S, R>(a.hin, ca, h);
    Nbr nb;
    nb.init(xa, y, z, a.nx, a.ny, a.nz);
    uint32_t lm = 0;
    int rec = 0;
    if (fa & F_WALL) {
      rec = a.widx[ca];
      lm = a.wmask[rec];
    }
    gather_g<S, R, ODD>(a, ca, lm, rec, nb, g);
    R s0 = R(0), m0 = R(0), m1 = R(0), m2 = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      phia += h[i];
      s0 += g[i];
      m0 += R(cx_of(i)) * g[i];
      m1 += R(cy_of(i)) * g[i];
      m2 += R(cz_of(i)) * g[i];
    }
    const R rho = a.m.rho_L + phia * a.m.rho_dif;
    ua[0] = (m0 + R(0.5) * a.m.Fx) / rho;
    ua[1] = (m1 + R(0.5) * a.m.Fy) / rho;
    ua[2] = (m2 + R(0.5) * a.m.Fz) / rho;
    Pa = s0 / R(3);
  }
  const int n = 2 * plane;
  if (sp.type[side] == 1) {
    bcm[j] = phia;
    bcm[n + j] = (R)xbc_value(sp, side, 0, t);
    bcm[2 * n + j] = ua[0];
    bcm[3 * n + j] = ua[1];
    bcm[4 * n + j] = ua[2];
  } else {
    bcm[j] = (R)xbc_value(sp, side, 4, t);
    bcm[n + j] = Pa;
    bcm[2 * n + j] = (R)xbc_value(sp, side, 1, t);
    bcm[3 * n + j] = (R)xbc_value(sp, side, 2, t);
    bcm[4 * n + j] = (R)xbc_value(sp, side, 3, t);
  }
}

template <class S, class R, bool ODD>
__global__ void k_xbc(const __grid_constant__ Args<S, R> a, const __grid_constant__ XbcSpec sp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * a.ny * a.nz) xbc_cell<S, R, ODD>(a, sp, a.bcm, j, sp.step0);
}

// Sets (on) or clears (off) the boundary flag of the fluid cells of the
// planes x = 0 and x = nx-1.
static __global__ void k_mark_xbc(uint8_t *flags, int nx, int plane, int on) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 2 * plane) return;
  const int side = j >= plane, yz = j - side * plane;
  const long long c = (side ? nx - 1 : 0) + (long long)nx * yz;
  const uint8_t f = flags[c];
  if (f & F_SOLID) return;
  flags[c] = on ? (uint8_t)(f | F_BC) : (uint8_t)(f & ~F_BC);
}

// ------------------------------------------------------------ init
// Equilibrium initial state from phi0 (reading: u = 0, P = P0, K from the
// initial gradient, ghosts = phi of the wall node).  Writes the h buffer
// given in h0 (the one step 0 reads) and wall populations into wp0.
template <class S, class R>
__global__ void k_init(const __grid_constant__ Args<S, R> a, const double *phi0, double P0,
                       S *h0base, S *wp0) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.N) return;
  const long long N = a.N;
  const uint8_t f = a.flags[c];
  if (f & F_SOLID) {
#pragma unroll
    for (int i = 0; i < h_slots<S>(); ++i) h0base[i * N + c] = enc_pop<S, R>(R(0), 0);
#pragma unroll
    for (int i = 0; i < Q; ++i) st_g<S, R>(a.g[i] + c, i, R(0));
    return;
  }
  const int x = c % a.nx, y = (c / a.nx) % a.ny, z = c / (a.nx * a.ny);
  Nbr nb;
  nb.init(x, y, z, a.nx, a.ny, a.nz);
  const R phi = (R)phi0[c];
  R val[Q];
  val[0] = phi;
  uint32_t lm = 0, lc = 0;
  int rec = 0;
  if (f & F_WALL) {
    rec = a.widx[c];
    lm = a.wmask[rec];
    if (a.wcut) lc = a.wcut[rec] & 0x7fffeu;
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    val[i] = ((lm >> i) & 1u) ? phi : (R)phi0[c + nb.off(i)];
    if ((lc >> i) & 1u) {  // a cut neighbour: s ghost + (1 - s) phi, ghost = phi here
      const R sy = a.sfrac[c + nb.off(i)];
      val[i] = sy * phi + (R(1) - sy) * val[i];
    }
  }
  if (f & F_WALL) {
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (((lm | lc) >> i) & 1u) a.ghost[(i - 1) * a.nw + rec] = phi;
  }
  R gx, gy, gz, lap;
  cd_stencil(val, gx, gy, gz, lap);
  const Model<R> &m = a.m;
  R h[Q];
  h_equilibrium(m, h, phi, gx, gy, gz, lap);
  // g = g_eq(P0, u = 0) = w_i P0/T - K_i/2 with K_i = w_i (mu c_i.grad + c_i.F)/T.
  S he[Q], h_lo;
  enc_h_cell<S, R>(h, he, &h_lo);
  if constexpr (Codec<S>::narrow) h0base[Q * N + c] = h_lo;
  const R mu = m.mu_a * phi * (phi - R(1)) * (phi - R(0.5)) - m.mu_b * lap;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R wi = R(w_of(i));
    const R cg = R(cx_of(i)) * gx + R(cy_of(i)) * gy + R(cz_of(i)) * gz;
    const R cF = R(cx_of(i)) * m.Fx + R(cy_of(i)) * m.Fy + R(cz_of(i)) * m.Fz;
    const R K = wi * R(3) * (mu * cg + cF);
    const R gi = wi * R(3) * (R)P0 - R(0.5) * K;
    h0base[i * N + c] = he[i];
    st_g<S, R>(a.g[i] + c, i, gi);
    if (i != 0 && ((lm >> opp_of(i)) & 1u)) st_g<S, R>(wp0 + ((i - 1) * a.nw + rec), i, gi);
  }
}

}  // namespace pflb
