// pflb_pipe.cuh -- fused step kernel with asynchronous staging of the next
// planes' populations in 16-byte chunks (8-byte chunks at 16-bit storage
// when nx is not a multiple of 8; any storage type, periodic x, nx a
// multiple of 4).
//
// The step is k_fused's (arXiv 2512.01032, Sec. II and Sec. III A): one
// thread per (x, y) column of a 32 x 4 tile marching a chunk of z planes,
// phi recomputed from h for the tile plus a one-cell ring, so no phi field
// goes to HBM.  What differs is how the populations reach the threads.
// k_fused loads each value when it needs it and waits for DRAM on every
// plane.  Here the block copies whole rows into shared memory with
// cp.async.cg (16 bytes per copy, through L2 only) one iteration before they
// are used:
//
//   iteration z:  wait for the copies issued in iteration z - 1; barrier;
//                 phi of plane z + 1 from its staged h into the phi ring;
//                 each thread takes its cell's h and g of plane z from
//                 shared memory into registers; barrier;
//                 issue the copies of h of plane z + 2, g of plane z + 1 and
//                 the flags of plane z + 3 into the buffers just read;
//                 update of plane z (collision, streaming stores).
//
// Staged rows span x0 - V .. x0 + 32 + V (V values per 16-byte chunk), so
// the ring cells' h and the A-A gather sources of odd steps (shifted by one
// cell in x) come from the same aligned chunks; because chunks are aligned
// and nx is a multiple of V, a chunk never straddles the periodic seam and
// wraps as a whole.  Rows and planes wrap individually.  Chunks whose cells
// are all solid are not copied, using flag words staged one iteration
// earlier still.  Wall nodes (a few percent of the cells; their update
// reads wall records, ghosts and wall populations) are taken out of the
// march: each block updates the wall nodes among its cells after its last
// plane, from a per-block list, while the SM's other blocks keep marching
// (the wall nodes' chains of dependent loads held whole blocks at the
// plane barriers when they were updated in the march).  16-bit storage
// stages the stored values and decodes them when they are read.
//
// Shared memory per block (FP32): h 2 planes x 19 x 6 rows x 40, g 19 x 4
// rows x 40, flags 4 planes x 6 x 10 words, phi 4 planes x 34 x 6: 54 KB,
// four blocks per SM.
//
// The collision is collide_pairs (the even/odd split of each opposite
// pair); the per-cell arithmetic is otherwise finish_cell's.
#pragma once
#include "pflb_async.cuh"
#include "pflb_kernels.cuh"

namespace pflb {

constexpr int PP_BX = 32, PP_BY = 4, PP_NT = PP_BX * PP_BY;
constexpr int PP_PW = PP_BX + 2, PP_PS = (PP_BX + 2) * (PP_BY + 2);
constexpr int PP_NR = 2 * PP_PW + 2 * PP_BY;  // ring cells around the tile
constexpr int PP_ROWS = PP_BY + 2;            // staged h rows: y0 - 1 .. y0 + BY
constexpr int PP_FW = (PP_BX + 8) / 4;        // flag words per staged row (x0 - 4 .. x0 + 36)
#ifndef PFLB_PIPE_MIN_BLOCKS
#define PFLB_PIPE_MIN_BLOCKS 4
#endif

// CB: bytes per staged chunk, 16 (cp.async.cg) or 8 (cp.async.ca; 16-bit
// storage with nx = 4 mod 8, whose odd rows start 8 bytes off a 16-byte
// boundary).
template <class S, class R, int CB = 16>
struct alignas(16) PipeSmem {
  static constexpr int V = CB / (int)sizeof(S);  // values per chunk
  static constexpr int W = PP_BX + 2 * V;        // staged row: x0 - V .. x0 + 32 + V
  static constexpr int NCH = W / V;              // chunks per staged row
  static constexpr int HS = h_slots<S>();        // 19, or 20 with the rest remainder
  S h[2][HS][PP_ROWS][W];   // h of planes z + 1 (phi) and z + 2 (in flight), slot = plane & 1
  S g[Q][PP_BY][W];         // g arriving at the cells of the next plane to update
  R phi[4][PP_PS];          // phi ring, slot = unwrapped plane & 3
  uint32_t fl[4][PP_ROWS][PP_FW];  // flag words, x0 - 4 .. x0 + 36, slot = plane & 3
};

__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
template <int CB>
__device__ __forceinline__ void cp_async_chunk(void *dst, const void *src) {
  if constexpr (CB == 16)
    cp_async_16(dst, src);
  else
    cp_async_8(dst, src);
}
__device__ __forceinline__ void cp_async_4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ uint8_t flag_byte(const uint32_t (*fl)[PP_FW], int row, int dx) {
  // dx: x offset from x0, in [-4, 36)
  return (uint8_t)(fl[row][(dx + 4) >> 2] >> (8 * ((dx + 4) & 3)));
}
__device__ __forceinline__ bool all_solid(uint32_t w) {
  return (w & 0x01010101u) == 0x01010101u;  // bit 0 (F_SOLID) of all four cells
}
// True if the flag words overlapping chunk ch of a staged row (x offsets
// ch V - V .. ch V - 1 from x0) say all their cells are solid; cells of the
// chunk outside x0 - 4 .. x0 + 36 are never read.
template <int V>
__device__ __forceinline__ bool chunk_solid(const uint32_t *flrow, int ch) {
  const int dx0 = ch * V - V, dx1 = dx0 + V;
  const int w0 = ((dx0 > -4 ? dx0 : -4) + 4) >> 2;
  const int w1 = ((dx1 < 36 ? dx1 : 36) + 7) >> 2;
  bool solid = true;
#pragma unroll
  for (int k = 0; k < (V + 7) / 4; ++k)
    if (w0 + k < w1) solid = solid && all_solid(flrow[w0 + k]);
  return solid;
}

// Update of wall node rec of lattice a (k_cell's per-cell step: populations,
// wall records and wall populations loaded directly; the neighbours' phi from
// the field the pipelined march wrote for exactly these reads; solid
// neighbours replaced by the lagged ghosts).
__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// A wall node's update is a chain of dependent loads (record -> cell ->
// link mask -> sources).  With only a few warps per SM nothing hides it, so
// every line the update will read is prefetched into L1 first, in two
// rounds: what the record indexes, then what the cell indexes.
template <class S, class R, bool ODD>
__device__ __forceinline__ void wall_prefetch(const Args<S, R> &a, int rec) {
  const int nw = a.nw;
  prefetch_l1(a.wcell + rec);
  prefetch_l1(a.wmask + rec);
#pragma unroll
  for (int k = 0; k < 5; ++k) prefetch_l1(a.wgeo + (k * nw + rec));
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    prefetch_l1(a.ghost + (i * nw + rec));
    prefetch_l1(a.wp_rd + (i * nw + rec));
  }
  const int c = a.wcell[rec];
  const int x = c % a.nx, y = (c / a.nx) % a.ny, z = c / (a.nx * a.ny);
  Nbr nb;
  nb.init(x, y, z, a.nx, a.ny, a.nz);
  prefetch_l1(a.flags + c);
  prefetch_l1(a.widx + c);
#pragma unroll
  for (int i = 0; i < h_slots<S>(); ++i) prefetch_l1(a.hin[i] + c);
#pragma unroll
  for (int i = 1; i < Q; ++i) prefetch_l1(a.phi_w + (c + nb.off(i)));
#pragma unroll
  for (int k = 0; k < Q; ++k)
    prefetch_l1(ODD ? a.g[opp_of(k)] + (c + nb.off(opp_of(k))) : a.g[k] + c);
}

template <class S, class R, bool ODD, bool DIAG>
__device__ __forceinline__ void wall_node(const Args<S, R> &a, int rec, DiagAcc<R> &acc) {
  wall_prefetch<S, R, ODD>(a, rec);
  const int c = a.wcell[rec];
  const uint8_t f = a.flags[c];
  const int x = c % a.nx, y = (c / a.nx) % a.ny, z = c / (a.nx * a.ny);
  Nbr nb;
  nb.init(x, y, z, a.nx, a.ny, a.nz);
  R h[Q], val[Q];
  ld_h_cell<S, R>(a.hin, c, h);
  R phi = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) phi += h[i];
  // the neighbours' phi from the field the march wrote in this launch
  // (plain loads through the written pointer: never the read-only path)
#pragma unroll
  for (int i = 1; i < Q; ++i) val[i] = a.phi_w[c + nb.off(i)];
  update_cell<S, R, ODD, MODE_STEP, DIAG, false, COLL_X2>(a, x, y, z, c, f, h, phi, val, acc);
}

// One tile column (x0, y0) over planes [zb, ze) of lattice a, by the whole
// block (PP_NT threads), with shared memory sm and the warp slots wacc of
// the diagnostics (flushed into a.diag at the end).  Wall records
// a.wl[w0 .. w1) are the wall nodes among the march's cells: the block
// updates them after the march (wall_node), from the phi of the cells
// around them, which it writes to the phi field as it sums them (own and
// ring cells of every plane it sums).  A block reads back only values it
// wrote itself in this launch, and a cell summed by two blocks gets the
// same bits from both (same staged h, same order), so the duplicate writes
// are benign.  Without per-block lists (a.wl_start null) the march writes the
// phi of its own cells in [zb, ze) that wall nodes read, for k_wall after
// the launch.  Every thread returns with no copy in flight; the caller
// separates two marches that reuse sm by a barrier.
template <class S, class R, bool ODD, bool DIAG, bool FORCE, int CB = 16>
__device__ __forceinline__ void pipe_march(const Args<S, R> &a, int x0, int y0, int zb, int ze,
                                           PipeSmem<S, R, CB> &sm, R (*wacc)[32], int w0 = 0,
                                           int w1 = 0) {
  using SM = PipeSmem<S, R, CB>;
  constexpr int V = SM::V, NCH = SM::NCH, HS = SM::HS;
  static_assert(F_SOLID == 1, "all_solid tests bit 0");
  const int tid = threadIdx.x, tx = tid % PP_BX, ty = tid / PP_BX;
  const int nx = a.nx, ny = a.ny, nz = a.nz, sz = nx * ny;
  // A column beyond a ragged lattice edge still sums the cell it wraps to:
  // that is the periodic neighbour the last valid column needs.
  const bool valid = (x0 + tx) < nx && (y0 + ty) < ny;
  const int cx0 = (x0 + tx) % nx, cy0 = (y0 + ty) % ny;
  const int col = cx0 + nx * cy0;
  // Side jobs (a ring cell's phi, staging units) go to the first `count`
  // threads in thread order, so that a warp's copies and ring reads are
  // contiguous (measured faster than spreading them evenly over the warps);
  // job_of returns the job of this thread among `count`, or -1.
  auto job_of = [&](int count) { return tid < count ? tid : -1; };
  const int rj = job_of(PP_NR);
  const bool ring = rj >= 0;
  int rx = 0, ry = 0;
  if (ring) {
    if (rj < PP_PW) {
      rx = rj;
      ry = 0;
    } else if (rj < 2 * PP_PW) {
      rx = rj - PP_PW;
      ry = PP_BY + 1;
    } else {
      const int k = rj - 2 * PP_PW;
      rx = (k & 1) ? PP_BX + 1 : 0;
      ry = 1 + (k >> 1);
    }
  }
  // phi field writes: 2 = own and ring cells of every summed plane (this
  // block's wall nodes read them), 1 = own cells of [zb, ze) (k_wall or
  // k_batch_wall reads them), 0 = none (block-uniform)
  const int phimode = w1 > w0 ? 2 : (a.wl_start ? 0 : 1);
  // Plane wrap by additions: the planes touched lie within a few of [0, nz).
  auto wrapz = [nz](int zu) {
    while (zu < 0) zu += nz;
    while (zu >= nz) zu -= nz;
    return zu;
  };
  auto wrap = [](int v, int n) { return ((v % n) + n) % n; };

  // Staging units, fixed for the whole march, so their periodic x and y
  // wraps (integer divisions) are computed once: a unit is one staged row
  // chunk (row r, chunk ch) and one half of the population slots.
  constexpr int HU = 2 * PP_ROWS * NCH, GU = 2 * PP_BY * NCH;
  constexpr int HPT = (HU + PP_NT - 1) / PP_NT, GPT = (GU + PP_NT - 1) / PP_NT;
  int h_rc[HPT], h_off[HPT];     // (half << 16 | r << 8 | ch), in-plane offset; -1: none
  int g_rc[GPT], g_off[GPT][3];  // offsets of the chunk in rows y0 + r - 1, y0 + r, y0 + r + 1
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int u = HU <= PP_NT ? job_of(HU) : tid + k * PP_NT;
    h_rc[k] = -1;
    h_off[k] = 0;
    if (u >= 0 && u < HU) {
      const int half = u >= HU / 2, v = u - half * (HU / 2);
      const int r = v / NCH, ch = v - r * NCH;
      h_rc[k] = half << 16 | r << 8 | ch;
      h_off[k] = wrap(x0 - V + ch * V, nx) + nx * wrap(y0 - 1 + r, ny);
    }
  }
#pragma unroll
  for (int k = 0; k < GPT; ++k) {
    const int u = GU <= PP_NT ? job_of(GU) : tid + k * PP_NT;
    g_rc[k] = -1;
    g_off[k][0] = g_off[k][1] = g_off[k][2] = 0;
    if (u >= 0 && u < GU) {
      const int half = u >= GU / 2, v = u - half * (GU / 2);
      const int r = v / NCH, ch = v - r * NCH;
      g_rc[k] = half << 16 | r << 8 | ch;
      const int xs = wrap(x0 - V + ch * V, nx);
#pragma unroll
      for (int d = 0; d < 3; ++d) g_off[k][d] = xs + nx * wrap(y0 + r - 1 + d, ny);
    }
  }
  const int fj = job_of(PP_ROWS * PP_FW);  // flag word fj % 10 of row fj / 10
  int fl_off = -1;
  if (fj >= 0) fl_off = wrap(x0 - 4 + 4 * (fj % PP_FW), nx) + nx * wrap(y0 - 1 + fj / PP_FW, ny);

  // Flag words of plane zu: 6 rows x 10 words, one copy per thread.
  auto stage_flags = [&](int zu) {
    if (fl_off >= 0)
      cp_async_4(&sm.fl[zu & 3][fj / PP_FW][fj % PP_FW], a.flags + (fl_off + sz * wrapz(zu)));
  };
  // h of plane zu into slot zu & 1: 6 rows x NCH chunks x HS slots, the
  // slots split into two halves over the block's two thread halves.
  auto stage_h = [&](int zu, bool skip_solid) {
    const int zoff = sz * wrapz(zu);
    const uint32_t (*fl)[PP_FW] = sm.fl[zu & 3];
    S(*dst)[PP_ROWS][SM::W] = sm.h[zu & 1];
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
      if (h_rc[k] < 0) continue;
      const int half = h_rc[k] >> 16, r = (h_rc[k] >> 8) & 0xff, ch = h_rc[k] & 0xff;
      if (skip_solid && chunk_solid<V>(fl[r], ch)) continue;
      const int cell = h_off[k] + zoff;
      if (!half) {
#pragma unroll
        for (int i = 0; i < 10; ++i) cp_async_chunk<CB>(&dst[i][r][ch * V], a.hin[i] + cell);
      } else {
#pragma unroll
        for (int i = 10; i < HS; ++i) cp_async_chunk<CB>(&dst[i][r][ch * V], a.hin[i] + cell);
      }
    }
  };
  // g arriving at the cells of plane zu: for direction k, row r holds the
  // source row of tile row r (A-A: slot k of the own cells on even steps,
  // slot opp(k) of x - c_k on odd steps), in the chunks that hold the
  // tile's sources.  Sources across a solid link are replaced from the wall
  // populations at the update.
  auto stage_g = [&](int zu) {
    const int z = wrapz(zu);
    const uint32_t (*fl)[PP_FW] = sm.fl[zu & 3];
#pragma unroll
    for (int u = 0; u < GPT; ++u) {
      if (g_rc[u] < 0) continue;
      const int half = g_rc[u] >> 16, r = (g_rc[u] >> 8) & 0xff, ch = g_rc[u] & 0xff;
      const int k0 = half ? 10 : 0, k1 = half ? Q : 10;
      if constexpr (!ODD) {
        if (ch == 0 || ch == NCH - 1) continue;  // own cells only
        if (chunk_solid<V>(fl[r + 1], ch)) continue;
        const int cell = g_off[u][1] + sz * z;
#pragma unroll
        for (int k = 0; k < Q; ++k)
          if (k >= k0 && k < k1) cp_async_chunk<CB>(&sm.g[k][r][ch * V], a.g[k] + cell);
      } else {
        const int zo[3] = {sz * wrapz(zu - 1), sz * z, sz * wrapz(zu + 1)};
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          if (k < k0 || k >= k1) continue;
          const int cxk = cx_of(k), cyk = cy_of(k), czk = cz_of(k);
          const int lo = (V - (cxk > 0 ? cxk : 0)) / V;
          const int hi = (V + PP_BX - 1 - (cxk < 0 ? cxk : 0)) / V;
          if (ch < lo || ch > hi) continue;
          // source row y - c_k and plane z - c_k
          cp_async_chunk<CB>(&sm.g[k][r][ch * V],
                             a.g[opp_of(k)] + (g_off[u][1 - cyk] + zo[1 - czk]));
        }
      }
    }
  };
  // phi of plane zu (own column and ring cell) into ring slot zu & 3; a
  // solid cell's phi is 0
  // staged h of one cell, decoded (the 16-bit rest population is high part
  // plus remainder), and its sum in the order cell_phi uses
  auto cell_h = [&](const S (*st)[PP_ROWS][SM::W], int row, int idx, R h[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = dec_pop<S, R>(st[i][row][idx], i);
    if constexpr (HS > Q) h[0] += dec_pop<S, R>(st[Q][row][idx], 0);
  };
  auto staged_phi = [&](const S (*st)[PP_ROWS][SM::W], int row, int idx) {
    R h[Q];
    cell_h(st, row, idx, h);
    R v = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) v += h[i];
    return v;
  };
  const int rcol = wrap(x0 - 1 + rx, nx) + nx * wrap(y0 - 1 + ry, ny);
  auto phi_plane = [&](int zu) {
    const S(*st)[PP_ROWS][SM::W] = sm.h[zu & 1];
    const uint32_t (*fl)[PP_FW] = sm.fl[zu & 3];
    R *dst = sm.phi[zu & 3];
    const uint8_t f = flag_byte(fl, ty + 1, tx);
    const R v = (f & F_SOLID) ? R(0) : staged_phi(st, ty + 1, V + tx);
    dst[(ty + 1) * PP_PW + tx + 1] = v;
    // (a column beyond a ragged edge sums the cell it wraps to, which a
    // wall node of the last valid column reads)
    if ((f & F_NEAR) && (phimode == 2 || (phimode == 1 && valid && zu >= zb && zu < ze)))
      a.phi_w[col + sz * wrapz(zu)] = v;
    if (ring) {
      const uint8_t fr = flag_byte(fl, ry, rx - 1);
      const R vr = (fr & F_SOLID) ? R(0) : staged_phi(st, ry, V - 1 + rx);
      dst[ry * PP_PW + rx] = vr;
      if (phimode == 2 && (fr & F_NEAR)) a.phi_w[rcol + sz * wrapz(zu)] = vr;
    }
  };

  DiagAcc<R> tot;
  tot.zero();
  if (DIAG) diag_block_zero(wacc);  // first use follows the loop's barriers

  // Prologue: flags of planes zb - 1 .. zb + 2 and h of zb - 1, zb (all
  // chunks), then phi of zb - 1 and zb; then h of zb + 1 (into the slot of
  // zb - 1) and g of zb.
  for (int zu = zb - 1; zu <= zb + 2; ++zu) stage_flags(zu);
  stage_h(zb - 1, false);
  stage_h(zb, false);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  phi_plane(zb - 1);
  phi_plane(zb);
  __syncthreads();  // slot of zb - 1 read before it is refilled
  stage_h(zb + 1, true);
  stage_g(zb);
  cp_async_commit();

  const int o = (ty + 1) * PP_PW + tx + 1;
  for (int z = zb; z < ze; ++z) {
    cp_async_wait_all();
    __syncthreads();  // staged h(z + 1), g(z), flags(z + 2) visible to all
    phi_plane(z + 1);
    const int c = col + sz * z;
    const uint8_t f = flag_byte(sm.fl[z & 3], ty + 1, tx);
    const bool fluid = valid && !(f & (F_SOLID | F_WALL));  // wall nodes: after the march
    R h[Q], g[Q];
    if (fluid) {
      cell_h(sm.h[z & 1], ty + 1, V + tx, h);
#pragma unroll
      for (int k = 0; k < Q; ++k)
        g[k] = dec_pop<S, R>(sm.g[k][ty][V + tx - (ODD ? cx_of(k) : 0)], k);
    }
    __syncthreads();  // phi ring complete; h slot z & 1 and the g buffer are free
    if (z + 2 <= ze) stage_h(z + 2, true);
    if (z + 1 < ze) stage_g(z + 1);
    if (z + 3 <= ze) stage_flags(z + 3);
    cp_async_commit();
    if (fluid) {
      Nbr nb;
      nb.init(cx0, cy0, z, nx, ny, nz);
      const R *p0 = sm.phi[z & 3], *pm = sm.phi[(z - 1) & 3], *pp = sm.phi[(z + 1) & 3];
      R val[Q];
      const R phi = p0[o];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const R *pl = cz_of(i) == 0 ? p0 : (cz_of(i) > 0 ? pp : pm);
        val[i] = pl[o + cy_of(i) * PP_PW + cx_of(i)];
      }
      DiagAcc<R> acc;
      acc.zero();
      // a bulk cell: no wall flag, no solid link
      finish_cell<S, R, ODD, MODE_STEP, DIAG, false, FORCE ? COLL_X2 : COLL_X2_NOF>(
          a, cx0, cy0, z, c, 0, 0u, 0, nb, h, g, phi, val, acc);
      if (DIAG) {
#pragma unroll
        for (int k = 0; k < D_UMAX; ++k) tot.v[k] += acc.v[k];
        tot.umax = tot.umax > acc.umax ? tot.umax : acc.umax;
        tot.front = tot.front > acc.front ? tot.front : acc.front;
        tot.rear = tot.rear > acc.rear ? tot.rear : acc.rear;
      }
    }
  }
  cp_async_wait_all();  // nothing is in flight at exit
  if (w1 > w0) {  // this block's wall nodes
    __syncthreads();  // the block's phi field writes are visible to all its threads
    for (int k = w0 + tid; k < w1; k += PP_NT) {
      DiagAcc<R> acc;
      acc.zero();
      wall_node<S, R, ODD, DIAG>(a, a.wl[k], acc);
      if (DIAG) {
#pragma unroll
        for (int q = 0; q < D_UMAX; ++q) tot.v[q] += acc.v[q];
        tot.umax = tot.umax > acc.umax ? tot.umax : acc.umax;
        tot.front = tot.front > acc.front ? tot.front : acc.front;
        tot.rear = tot.rear > acc.rear ? tot.rear : acc.rear;
      }
    }
  }
  if (DIAG) {
    diag_warp_add(wacc[tid >> 5], tot);
    diag_block_flush(a.diag, wacc);
  }
}

// One lattice: a grid of (tile column, chunk of lz planes) blocks.  FORCE
// = false is the variant for a lattice without body force; CB the staged
// chunk size (PipeSmem).
template <class S, class R, bool ODD, bool DIAG, bool FORCE, int CB = 16>
__global__ void __launch_bounds__(PP_NT, PFLB_PIPE_MIN_BLOCKS)
    k_pipe(const __grid_constant__ Args<S, R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  zero_next_diag(a);
  // z chunks alternate from both ends of the lattice (0, n-1, 1, n-2, ...)
  // so that the chunks next to the bounding walls, whose blocks carry the
  // most wall nodes, are dispatched early instead of last
  const int nch = gridDim.z, bz = blockIdx.z;
  const int zb = ((bz & 1) ? nch - 1 - (bz >> 1) : (bz >> 1)) * a.lz;
  int w0 = 0, w1 = 0;
  if (a.wl_start) {
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * bz);
    w0 = a.wl_start[b];
    w1 = a.wl_start[b + 1];
  }
  pipe_march<S, R, ODD, DIAG, FORCE, CB>(a, blockIdx.x * PP_BX, blockIdx.y * PP_BY, zb,
                                         min(zb + a.lz, a.nz),
                                         *reinterpret_cast<PipeSmem<S, R, CB> *>(smem_raw),
                                         wacc, w0, w1);
}

// Many lattices: a persistent grid pulls work items (lattice, x0, y0, z0)
// from an atomic counter, copies the lattice's step descriptor for its A-A
// parity at this batch step ((par0[l] + t) & 1) into shared memory and
// marches the item's tile column over LZ planes.  The first item of each
// lattice zeroes its next diagnostic accumulator.
// One launch marches one parity (ODD): the items of lattices at the other
// parity are skipped, and the host launches the second parity only when a
// lattice of the batch is at it.  With both marches in one kernel the step
// descriptor's fields in shared memory cost registers that k_pipe's
// constant-bank parameters do not (168 per thread, three blocks per SM);
// with one, the march fits k_pipe's 128 registers and four blocks per SM
// without spilling.  CB: the staged chunk size of the items' lattices (the
// host builds one work list per chunk size).
template <class S, class R, bool ODD, bool DIAG, int CB = 16>
__global__ void __launch_bounds__(PP_NT, 4)
    k_batch_pipe(const Args<S, R> *__restrict__ descs, const int *__restrict__ par0,
                 const int4 *__restrict__ items, int nitems, int *counter, const int *bstep,
                 int LZ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PipeSmem<S, R, CB> &sm = *reinterpret_cast<PipeSmem<S, R, CB> *>(smem_raw);
  Args<S, R> *sa = reinterpret_cast<Args<S, R> *>(smem_raw + sizeof(PipeSmem<S, R, CB>));
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const int t = *bstep;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = s_item;
    if (idx >= nitems) break;
    const int4 it = items[idx];
    const int p = (par0[it.x] + t) & 1;
    if (p != (ODD ? 1 : 0)) {  // the other parity's launch marches this item
      __syncthreads();         // s_item is read before it is replaced
      continue;
    }
    const int *src = reinterpret_cast<const int *>(descs + 2 * it.x + p);
    int *dst = reinterpret_cast<int *>(sa);
    for (int k = tid; k < (int)(sizeof(Args<S, R>) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    const Args<S, R> &a = *sa;
    if (DIAG && it.y == 0 && it.z == 0 && it.w == 0 && tid < 32 && a.diag_zero)
      a.diag_zero[tid] = 0.0;
    const int ze = min(it.w + LZ, a.nz);
    pipe_march<S, R, ODD, DIAG, true, CB>(a, it.y, it.z, it.w, ze, sm, wacc);
    __syncthreads();  // shared descriptor and staging buffers are reused by the next item
  }
}

// Wall nodes of a step whose bulk cells k_pipe updates, one thread per wall
// node, launched after k_pipe on the same stream (used when the per-block
// wall lists are not built for the launch shape in effect).  The two
// kernels touch disjoint data: under A-A every g slot is read and written
// by one cell, h is pushed from each cell into slots no other cell writes,
// and only wall nodes use the ghosts and wall populations.
template <class S, class R, bool ODD, bool DIAG>
__global__ void __launch_bounds__(128, 4) k_wall(const __grid_constant__ Args<S, R> a) {
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  if (DIAG) {
    diag_block_zero(wacc);
    __syncthreads();
  }
  const int rec = blockIdx.x * blockDim.x + threadIdx.x;
  DiagAcc<R> acc;
  acc.zero();
  if (rec < a.nw) wall_node<S, R, ODD, DIAG>(a, rec, acc);
  if (DIAG) {
    diag_warp_add(wacc[threadIdx.x >> 5], acc);
    diag_block_flush(a.diag, wacc);
  }
}

// Wall nodes of the batch's pipelined lattices: block b takes item
// (lattice, first record) = witems[b] and its 128 records, for the
// lattice's parity at this batch step.
template <class S, class R, bool DIAG>
__global__ void __launch_bounds__(128)
    k_batch_wall(const Args<S, R> *__restrict__ descs, const int *__restrict__ par0,
                 const int2 *__restrict__ witems, const int *bstep) {
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  __shared__ __align__(16) unsigned char sa_raw[sizeof(Args<S, R>)];
  Args<S, R> *sa = reinterpret_cast<Args<S, R> *>(sa_raw);
  const int2 it = witems[blockIdx.x];
  const int p = (par0[it.x] + *bstep) & 1;
  const int *src = reinterpret_cast<const int *>(descs + 2 * it.x + p);
  int *dst = reinterpret_cast<int *>(sa);
  for (int k = threadIdx.x; k < (int)(sizeof(Args<S, R>) / 4); k += blockDim.x) dst[k] = src[k];
  if (DIAG) diag_block_zero(wacc);
  __syncthreads();
  const Args<S, R> &a = *sa;
  const int rec = it.y + threadIdx.x;
  DiagAcc<R> acc;
  acc.zero();
  if (rec < a.nw) {
    if (p)
      wall_node<S, R, true, DIAG>(a, rec, acc);
    else
      wall_node<S, R, false, DIAG>(a, rec, acc);
  }
  if (DIAG) {
    diag_warp_add(wacc[threadIdx.x >> 5], acc);
    diag_block_flush(a.diag, wacc);
  }
}

}  // namespace pflb
