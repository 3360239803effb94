// pflb_async.cuh -- fused step kernel with TMA staging of the h
// populations (FP32 storage, nx a multiple of 4, nx >= 64).
//
// Same arithmetic as k_fused (update of one cell per thread per plane), but
// each plane's h data for the tile plus a one-cell halo, all 19 directions,
// is fetched global -> shared by one cp.async.bulk.tensor (a 4-D tensor map
// over (x, y, z, direction), box 40 x 10 x 1 x 19) two planes ahead of its
// use, completing on an mbarrier.  phi of a plane (tile plus ring) and the
// own cell's h then come from shared memory; only g, the cell flags and the
// wall data are read with ordinary loads, and g's loads are issued before
// the phi work of the iteration so their latency overlaps it.
//
// Tile: 32 x 8 columns (256 threads) marching a chunk of z planes.  The box
// starts at x0 - 4 (16-byte aligned because x0 and nx are multiples of 4)
// and y0 - 1; where it leaves the box of the lattice the TMA unit fills
// zeros, and the few halo cells that wrap periodically are then copied in
// from the other side with ordinary loads.
// Shared memory: 3 stages x 30 KB (+ phi ring), 2 blocks per SM.
#pragma once
#include <cuda.h>

#include "pflb_kernels.cuh"

namespace pflb {

constexpr int AB_X = 32, AB_Y = 8, AB_W = 40, AB_ROWS = AB_Y + 2, AB_STAGES = 3;
constexpr unsigned AB_STAGE_BYTES = Q * AB_ROWS * AB_W * 4u;  // bytes one box delivers
constexpr int AB_STAGE_FLOATS = 7616;  // stage stride: box rounded up to 128-byte alignment
constexpr int AB_PW = AB_X + 2, AB_PS = (AB_X + 2) * (AB_Y + 2);
// + 128: room to align the stage base to 128 bytes (TMA destination rule)
constexpr size_t AB_SMEM = (size_t)AB_STAGES * AB_STAGE_FLOATS * 4 + 3 * AB_PS * 4 + 64 + 128;

// Spin limit of an mbarrier wait (each try_wait may also suspend in hardware).
constexpr unsigned long long AB_WAIT_LIMIT = 1ull << 26;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait on an mbarrier phase: on running out of `limit` polls, raise
// the error flag and return false (the caller stops using what it waited for).
__device__ __forceinline__ bool bounded_wait(uint64_t *bar, unsigned parity, int *err,
                                             unsigned long long limit) {
  unsigned long long it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++it > limit) {
      if (err) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

// Wait for a stage of the staged step kernel.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, unsigned parity, int *err) {
  return bounded_wait(bar, parity, err, AB_WAIT_LIMIT);
}

// One TMA load of plane zw of the h buffer (tile + halo, 19 directions)
// into a stage, by a single thread that also announces the byte count.
__device__ __forceinline__ void stage_issue(const void *tmap, float *stage, uint64_t *bar,
                                            int x0, int y0, int zw) {
  mbar_arrive_expect_tx(bar, AB_STAGE_BYTES);
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(stage)),
      "l"(tmap), "r"(x0 - 4), "r"(y0 - 1), "r"(zw), "r"(0), "r"(smem_addr(bar))
      : "memory");
}

// Periodic halo of a staged plane: the box cells outside the lattice were
// filled with zeros; copy in the wrapped cells (only the columns 3..36 and
// rows 0..9 that phi and the own-cell reads use).  Tile-uniform condition.
__device__ __forceinline__ void stage_fix_wrap(const Args<float, float> &a, float *stage, int x0,
                                               int y0, int zw) {
  const int nx = a.nx, ny = a.ny;
  const int zoff = zw * nx * ny;
  // columns c with x = x0 - 4 + c outside [0, nx): c = 3 on the left edge,
  // c >= nx - x0 + 4 on the right edge
  const int cl = x0 == 0 ? 4 : 3;                    // first in-range column
  const int cr = min(37, nx - x0 + 4);               // first wrapped column on the right
  const int nbadc = (cl - 3) + (37 - cr);
  const int rlo = y0 == 0 ? 1 : 0;                   // first in-range row
  const int rhi = min(AB_ROWS, ny - y0 + 1);         // first wrapped row at the top
  const int nbadr = rlo + (AB_ROWS - rhi);
  const int ncol_items = Q * AB_ROWS * nbadc, nrow_items = Q * nbadr * 34;
  for (int k = threadIdx.x; k < ncol_items + nrow_items; k += blockDim.x) {
    int i, r, c;
    if (k < ncol_items) {
      i = k / (AB_ROWS * nbadc);
      const int rem = k - i * AB_ROWS * nbadc;
      r = rem / nbadc;
      const int j = rem - r * nbadc;
      c = j < cl - 3 ? 3 + j : cr + (j - (cl - 3));
    } else {
      const int kk = k - ncol_items;
      i = kk / (nbadr * 34);
      const int rem = kk - i * nbadr * 34;
      const int jr = rem / 34;
      c = 3 + (rem - jr * 34);
      r = jr < rlo ? jr : rhi + (jr - rlo);
    }
    const int x = ((x0 - 4 + c) % nx + nx) % nx;
    const int y = ((y0 - 1 + r) % ny + ny) % ny;
    stage[(i * AB_ROWS + r) * AB_W + c] = a.hin[i][zoff + y * nx + x];
  }
}

template <bool ODD, bool DIAG>
__global__ void __launch_bounds__(256, 2)
    k_fused_async(const __grid_constant__ Args<float, float> a,
                  const __grid_constant__ CUtensorMap tmap, int *err) {
  using R = float;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char *smem_raw = smem_dyn + ((128u - (smem_addr(smem_dyn) & 127u)) & 127u);
  float *stages = reinterpret_cast<float *>(smem_raw);
  R *sphi = reinterpret_cast<R *>(smem_raw + (size_t)AB_STAGES * AB_STAGE_FLOATS * 4);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)AB_STAGES * AB_STAGE_FLOATS * 4 +
                                                3 * AB_PS * sizeof(R));
  zero_next_diag(a);
  const int tid = threadIdx.x;
  const int tx = tid % AB_X, ty = tid / AB_X;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int sz = nx * ny;
  const int x0 = blockIdx.x * AB_X, y0 = blockIdx.y * AB_Y;
  const int zb = blockIdx.z * a.lz;
  const int ze = min(zb + a.lz, nz);
  const bool valid = (x0 + tx) < nx && (y0 + ty) < ny;
  const int gx = (x0 + tx) % nx, gy = (y0 + ty) % ny;
  const int col = gx + nx * gy;
  const bool wraps = x0 == 0 || x0 + AB_X + 1 > nx || y0 == 0 || y0 + AB_Y + 1 > ny;

  if (tid == 0) {
    for (int s = 0; s < AB_STAGES; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned phase_bits = 0;  // bit s: parity of the next completion of stage s
  bool ok = true;
  auto stage_of = [](int zu) { return ((zu % AB_STAGES) + AB_STAGES) % AB_STAGES; };
  auto zwrap = [nz](int zu) { return ((zu % nz) + nz) % nz; };
  auto issue = [&](int zu) {
    if (tid == 0) {
      const int s = stage_of(zu);
      stage_issue(&tmap, stages + s * AB_STAGE_FLOATS, &bars[s], x0, y0, zwrap(zu));
    }
  };
  auto wait = [&](int zu) {
    const int s = stage_of(zu);
    if (ok) ok = stage_wait(&bars[s], (phase_bits >> s) & 1u, err);
    phase_bits ^= 1u << s;
    if (wraps) {
      stage_fix_wrap(a, stages + s * AB_STAGE_FLOATS, x0, y0, zwrap(zu));
      __syncthreads();
    }
  };
  // phi of (unwrapped) plane zu over tile + ring, from its stage, into the ring
  auto plane_phi = [&](int zu) {
    const float *st = stages + stage_of(zu) * AB_STAGE_FLOATS;
    R *dst = sphi + (((zu % 3) + 3) % 3) * AB_PS;
    for (int p = tid; p < AB_PS; p += blockDim.x) {
      const int ry = p / AB_PW, rx = p - ry * AB_PW;
      const float *src = st + ry * AB_W + rx + 3;  // x = x0 - 1 + rx -> column rx + 3
      R s = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) s += src[i * AB_ROWS * AB_W];
      dst[p] = s;  // solid cells hold zero populations, so their phi is 0
    }
  };
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  if (DIAG) diag_block_zero(wacc);  // first use follows a barrier below
  issue(zb - 1);
  issue(zb);
  issue(zb + 1);
  wait(zb - 1);
  plane_phi(zb - 1);
  wait(zb);
  plane_phi(zb);
  // ring / stage slots of planes z - 1, z, z + 1 (both rings are indexed by
  // the unwrapped plane number modulo 3), advanced incrementally
  int sm = stage_of(zb - 1), s0 = stage_of(zb), sp = stage_of(zb + 1);
  const int o = (ty + 1) * AB_PW + tx + 1;
  for (int z = zb; z < ze; ++z) {
    // g loads of this cell first (A-A gather), so they are in flight during
    // the phi work below.
    const int c = col + sz * z;
    const uint8_t f = valid ? a.flags[c] : F_SOLID;
    const bool fluid = !(f & F_SOLID);
    Nbr nb;
    nb.init(gx, gy, z, nx, ny, nz);
    uint32_t lm = 0;
    int rec = 0;
    if (fluid && (f & F_WALL)) {
      rec = a.widx[c];
      lm = a.wmask[rec];
    }
    R g[Q];
    if (fluid) gather_g<float, R, ODD>(a, c, lm, rec, nb, g);
    wait(z + 1);
    plane_phi(z + 1);
    __syncthreads();
    // stage of plane z - 1 is free now: prefetch plane z + 2 into it
    if (z + 2 <= ze) {
      fence_async_shared();  // generic halo writes before the next async write
      issue(z + 2);
    }
    DiagAcc<R> acc;
    acc.zero();
    if (fluid) {
      const float *st = stages + s0 * AB_STAGE_FLOATS + (ty + 1) * AB_W + tx + 4;
      R h[Q], val[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) h[i] = st[i * AB_ROWS * AB_W];
      const R *p0 = sphi + s0 * AB_PS, *pm = sphi + sm * AB_PS, *pp = sphi + sp * AB_PS;
      const R phi = p0[o];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const R *pl = cz_of(i) == 0 ? p0 : (cz_of(i) > 0 ? pp : pm);
        val[i] = pl[o + cy_of(i) * AB_PW + cx_of(i)];
      }
      finish_cell<float, R, ODD, MODE_STEP, DIAG>(a, gx, gy, z, c, f, lm, rec, nb, h, g, phi, val, acc);
    }
    if (DIAG) diag_warp_add(wacc[tid >> 5], acc);
    __syncthreads();
    const int t = sm;
    sm = s0;
    s0 = sp;
    sp = t;
  }
  // Every issued stage (planes zb - 1 .. ze) has been waited for above, so
  // no copy into shared memory is in flight when the block exits.
  if (DIAG) diag_block_flush(a.diag, wacc);
}

}  // namespace pflb
