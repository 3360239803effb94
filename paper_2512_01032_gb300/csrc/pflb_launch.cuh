// pflb_launch.cuh -- per-precision kernel launchers (included by one
// translation unit per storage type).
#pragma once
#include <cstring>
#include <type_traits>

#include "pflb_async.cuh"
#include "pflb_batch.cuh"
#include "pflb_internal.h"
#include "pflb_kernels.cuh"
#include "pflb_pipe.cuh"

namespace pflb {

template <class R>
static Model<R> make_model(const pflb_params &p) {
  const double T = 1.0 / 3.0;
  Model<R> m;
  m.sigma = (R)p.sigma;
  m.W = (R)p.W;
  m.M = (R)p.M;
  m.rho_L = (R)p.rho_L;
  m.rho_dif = (R)(p.rho_H - p.rho_L);
  m.tau_H = (R)(p.nu_H / T + 0.5);
  m.tau_L = (R)(p.nu_L / T + 0.5);
  m.Fx = (R)p.Fex[0];
  m.Fy = (R)p.Fex[1];
  m.Fz = (R)p.Fex[2];
  m.gamma = (R)p.gamma;
  m.phi_M = (R)p.phi_M;
  m.phi_m = (R)p.phi_m;
  m.inv_D = (R)(1.0 / p.D);
  m.eps = (R)p.eps;
  m.blend = (R)p.blend;
  m.band_lo = (R)p.band_lo;
  m.band_hi = (R)p.band_hi;
  m.F_tilde = (R)p.F_tilde;
  m.inv_F_width = (R)(1.0 / p.F_width);
  m.inv_tau_phi = (R)(1.0 / (p.M / T + 0.5));
  m.theta_coef = (R)(p.M / (T * p.W));
  m.mu_a = (R)(48.0 * p.sigma / p.W);
  m.mu_b = (R)(1.5 * p.sigma * p.W);
  m.two_over_W = (R)(2.0 / p.W);
  m.F_mode = p.F_mode;
  m.mobility_corr = p.mobility_corr;
  m.free_slip = p.free_slip;
  return m;
}

template <class S, class R>
static Args<S, R> make_args(Lattice &L) {
  Args<S, R> a;
  a.nx = L.nx; a.ny = L.ny; a.nz = L.nz; a.lz = L.lz;
  a.N = (int)L.N;
  a.nw = L.nw;
  const int rd = (int)(L.step & 1);
  for (int i = 0; i < Q + 1; ++i) {
    const bool have = i < h_slots<S>();
    a.hin[i] = have ? (const S *)L.h[rd] + (size_t)i * L.N : nullptr;
    a.hout[i] = have ? (S *)L.h[rd ^ 1] + (size_t)i * L.N : nullptr;
  }
  for (int i = 0; i < Q; ++i) a.g[i] = (S *)L.g + (size_t)i * L.N;
  a.flags = L.flags;
  a.widx = L.widx;
  a.wmask = L.wmask;
  a.wcell = L.wcell;
  a.wgeo = (const R *)L.wgeo;
  a.wcut = L.wcut;
  a.sfrac = (const R *)L.sfrac;
  a.ghost = (R *)L.ghost;
  a.wp_rd = (const S *)L.wp[rd];
  a.wp_wr = (S *)L.wp[rd ^ 1];
  a.phi = (const R *)L.phi;
  a.phi_w = (R *)L.phi;
  a.m = make_model<R>(L.p);
  a.diag = nullptr;
  a.diag_zero = nullptr;
  for (int k = 0; k < 6; ++k) a.reg[k] = L.reg[k];
  a.out = nullptr;
  a.bcm = L.bc_on ? (R *)L.bcm : nullptr;
  a.nbc = 2 * L.ny * L.nz;
  a.wl = nullptr;  // set by the pipelined launch when its lists are current
  a.wl_start = nullptr;
  return a;
}

// Boundary states of the open x planes for the state the next launch reads.
template <class S, class R>
static cudaError_t launch_xbc(Lattice &L, const Args<S, R> &a) {
  if (!L.bc_on) return cudaSuccess;
  const XbcSpec sp = xbc_spec(L, L.step);
  const int n = 2 * L.ny * L.nz, T = 128;
  if (L.step & 1)
    k_xbc<S, R, true><<<(n + T - 1) / T, T, 0, L.stream>>>(a, sp);
  else
    k_xbc<S, R, false><<<(n + T - 1) / T, T, 0, L.stream>>>(a, sp);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t set_model(Lattice &) { return cudaSuccess; }

template <class S, class R>
int max_block_threads() { return 256; }

template <class S, class R>
cudaError_t launch_init(Lattice &L, const double *d_phi0, double P0) {
  L.step = 0;
  L.ndiag = 0;
  L.last_diag_step = -1;
  Args<S, R> a = make_args<S, R>(L);
  cudaError_t e = cudaMemsetAsync(L.diag, 0, 96 * sizeof(double), L.stream);
  if (e != cudaSuccess) return e;
  const int T = 256;
  const long long B = (L.N + T - 1) / T;
  k_init<S, R><<<(unsigned)B, T, 0, L.stream>>>(a, d_phi0, P0, (S *)L.h[0], (S *)L.wp[0]);
  return cudaGetLastError();
}

// The staged kernel (FP32, x extent a multiple of 4 and at least 64).
inline bool async_eligible(const Lattice &L) {
  return L.kernel == PFLB_KERNEL_FUSED_TMA && L.p.storage == PFLB_STORAGE_FP32 && L.tma_ok &&
         !L.bc_on;
}

template <bool ODD, bool DIAG>
static cudaError_t async_attrs() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_async<ODD, DIAG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AB_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fused_async<ODD, DIAG>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

template <bool ODD, bool DIAG>
static cudaError_t launch_async_t(Lattice &L, Args<float, float> &a) {
  cudaError_t e0 = async_attrs<ODD, DIAG>();
  if (e0 != cudaSuccess) return e0;
  dim3 grid((L.nx + AB_X - 1) / AB_X, (L.ny + AB_Y - 1) / AB_Y, (L.nz + L.lz - 1) / L.lz);
  k_fused_async<ODD, DIAG><<<grid, AB_X * AB_Y, AB_SMEM, L.stream>>>(a, L.tmap[L.step & 1], L.err);
  return cudaGetLastError();
}

// The pipelined kernel (periodic x; nx a multiple of 4).
template <class S>
constexpr bool pipe_storage() {
  return true;
}
inline bool pipe_eligible(const Lattice &L) { return pipe_kernel_runs(L); }

// Dynamic shared memory above 48 KB is opted into once per device.
template <class S, class R, bool ODD, bool DIAG, bool FORCE, int CB = 16>
static cudaError_t pipe_attrs() {
  static unsigned long long done = 0;  // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_pipe<S, R, ODD, DIAG, FORCE, CB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(PipeSmem<S, R, CB>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pipe<S, R, ODD, DIAG, FORCE, CB>,
                           cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  done |= bit;
  return cudaSuccess;
}

template <class S, class R, bool ODD, bool DIAG, bool FORCE, int CB = 16>
static cudaError_t launch_pipe_f(Lattice &L, Args<S, R> &a) {
  cudaError_t e = pipe_attrs<S, R, ODD, DIAG, FORCE, CB>();
  if (e != cudaSuccess) return e;
  const dim3 grid((L.nx + PP_BX - 1) / PP_BX, (L.ny + PP_BY - 1) / PP_BY,
                  (L.nz + L.lz - 1) / L.lz);
  // wall nodes inside the march when the per-block lists match the launch
  // shape, else by k_wall after it
  const bool inblock = L.nw > 0 && L.wl && L.wl_lz == L.lz;
  a.wl = inblock ? L.wl : nullptr;
  a.wl_start = inblock ? L.wl_start : nullptr;
  k_pipe<S, R, ODD, DIAG, FORCE, CB><<<grid, PP_NT, sizeof(PipeSmem<S, R, CB>), L.stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || L.nw == 0 || inblock) return e;
  k_wall<S, R, ODD, DIAG><<<(L.nw + 127) / 128, 128, 0, L.stream>>>(a);
  return cudaGetLastError();
}

// The variant without body-force terms when F_ex = 0 (they vanish there);
// 16-bit lattices with nx = 4 mod 8 staged in 8-byte chunks.
template <class S, class R, bool ODD, bool DIAG>
static cudaError_t launch_pipe_t(Lattice &L, Args<S, R> &a) {
  if constexpr (sizeof(S) == 2) {
    if (pipe_chunk_bytes(L) == 8) return launch_pipe_f<S, R, ODD, DIAG, true, 8>(L, a);
  }
  if constexpr (std::is_same<R, float>::value) {  // FP64 keeps one form (parity)
    if (a.m.Fx == R(0) && a.m.Fy == R(0) && a.m.Fz == R(0))
      return launch_pipe_f<S, R, ODD, DIAG, false>(L, a);
  }
  return launch_pipe_f<S, R, ODD, DIAG, true>(L, a);
}

template <class S, class R, bool ODD, bool DIAG>
static cudaError_t launch_fused_t(Lattice &L, Args<S, R> &a) {
  if constexpr (pipe_storage<S>()) {
    if (pipe_eligible(L)) return launch_pipe_t<S, R, ODD, DIAG>(L, a);
  }
  if constexpr (std::is_same<S, float>::value && std::is_same<R, float>::value) {
    if (async_eligible(L)) return launch_async_t<ODD, DIAG>(L, a);
  }
  const int bx = L.bx, by = L.by;
  dim3 grid((L.nx + bx - 1) / bx, (L.ny + by - 1) / by, (L.nz + L.lz - 1) / L.lz);
  const size_t smem = fused_smem_bytes<R>(bx, by, DIAG);
  if (L.bc_on)  // open x boundaries: the variant with boundary cells
    k_fused<S, R, ODD, DIAG, true><<<grid, bx * by, smem, L.stream>>>(a, bx, by);
  else
    k_fused<S, R, ODD, DIAG, false><<<grid, bx * by, smem, L.stream>>>(a, bx, by);
  return cudaGetLastError();
}

template <class S, class R, bool ODD, int MODE, bool DIAG>
static cudaError_t launch_cell_t(Lattice &L, Args<S, R> &a) {
  const int T = 256;
  const long long B = (L.N + T - 1) / T;
  if (L.bc_on)
    k_phi<S, R, true><<<(unsigned)B, T, 0, L.stream>>>(a, (R *)L.phi);
  else
    k_phi<S, R, false><<<(unsigned)B, T, 0, L.stream>>>(a, (R *)L.phi);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (L.bc_on)
    k_cell<S, R, ODD, MODE, DIAG, true><<<(unsigned)B, T, 0, L.stream>>>(a);
  else
    k_cell<S, R, ODD, MODE, DIAG, false><<<(unsigned)B, T, 0, L.stream>>>(a);
  return cudaGetLastError();
}

// Planes per block for the fused kernels.  Blocks all do the same work, so
// a launch takes ceil(blocks / resident slots) rounds of one block's time;
// a block of lz planes also recomputes phi on two halo planes (about 0.3 of
// a plane's cost each).  Chooses lz in [2, 32] minimising
// rounds x (lz + 0.6), e.g. 7 for 128^3 with 32 x 4 tiles on 152 SMs x 4
// blocks (19 chunks x 128 columns = 4 full rounds).
template <class S, class R>
int auto_lz(const Lattice &L) {
  int dev = 0, nsm = 0, per = 0;
  bool tma = false, pipe = false;
  if constexpr (std::is_same<S, float>::value && std::is_same<R, float>::value)
    tma = async_eligible(L);
  if constexpr (pipe_storage<S>()) pipe = pipe_eligible(L);
  const int bx = pipe ? PP_BX : (tma ? AB_X : L.bx), by = pipe ? PP_BY : (tma ? AB_Y : L.by);
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (pipe) {
      if constexpr (pipe_storage<S>()) {
        e = pipe_attrs<S, R, false, true, true>();
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
              &per, k_pipe<S, R, false, true, true>, PP_NT, sizeof(PipeSmem<S, R>));
      }
    } else if (tma) {
      if constexpr (std::is_same<S, float>::value && std::is_same<R, float>::value) {
        e = async_attrs<false, true>();
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused_async<false, true>,
                                                            bx * by, AB_SMEM);
      }
    } else {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused<S, R, false, true>,
                                                        bx * by,
                                                        fused_smem_bytes<R>(bx, by, true));
    }
  }
  if (e != cudaSuccess || nsm < 1 || per < 1) {
    cudaGetLastError();
    return L.nz < 16 ? L.nz : 16;
  }
  const long long slots = (long long)nsm * per;
  const long long cols = (long long)((L.nx + bx - 1) / bx) * ((L.ny + by - 1) / by);
  int best = L.nz < 16 ? L.nz : 16;
  double best_cost = 1e300;
  for (int lz = (L.nz < 32 ? L.nz : 32); lz >= 2; --lz) {
    const long long blocks = cols * ((L.nz + lz - 1) / lz);
    const double cost = (double)((blocks + slots - 1) / slots) * (lz + 0.6);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = lz;
    }
  }
  return best;
}

template <class S, class R>
cudaError_t launch_step(Lattice &L, bool diag) {
  Args<S, R> a = make_args<S, R>(L);
  const bool odd = (L.step & 1) != 0;
  cudaError_t e = launch_xbc<S, R>(L, a);
  if (e != cudaSuccess) return e;
  if (diag) {
    // Diagnostic launch d accumulates into buffer d&1 and zeroes the other.
    a.diag = L.diag + 32 * (L.ndiag & 1);
    a.diag_zero = L.diag + 32 * ((L.ndiag + 1) & 1);
  }
  if (L.kernel != PFLB_KERNEL_TWOPASS) {  // fused, its TMA-staged and pipelined forms
    if (odd) e = diag ? launch_fused_t<S, R, true, true>(L, a) : launch_fused_t<S, R, true, false>(L, a);
    else e = diag ? launch_fused_t<S, R, false, true>(L, a) : launch_fused_t<S, R, false, false>(L, a);
  } else {
    if (odd) e = diag ? launch_cell_t<S, R, true, MODE_STEP, true>(L, a)
                      : launch_cell_t<S, R, true, MODE_STEP, false>(L, a);
    else e = diag ? launch_cell_t<S, R, false, MODE_STEP, true>(L, a)
                  : launch_cell_t<S, R, false, MODE_STEP, false>(L, a);
  }
  if (e == cudaSuccess) {
    if (diag) {
      L.last_diag_step = L.step;
      L.ndiag++;
    }
    L.step++;
  }
  return e;
}

template <class S, class R>
cudaError_t launch_macro(Lattice &L, bool fields) {
  Args<S, R> a = make_args<S, R>(L);
  a.out = fields ? L.out : nullptr;
  a.diag = L.diag + 64;
  a.diag_zero = nullptr;
  cudaError_t e = cudaMemsetAsync(a.diag, 0, 32 * sizeof(double), L.stream);
  if (e == cudaSuccess) e = launch_xbc<S, R>(L, a);
  if (e != cudaSuccess) return e;
  if (L.step & 1) return launch_cell_t<S, R, true, MODE_MACRO, true>(L, a);
  return launch_cell_t<S, R, false, MODE_MACRO, true>(L, a);
}

template <class S, class R>
cudaError_t mark_xbc(Lattice &L, bool on) {
  const int plane = L.ny * L.nz, T = 128;
  k_mark_xbc<<<(2 * plane + T - 1) / T, T, 0, L.stream>>>(L.flags, L.nx, plane, on ? 1 : 0);
  return cudaGetLastError();
}

template <class S, class R>
size_t batch_desc_bytes() { return sizeof(Args<S, R>); }

template <class S, class R>
void batch_build_descs(Lattice *const *lats, int n, char *host) {
  for (int l = 0; l < n; ++l) {
    for (int p = 0; p < 2; ++p) {
      Lattice tmp = *lats[l];
      tmp.step = p;  // selects buffers and A-A parity
      Args<S, R> a = make_args<S, R>(tmp);
      a.diag = lats[l]->diag + 32 * (lats[l]->ndiag & 1);
      a.diag_zero = lats[l]->diag + 32 * ((lats[l]->ndiag + 1) & 1);
      std::memcpy(host + (2 * (size_t)l + p) * sizeof(Args<S, R>), &a, sizeof a);
    }
  }
}

template <class S, class R, bool ODD, bool DIAG, int CB = 16>
static cudaError_t batch_pipe_attrs() {
  static unsigned long long done = 0;  // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_batch_pipe<S, R, ODD, DIAG, CB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(PipeSmem<S, R, CB>) + sizeof(Args<S, R>)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_batch_pipe<S, R, ODD, DIAG, CB>,
                           cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  done |= bit;
  return cudaSuccess;
}

template <class S, class R>
int batch_pipe_blocks_per_sm() {
  int nb = 0;
  if (batch_pipe_attrs<S, R, false, true>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &nb, k_batch_pipe<S, R, false, true>, PP_NT,
          sizeof(PipeSmem<S, R>) + sizeof(Args<S, R>)) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

// One launch over the work list of one chunk size (the two lists share the
// counter, reset before each launch on the batch stream).
template <class S, class R, bool ODD, bool DIAG, int CB>
static cudaError_t batch_pipe_list(const BatchDev &b, const void *items, int n) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = batch_pipe_attrs<S, R, ODD, DIAG, CB>();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(b.pcounter, 0, sizeof(int), b.stream);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(PipeSmem<S, R, CB>) + sizeof(Args<S, R>);
  const int grid = n < b.pgrid ? n : b.pgrid;
  k_batch_pipe<S, R, ODD, DIAG, CB><<<grid, PP_NT, smem, b.stream>>>(
      (const Args<S, R> *)b.descs, b.par0, (const int4 *)items, n, b.pcounter, b.bstep, b.plz);
  return cudaGetLastError();
}

template <class S, class R, bool ODD, bool DIAG>
static cudaError_t batch_pipe_one(const BatchDev &b) {
  cudaError_t e = batch_pipe_list<S, R, ODD, DIAG, 16>(b, b.pitems, b.npitems);
  if constexpr (sizeof(S) == 2) {
    if (e == cudaSuccess) e = batch_pipe_list<S, R, ODD, DIAG, 8>(b, b.pitems8, b.npitems8);
  }
  return e;
}

// The pipelined lattices of a batch: their march (one launch per A-A parity
// present at this step; tpar = parity of the batch step), then their wall
// nodes.
template <class S, class R>
static cudaError_t batch_launch_pipe(const BatchDev &b, bool diag, int tpar) {
  if (b.npitems + b.npitems8 == 0) return cudaSuccess;
  const Args<S, R> *d = (const Args<S, R> *)b.descs;
  cudaError_t e = cudaSuccess;
  for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
    if (!((b.pmask >> (par ^ tpar)) & 1)) continue;  // no lattice at this parity now
    if (par)
      e = diag ? batch_pipe_one<S, R, true, true>(b) : batch_pipe_one<S, R, true, false>(b);
    else
      e = diag ? batch_pipe_one<S, R, false, true>(b) : batch_pipe_one<S, R, false, false>(b);
  }
  if (e != cudaSuccess || b.nwitems == 0) return e;
  const int2 *wit = (const int2 *)b.witems;
  if (diag)
    k_batch_wall<S, R, true><<<b.nwitems, 128, 0, b.stream>>>(d, b.par0, wit, b.bstep);
  else
    k_batch_wall<S, R, false><<<b.nwitems, 128, 0, b.stream>>>(d, b.par0, wit, b.bstep);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t batch_launch_step(const BatchDev &b, bool diag, int tpar) {
  cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(int), b.stream);
  if (e != cudaSuccess) return e;
  const size_t smem = batch_smem<S, R>(b.bx, b.by, diag);
  const Args<S, R> *d = (const Args<S, R> *)b.descs;
  const int4 *it = (const int4 *)b.items;
  if (b.nxbc > 0) {  // boundary states of the open-boundary lattices first
    k_batch_xbc<S, R><<<dim3(b.nxbc, 32), 128, 0, b.stream>>>(d, b.par0, b.xlist, b.xspecs,
                                                              b.bstep);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = batch_launch_pipe<S, R>(b, diag, tpar);
  if (e != cudaSuccess) return e;
  if (b.nitems == 0) {  // every lattice ran the pipelined march
    k_batch_tick<<<1, 1, 0, b.stream>>>(b.bstep);
    return cudaGetLastError();
  }
  const dim3 grid(b.grid), block(b.bx * b.by);
  if (diag && b.nxbc > 0)
    k_batch<S, R, true, true><<<grid, block, smem, b.stream>>>(d, b.par0, it, b.nitems, b.counter,
                                                               b.bstep, b.bx, b.by, b.lz);
  else if (diag)
    k_batch<S, R, true, false><<<grid, block, smem, b.stream>>>(d, b.par0, it, b.nitems,
                                                                b.counter, b.bstep, b.bx, b.by,
                                                                b.lz);
  else if (b.nxbc > 0)
    k_batch<S, R, false, true><<<grid, block, smem, b.stream>>>(d, b.par0, it, b.nitems,
                                                                b.counter, b.bstep, b.bx, b.by,
                                                                b.lz);
  else
    k_batch<S, R, false, false><<<grid, block, smem, b.stream>>>(d, b.par0, it, b.nitems,
                                                                 b.counter, b.bstep, b.bx, b.by,
                                                                 b.lz);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_batch_tick<<<1, 1, 0, b.stream>>>(b.bstep);
  return cudaGetLastError();
}

template <class S, class R>
int batch_max_blocks_per_sm(int bx, int by) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<S, R, true>, bx * by,
                                                    batch_smem<S, R>(bx, by, true)) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

#define PFLB_INSTANTIATE(S, R)                                                   \
  template int batch_pipe_blocks_per_sm<S, R>();                                 \
  template size_t batch_desc_bytes<S, R>();                                      \
  template void batch_build_descs<S, R>(Lattice *const *, int, char *);         \
  template cudaError_t batch_launch_step<S, R>(const BatchDev &, bool, int);          \
  template int batch_max_blocks_per_sm<S, R>(int, int);                          \
  template cudaError_t launch_init<S, R>(Lattice &, const double *, double);     \
  template cudaError_t launch_step<S, R>(Lattice &, bool);                       \
  template cudaError_t launch_macro<S, R>(Lattice &, bool);                      \
  template cudaError_t set_model<S, R>(Lattice &);                               \
  template int max_block_threads<S, R>();                                        \
  template int auto_lz<S, R>(const Lattice &);                                  \
  template cudaError_t mark_xbc<S, R>(Lattice &, bool);

}  // namespace pflb
