// pflb_internal.h -- host-side lattice record shared by the C ABI and the
// per-precision launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pflb.h"

namespace pflb {

constexpr int kAsyncReads = 16;  // asynchronous diagnostic reads in flight per lattice

struct Lattice {
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  int nw = 0;                 // wall nodes
  pflb_params p{};
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;       // private stream for host uploads
  cudaEvent_t ev_init = nullptr;    // recorded after each init launch
  cudaEvent_t aev[16] = {};         // completion of asynchronous diagnostic reads
  int64_t aticket = 0;              // next asynchronous read ticket
  size_t elem = 4;            // bytes per stored population
  // device buffers
  void *h[2] = {nullptr, nullptr};  // [19][N] each
  void *g = nullptr;                // [19][N]
  void *wp[2] = {nullptr, nullptr}; // [18][nw] each
  uint8_t *flags = nullptr;         // [N]
  int *widx = nullptr;              // [N]
  uint32_t *wmask = nullptr;        // [nw]
  int *wcell = nullptr;             // [nw] cell of each wall node
  void *wgeo = nullptr;             // [5][nw] compute type
  uint32_t *wcut = nullptr;         // [nw] cut links | c_n << 24 (sub-voxel walls), or null
  void *sfrac = nullptr;            // [N] solid volume fraction, compute type, or null
  void *ghost = nullptr;            // [18][nw] compute type
  void *phi = nullptr;              // [N] compute type (two-pass path)
  double *diag = nullptr;           // [32]
  double *out = nullptr;            // [6][N] lazily allocated
  double *phi0 = nullptr;           // [N] init scratch, lazily allocated
  int *err = nullptr;               // device error flag (bounded waits that ran out)
  CUtensorMap tmap[2];              // TMA maps of the two h buffers (staged kernel)
  bool tma_ok = false;
  int64_t step = 0;
  int64_t ndiag = 0;          // diagnostic launches since init (ping-pong index)
  int64_t last_diag_step = -1;
  int diag_every = 0;         // pflb_step accumulates diagnostics every k-th step
  int kernel = PFLB_KERNEL_PIPE;
  int bx = 32, by = 4, lz = 16;   // lz: planes per block in effect
  int lz_req = 0;                  // requested planes per block, 0 = automatic
  // open x boundaries (reading R22)
  bool bc_on = false;
  int bc_type[2] = {0, 0};         // 1 pressure, 2 velocity
  double bc_val[2][5] = {};        // P, ux, uy, uz, phi (targets)
  double bc_from[2][5] = {};       // values at the start of the ramp
  int64_t bc_t0 = 0, bc_ramp = 0;  // ramp start step and length
  void *bcm = nullptr;             // [5][2 ny nz] boundary states, compute type
  int reg[6] = {0, 0, 0, 0, 0, 0};
  // per-block wall lists of the pipelined kernel (wall records grouped by
  // the 32 x 4 x lz block whose march covers them), built for lz = wl_lz
  int *wl = nullptr;               // [nw]
  int *wl_start = nullptr;         // [blocks + 1], sized for lz = 1
  int wl_lz = 0;
  std::vector<int> wcell_h;        // host copy of wcell
  bool poisoned = false;
  int64_t dev_bytes = 0;
};

// Device side of a batch of lattices stepped by one persistent kernel.
// Open x boundaries of one lattice as the boundary-state kernels take them.
struct XbcSpec {
  int type[2];        // 1 pressure (P given), 2 velocity (u and phi given); 0 closed
  double val[2][5];   // P, ux, uy, uz, phi (targets)
  double from[2][5];  // values at the start of the ramp
  long long t0;       // step at which the ramp started
  long long ramp;     // ramp length in steps (0: targets at once)
  long long step0;    // step of the launch (batches add the batch step)
};

struct BatchDev {
  void *descs = nullptr;   // [nlat][2] step descriptors (Args), both parities
  int *par0 = nullptr;     // [nlat] parity of each lattice at batch step 0
  void *items = nullptr;   // [nitems] int4 (lattice, x0, y0, z0)
  int nitems = 0;
  int *counter = nullptr;  // work-list cursor, reset before each step
  int *bstep = nullptr;    // batch steps since par0 was set
  int bx = 32, by = 4, lz = 16, grid = 0;
  cudaStream_t stream = nullptr;
  XbcSpec *xspecs = nullptr;  // [nlat] open-boundary specs (type 0: periodic x)
  int *xlist = nullptr;       // [nxbc] lattices with open boundaries
  int nxbc = 0;
  // lattices run by the pipelined march (pipe_layout_ok): their own work
  // list of 32 x 4 tile columns in chunks of plz planes, and their wall
  // nodes in chunks of 128 records (int2: lattice, first record)
  void *pitems = nullptr;
  int npitems = 0;
  void *pitems8 = nullptr;  // the same for lattices staged in 8-byte chunks
  int npitems8 = 0;
  int *pcounter = nullptr;
  int plz = 8, pgrid = 0;
  int pmask = 0;  // bit q: a pipelined lattice starts the batch call at A-A parity q
  void *witems = nullptr;
  int nwitems = 0;
};

// The pipelined step kernel runs with periodic x and nx a multiple of 4 (its
// 4-byte flag words), so that its row chunks and flag words are aligned;
// elsewhere PFLB_KERNEL_PIPE falls back to the fused kernel.  It stages rows
// in 16-byte chunks, or in 8-byte chunks at 16-bit storage when nx is not a
// multiple of 8 (pipe_chunk_bytes).
inline bool pipe_layout_ok(const Lattice &L) { return !L.bc_on && L.nx % 4 == 0; }
inline int pipe_chunk_bytes(const Lattice &L) {
  return (L.elem == 2 && L.nx % 8 != 0) ? 8 : 16;
}
inline bool pipe_kernel_runs(const Lattice &L) {
  return L.kernel == PFLB_KERNEL_PIPE && pipe_layout_ok(L);
}

// Sets the thread-local message returned by pflb_last_error().
void set_last_error(const char *msg);

// Per-precision launchers (pflb_launch.cuh, instantiated per storage type).
// All enqueue work on L.stream; none synchronises.
// Given boundary value k (P, ux, uy, uz, phi) of side s at step t: linear
// ramp from `from` (at step t0) to `val` (at step t0 + ramp).
__host__ __device__ inline double xbc_value(const XbcSpec &sp, int s, int k, long long t) {
  if (sp.ramp <= 0 || t >= sp.t0 + sp.ramp) return sp.val[s][k];
  const double f = t <= sp.t0 ? 0.0 : (double)(t - sp.t0) / (double)sp.ramp;
  return sp.from[s][k] + f * (sp.val[s][k] - sp.from[s][k]);
}

// The open-boundary spec of a lattice for launches starting at step step0.
inline XbcSpec xbc_spec(const Lattice &L, long long step0) {
  XbcSpec sp;
  for (int side = 0; side < 2; ++side) {
    sp.type[side] = L.bc_on ? L.bc_type[side] : 0;
    for (int k = 0; k < 5; ++k) {
      sp.val[side][k] = L.bc_val[side][k];
      sp.from[side][k] = L.bc_from[side][k];
    }
  }
  sp.t0 = L.bc_t0;
  sp.ramp = L.bc_ramp;
  sp.step0 = step0;
  return sp;
}

template <class S, class R> cudaError_t launch_init(Lattice &L, const double *d_phi0, double P0);
template <class S, class R> cudaError_t launch_step(Lattice &L, bool diag);
template <class S, class R> cudaError_t launch_macro(Lattice &L, bool fields);
template <class S, class R> cudaError_t set_model(Lattice &L);
template <class S, class R> int max_block_threads();
template <class S, class R> int auto_lz(const Lattice &L);
template <class S, class R> cudaError_t mark_xbc(Lattice &L, bool on);
// Batch: size of one descriptor, host-side descriptor build (2 per lattice,
// diagnostics pointers for the next diagnostic launch), one step launch,
// and the occupancy-limited blocks per SM of the batch kernel.
template <class S, class R> size_t batch_desc_bytes();
template <class S, class R> void batch_build_descs(Lattice *const *lats, int n, char *host);
template <class S, class R> cudaError_t batch_launch_step(const BatchDev &b, bool diag,
                                                         int tpar);
template <class S, class R> int batch_max_blocks_per_sm(int bx, int by);
template <class S, class R> int batch_pipe_blocks_per_sm();

}  // namespace pflb

// The opaque handle of the C ABI is the lattice state itself.
struct pflb_lattice : public pflb::Lattice {};
