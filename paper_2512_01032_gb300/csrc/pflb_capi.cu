// pflb_capi.cu -- C ABI of the phase-field lattice Boltzmann library
// (declarations and contracts in include/pflb.h).
//
// Host side of lattice creation: the voxel mask becomes per-cell flags
// (solid, wall node), a wall-node list in cell order with each node's
// solid-link bits, wall normal and contact angle (Sec. II B), then
// everything is uploaded once.  Stepping only enqueues kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "pflb_internal.h"
#include "pflb_model.cuh"

using pflb::Lattice;


struct pflb_batch {
  std::vector<Lattice *> lats;
  int storage = PFLB_STORAGE_FP32;
  pflb::BatchDev dev;
  size_t desc_bytes = 0;
  size_t items_cap = 0;
  int blocks_per_sm = 0;  // requested; 0 = as many as fit, at most 4
  int per_sm = 0;         // in use (the grid may be smaller when items are few)
  int nsm = 0;
  bool own_stream = false;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;  // kGraphSteps plain steps
  int graph_nxbc = -1;               // open-boundary lattice count the graph was captured for
  int graph_pmask = -1;              // A-A parities of the pipelined lattices at capture
  std::vector<char> pipe_set;        // lattices the work lists were built to march pipelined
  bool poisoned = false;
};
static constexpr int kGraphSteps = 16;

namespace {

thread_local std::string g_err;

pflb_status fail(pflb_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

// A failed device allocation: out of memory only when the allocator says so;
// any other error (no usable device, a driver too old) is a CUDA error.
pflb_status alloc_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? PFLB_ERR_OOM : PFLB_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

pflb_status cuda_fail(Lattice *L, cudaError_t e, const char *what) {
  if (L) L->poisoned = true;
  return fail(PFLB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(L, call)                                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(L, e_, #call); \
  } while (0)

bool is_fp64(const Lattice *L) { return L->p.storage == PFLB_STORAGE_FP64; }

// Storage-type dispatch (compute in FP64 for FP64 storage, else FP32).
template <class F>
cudaError_t dispatch(Lattice *L, F &&f) {
  switch (L->p.storage) {
    case PFLB_STORAGE_FP64: return f((double *)nullptr, (double *)nullptr);
    case PFLB_STORAGE_FP32: return f((float *)nullptr, (float *)nullptr);
    case PFLB_STORAGE_FP16: return f((__half *)nullptr, (float *)nullptr);
    default: return f((__nv_bfloat16 *)nullptr, (float *)nullptr);
  }
}
cudaError_t do_init(Lattice *L, const double *d_phi0, double P0) {
  return dispatch(L, [&](auto *s, auto *r) {
    using S = std::remove_pointer_t<decltype(s)>;
    using R = std::remove_pointer_t<decltype(r)>;
    return pflb::launch_init<S, R>(*L, d_phi0, P0);
  });
}
cudaError_t do_step(Lattice *L, bool diag) {
  return dispatch(L, [&](auto *s, auto *r) {
    using S = std::remove_pointer_t<decltype(s)>;
    using R = std::remove_pointer_t<decltype(r)>;
    return pflb::launch_step<S, R>(*L, diag);
  });
}
cudaError_t do_macro(Lattice *L, bool fields) {
  return dispatch(L, [&](auto *s, auto *r) {
    using S = std::remove_pointer_t<decltype(s)>;
    using R = std::remove_pointer_t<decltype(r)>;
    return pflb::launch_macro<S, R>(*L, fields);
  });
}
template <class F>
auto dispatch_storage(int storage, F &&f) {
  switch (storage) {
    case PFLB_STORAGE_FP64: return f((double *)nullptr, (double *)nullptr);
    case PFLB_STORAGE_FP32: return f((float *)nullptr, (float *)nullptr);
    case PFLB_STORAGE_FP16: return f((__half *)nullptr, (float *)nullptr);
    default: return f((__nv_bfloat16 *)nullptr, (float *)nullptr);
  }
}
#define PFLB_SR_TYPES                                   \
  using S = std::remove_pointer_t<decltype(s_)>;       \
  using R = std::remove_pointer_t<decltype(r_)>;

size_t storage_bytes(int storage) {
  return storage == PFLB_STORAGE_FP64 ? 8 : (storage == PFLB_STORAGE_FP32 ? 4 : 2);
}
size_t compute_bytes(int storage) { return storage == PFLB_STORAGE_FP64 ? 8 : 4; }
// h slots per cell: the 16-bit formats keep the rest population's remainder.
size_t h_slots_of(int storage) { return storage_bytes(storage) == 2 ? 20 : 19; }

// Planes per block in effect: the requested value, else the automatic one.
int resolve_lz(Lattice *L) {
  if (L->lz_req > 0) return L->lz_req;
  return dispatch_storage(L->p.storage, [&](auto *s_, auto *r_) {
    PFLB_SR_TYPES
    return pflb::auto_lz<S, R>(*L);
  });
}

// Per-block wall lists of the pipelined kernel for the lz in effect: wall
// records grouped by the block (32 x 4 tile, chunk of lz planes) whose march
// covers their cell, in the kernel's block numbering (x, then y, then the z
// chunks alternating from both ends: chunk c < ceil(n/2) is block row 2c,
// the others 2 (n - 1 - c) + 1).  Copied on stream st (the lattice's
// stream once created, so that steps queued before use the previous lists);
// copies from pageable memory have read the host vectors on return.
cudaError_t ensure_wall_lists(Lattice *L, cudaStream_t st) {
  if (!L->wl || L->nw == 0 || L->wl_lz == L->lz || !pflb::pipe_layout_ok(*L)) return cudaSuccess;
  const int lz = L->lz, gx = (L->nx + 31) / 32, gy = (L->ny + 3) / 4;
  const int nch = (L->nz + lz - 1) / lz;
  const size_t nb = (size_t)gx * gy * nch;
  std::vector<int> start(nb + 1, 0), list((size_t)L->nw), blk((size_t)L->nw);
  const long long sxy = (long long)L->nx * L->ny;
  for (int r = 0; r < L->nw; ++r) {
    const long long c = L->wcell_h[(size_t)r];
    const int x = (int)(c % L->nx), y = (int)((c / L->nx) % L->ny), z = (int)(c / sxy);
    const int ch = z / lz;
    const int bz = ch < (nch + 1) / 2 ? 2 * ch : 2 * (nch - 1 - ch) + 1;
    blk[(size_t)r] = x / 32 + gx * (y / 4 + gy * bz);
    ++start[(size_t)blk[(size_t)r] + 1];
  }
  for (size_t b = 0; b < nb; ++b) start[b + 1] += start[b];
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (int r = 0; r < L->nw; ++r) list[(size_t)fill[(size_t)blk[(size_t)r]]++] = r;
  cudaError_t e = cudaMemcpyAsync(L->wl, list.data(), list.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L->wl_start, start.data(), start.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) L->wl_lz = lz;
  return e;
}

// Blocks of the pipelined grid at one plane per block (the size of wl_start).
size_t wall_list_blocks(long long nx, long long ny, long long nz) {
  return (size_t)(((nx + 31) / 32) * ((ny + 3) / 4) * nz);
}

pflb_status check_lattice(const pflb_lattice *L) {
  if (!L) return fail(PFLB_ERR_ARG, "null lattice");
  if (L->poisoned) return fail(PFLB_ERR_STATE, "lattice poisoned by an earlier CUDA error");
  return PFLB_OK;
}

pflb_status check_params(const pflb_params *p) {
  if (!p) return fail(PFLB_ERR_ARG, "null params");
  if (!(p->W > 0) || !(p->M > 0) || !(p->sigma >= 0))
    return fail(PFLB_ERR_ARG, "need W > 0, M > 0, sigma >= 0");
  if (!(p->nu_H > 0) || !(p->nu_L > 0))
    return fail(PFLB_ERR_ARG, "need nu > 0 (tau = nu/T + 1/2 > 1/2)");
  if (!(p->rho_H > 0) || !(p->rho_L > 0)) return fail(PFLB_ERR_ARG, "need rho_H, rho_L > 0");
  if (!(p->blend >= 0 && p->blend <= 1)) return fail(PFLB_ERR_ARG, "need 0 <= blend <= 1");
  if (!(p->D > 0) || !(p->F_width > 0)) return fail(PFLB_ERR_ARG, "need D > 0, F_width > 0");
  if (p->storage < PFLB_STORAGE_FP64 || p->storage > PFLB_STORAGE_BF16)
    return fail(PFLB_ERR_ARG, "unknown storage");
  if (p->F_mode != 0 && p->F_mode != 1) return fail(PFLB_ERR_ARG, "F_mode must be 0 or 1");
  return PFLB_OK;
}

inline long long wrap(long long a, long long n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Runs fn(z0, z1) over [0, nz) split into contiguous chunks on up to 16
// host threads (the chunks write disjoint outputs).
template <class F>
void parallel_z(int nz, long long cells, F &&fn) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::min<unsigned>(hw ? hw : 1, 16u);
  if (cells < (1 << 16)) nt = 1;
  nt = std::max(1, std::min(nt, nz));
  if (nt == 1) {
    fn(0, nz);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    const int z0 = (int)((long long)nz * t / nt), z1 = (int)((long long)nz * (t + 1) / nt);
    th.emplace_back([&fn, z0, z1] { fn(z0, z1); });
  }
  for (auto &t : th) t.join();
}

// Solid-link bits (bit i set when x + c_i is solid, periodic wrap) of every
// fluid cell; 0 for solid cells.
std::vector<uint32_t> link_masks(const pflb_geometry *g) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const long long N = (long long)nx * ny * nz;
  std::vector<uint32_t> mask((size_t)N, 0);
  std::vector<int> xw(nx + 2), yw(ny + 2), zw(nz + 2);  // coordinate + 1 -> wrapped
  for (int a = -1; a <= nx; ++a) xw[a + 1] = (int)wrap(a, nx);
  for (int a = -1; a <= ny; ++a) yw[a + 1] = (int)wrap(a, ny);
  for (int a = -1; a <= nz; ++a) zw[a + 1] = (int)wrap(a, nz);
  const uint8_t *solid = g->solid;
  parallel_z(nz, N, [&](int z0, int z1) {
    for (int z = z0; z < z1; ++z)
      for (int y = 0; y < ny; ++y) {
        const long long row = (long long)nx * (y + (long long)ny * z);
        for (int x = 0; x < nx; ++x) {
          if (solid[row + x]) continue;
          uint32_t m = 0;
          for (int i = 1; i < pflb::Q; ++i) {
            const long long nb = xw[x + pflb::cx_of(i) + 1] +
                                 (long long)nx * (yw[y + pflb::cy_of(i) + 1] +
                                                  (long long)ny * zw[z + pflb::cz_of(i) + 1]);
            if (solid[nb]) m |= 1u << i;
          }
          mask[(size_t)(row + x)] = m;
        }
      }
  });
  return mask;
}

// Solid volume fraction of cell c (sub-voxel walls): 1 on solid voxels.
inline double cell_frac(const pflb_geometry *g, long long c) {
  return g->solid[c] ? 1.0 : (g->solid_frac ? g->solid_frac[c] : 0.0);
}

// Cut-link bits (bit i set when x + c_i is a fluid cell with solid fraction
// > 0) of every fluid cell; all zero without fractions.
std::vector<uint32_t> cut_masks(const pflb_geometry *g) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  const long long N = (long long)nx * ny * nz;
  std::vector<uint32_t> mask((size_t)N, 0);
  if (!g->solid_frac) return mask;
  parallel_z(nz, N, [&](int z0, int z1) {
    for (int z = z0; z < z1; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const long long c = x + (long long)nx * (y + (long long)ny * z);
          if (g->solid[c]) continue;
          uint32_t m = 0;
          for (int i = 1; i < pflb::Q; ++i) {
            const long long nb = wrap(x + pflb::cx_of(i), nx) +
                                 (long long)nx * (wrap(y + pflb::cy_of(i), ny) +
                                                  (long long)ny * wrap(z + pflb::cz_of(i), nz));
            if (!g->solid[nb] && g->solid_frac[nb] > 0.0) m |= 1u << i;
          }
          mask[(size_t)c] = m;
        }
  });
  return mask;
}

// True if every fluid cell's solid fraction is in [0, 1).
bool fractions_ok(const pflb_geometry *g) {
  if (!g->solid_frac) return true;
  const long long N = (long long)g->nx * g->ny * g->nz;
  for (long long c = 0; c < N; ++c)
    if (!g->solid[c] && !(g->solid_frac[c] >= 0.0 && g->solid_frac[c] < 1.0)) return false;
  return true;
}

struct HostGeom {
  std::vector<uint8_t> flags;
  std::vector<int> widx;
  std::vector<int> wcell;    // [nw] cell of each wall node
  std::vector<uint32_t> wmask;
  std::vector<double> wgeo;  // [5][nw]
  std::vector<uint32_t> wcut;   // [nw] cut links | c_n << 24; empty without cut cells
  std::vector<double> sfrac;    // [N]; empty without cut cells
};

// Flags, wall list (cell order), solid-link masks, normals and angles.
void build_geometry(const pflb_geometry *g, const pflb_params *p, HostGeom &hg) {
  const long long N = (long long)g->nx * g->ny * g->nz;
  const std::vector<uint32_t> all = link_masks(g);
  const std::vector<uint32_t> cut = cut_masks(g);
  bool has_cut = false;
  if (g->solid_frac)
    for (long long c = 0; c < N && !has_cut; ++c) has_cut = !g->solid[c] && g->solid_frac[c] > 0;
  hg.flags.assign(N, 0);
  hg.widx.assign(N, -1);
  std::vector<uint32_t> masks, cuts;
  std::vector<long long> cells;
  for (long long c = 0; c < N; ++c) {
    if (g->solid[c]) {
      hg.flags[c] = pflb::F_SOLID;
    } else if (all[c] || cut[c]) {
      hg.flags[c] = pflb::F_WALL;
      hg.widx[c] = (int)cells.size();
      cells.push_back(c);
      masks.push_back(all[c]);
      cuts.push_back(cut[c]);
    }
  }
  const size_t nw = cells.size();
  hg.wmask = masks;
  hg.wcell.assign(cells.begin(), cells.end());
  // cells whose phi a wall node's stencil reads: the node and its fluid
  // neighbours (periodic wrap)
  for (size_t k = 0; k < nw; ++k) {
    const long long c = cells[k];
    const int x = (int)(c % g->nx), y = (int)((c / g->nx) % g->ny), z = (int)(c / ((long long)g->nx * g->ny));
    for (int i = 0; i < pflb::Q; ++i) {
      const long long nb = wrap(x + pflb::cx_of(i), g->nx) +
                           (long long)g->nx * (wrap(y + pflb::cy_of(i), g->ny) +
                                               (long long)g->ny * wrap(z + pflb::cz_of(i), g->nz));
      if (!(hg.flags[nb] & pflb::F_SOLID)) hg.flags[nb] |= pflb::F_NEAR;
    }
  }
  hg.wgeo.assign(5 * nw, 0.0);
  for (size_t k = 0; k < nw; ++k) {
    const long long c = cells[k];
    double n[3] = {0, 0, 0};
    const int x = (int)(c % g->nx), y = (int)((c / g->nx) % g->ny);
    const int z = (int)(c / ((long long)g->nx * g->ny));
    auto nbr = [&](int i) {
      return wrap(x + pflb::cx_of(i), g->nx) +
             (long long)g->nx * (wrap(y + pflb::cy_of(i), g->ny) +
                                 (long long)g->ny * wrap(z + pflb::cz_of(i), g->nz));
    };
    if (g->wall_normal) {
      for (int a = 0; a < 3; ++a) n[a] = g->wall_normal[3 * c + a];
    } else {
      // -sum_i w_i c_i s(x + c_i), s = 1 on solid voxels
      for (int i = 1; i < pflb::Q; ++i) {
        const double sf = ((masks[k] >> i) & 1u) ? 1.0 : (((cuts[k] >> i) & 1u) ? cell_frac(g, nbr(i)) : 0.0);
        n[0] -= pflb::w_of(i) * pflb::cx_of(i) * sf;
        n[1] -= pflb::w_of(i) * pflb::cy_of(i) * sf;
        n[2] -= pflb::w_of(i) * pflb::cz_of(i) * sf;
      }
      const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      if (nn > 0)
        for (int a = 0; a < 3; ++a) n[a] /= nn;
    }
    if (has_cut) {
      // c_n: the axis direction (1..6) with the largest c . n_w (first on
      // ties); 0 when the node is not cut or that neighbour is solid
      int cn = 0;
      double best = 0.0;
      for (int i = 1; i <= 6; ++i) {
        const double d = pflb::cx_of(i) * n[0] + pflb::cy_of(i) * n[1] + pflb::cz_of(i) * n[2];
        if (d > best) { best = d; cn = i; }
      }
      if (!(cell_frac(g, c) > 0.0) || g->solid[nbr(cn)]) cn = 0;
      // only links into the wall (c_i . n_w < 0) cross it; links to cut
      // cells parallel to the wall or away from it take the cell's phi
      uint32_t cm = cuts[k];
      for (int i = 1; i < pflb::Q; ++i)
        if (!(pflb::cx_of(i) * n[0] + pflb::cy_of(i) * n[1] + pflb::cz_of(i) * n[2] < -1e-9))
          cm &= ~(1u << i);
      hg.wcut.push_back(cm | ((uint32_t)cn << 24));
    }
    const double th = (g->theta_deg ? g->theta_deg[c] : p->theta_deg) * (3.14159265358979323846 / 180.0);
    hg.wgeo[0 * nw + k] = n[0];
    hg.wgeo[1 * nw + k] = n[1];
    hg.wgeo[2 * nw + k] = n[2];
    hg.wgeo[3 * nw + k] = std::cos(th);
    hg.wgeo[4 * nw + k] = std::sin(th);
  }
  if (has_cut) {
    hg.sfrac.resize((size_t)N);
    for (long long c = 0; c < N; ++c) hg.sfrac[(size_t)c] = cell_frac(g, c);
  }
}

template <class T>
cudaError_t dev_alloc(Lattice *L, T **ptr, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
  if (e == cudaSuccess) L->dev_bytes += (int64_t)(count * sizeof(T));
  return e;
}

void free_all(Lattice *L) {
  void *ptrs[] = {L->h[0], L->h[1], L->g, L->wp[0], L->wp[1], L->flags, L->widx, L->wmask,
                  L->wgeo, L->ghost, L->phi, L->diag, L->out, L->phi0, L->err, L->bcm,
                  L->wcell, L->wcut, L->sfrac, L->wl, L->wl_start};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (L->aux) cudaStreamDestroy(L->aux);
  if (L->ev_init) cudaEventDestroy(L->ev_init);
  for (cudaEvent_t &ev : L->aev)
    if (ev) cudaEventDestroy(ev), ev = nullptr;
  L->aux = nullptr;
  L->ev_init = nullptr;
}

int64_t bytes_for(long long nx, long long ny, long long nz, long long nw, int storage,
                  bool has_cut = false) {
  const long long N = nx * ny * nz;
  const int64_t e = (int64_t)storage_bytes(storage);
  const int64_t r = (int64_t)compute_bytes(storage);
  const int64_t flag_bytes = (N + 3) & ~(int64_t)3;  // whole 4-byte words
  const int64_t lists = nw ? nw * 4 + ((int64_t)wall_list_blocks(nx, ny, nz) + 1) * 4 : 0;
  return (2 * (int64_t)h_slots_of(storage) + 19) * N * e + 2 * 18 * nw * e + flag_bytes +
         N * 4 + nw * 8 + 5 * nw * r + 18 * nw * r + N * r + 96 * 8 + 4 + lists +
         (has_cut ? nw * 4 + N * r : 0);
}

// TMA descriptors of the two h buffers (4-D: x, y, z, direction; box
// 40 x 10 x 1 x 19 floats) for the staged step kernel.  Needs FP32 storage,
// nx a multiple of 4 (16-byte row strides) and nx >= 64.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)ptr;
    cudaGetLastError();
  }
  return fn;
}

void make_tmaps(Lattice *L) {
  L->tma_ok = false;
  if (L->p.storage != PFLB_STORAGE_FP32 || L->nx % 4 != 0 || L->nx < 64) return;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return;
  const cuuint64_t dims[4] = {(cuuint64_t)L->nx, (cuuint64_t)L->ny, (cuuint64_t)L->nz, 19};
  const cuuint64_t strides[3] = {(cuuint64_t)L->nx * 4, (cuuint64_t)L->nx * L->ny * 4,
                                 (cuuint64_t)L->N * 4};
  const cuuint32_t box[4] = {40, 10, 1, 19};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int b = 0; b < 2; ++b) {
    CUresult r = fn(&L->tmap[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L->h[b], dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
  }
  L->tma_ok = true;
}

}  // namespace

void pflb::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

extern "C" {

void pflb_default_params(pflb_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->sigma = 0.01;
  p->W = 4.0;
  p->M = 0.02;
  p->rho_H = 1.0;
  p->rho_L = 1e-3;
  p->nu_H = 0.1;
  p->nu_L = 0.1;
  p->theta_deg = 90.0;
  p->gamma = -22.5;
  p->phi_M = 0.8;
  p->phi_m = 0.2;
  p->D = 1e-4;
  p->eps = 1e-10;
  p->blend = 0.95;
  p->band_lo = 0.5;
  p->band_hi = 0.95;
  p->F_tilde = 0.1;
  p->F_width = 0.001;
  p->F_mode = 0;
  p->mobility_corr = 1;
  p->free_slip = 0;
  p->storage = PFLB_STORAGE_FP32;
}

pflb_status pflb_create(const pflb_geometry *geom, const pflb_params *params, void *cuda_stream,
                        pflb_lattice **out) {
  if (!out) return fail(PFLB_ERR_ARG, "null out");
  *out = nullptr;
  if (!geom || !geom->solid) return fail(PFLB_ERR_ARG, "null geometry or mask");
  if (geom->nx < 1 || geom->ny < 1 || geom->nz < 1)
    return fail(PFLB_ERR_ARG, "dimensions must be >= 1");
  if ((long long)geom->nx * geom->ny * geom->nz >= (1LL << 31))
    return fail(PFLB_ERR_ARG, "lattice too large (nx*ny*nz must be below 2^31)");
  pflb_status s = check_params(params);
  if (s != PFLB_OK) return s;
  if (!fractions_ok(geom)) return fail(PFLB_ERR_ARG, "solid_frac of a fluid cell outside [0, 1)");

  pflb_lattice *L = new (std::nothrow) pflb_lattice();
  if (!L) return fail(PFLB_ERR_OOM, "host allocation failed");
  L->nx = geom->nx; L->ny = geom->ny; L->nz = geom->nz;
  L->N = (long long)L->nx * L->ny * L->nz;
  L->p = *params;
  L->stream = (cudaStream_t)cuda_stream;
  L->elem = storage_bytes(L->p.storage);
  L->reg[1] = L->nx; L->reg[3] = L->ny; L->reg[5] = L->nz;
  L->lz = L->nz < 16 ? L->nz : 16;  // replaced by the automatic choice once created

  HostGeom hg;
  try {
    build_geometry(geom, params, hg);
  } catch (...) {
    delete L;
    return fail(PFLB_ERR_OOM, "host allocation failed while building geometry");
  }
  L->nw = (int)hg.wmask.size();
  const size_t N = (size_t)L->N, nw = (size_t)L->nw;
  const size_t E = L->elem, Rb = compute_bytes(L->p.storage);
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaSuccess) L->dev_bytes += (int64_t)bytes;
  };
  const size_t HS = h_slots_of(L->p.storage);
  A(&L->h[0], HS * N * E);
  A(&L->h[1], HS * N * E);
  A(&L->g, 19 * N * E);
  A(&L->wp[0], 18 * nw * E);
  A(&L->wp[1], 18 * nw * E);
  A((void **)&L->flags, (N + 3) & ~(size_t)3);  // whole 4-byte words (staged copies)
  A((void **)&L->widx, N * sizeof(int));
  A((void **)&L->wmask, nw * sizeof(uint32_t));
  A((void **)&L->wcell, nw * sizeof(int));
  A(&L->wgeo, 5 * nw * Rb);
  if (!hg.sfrac.empty()) {
    A((void **)&L->wcut, nw * sizeof(uint32_t));
    A(&L->sfrac, N * Rb);
  }
  A(&L->ghost, 18 * nw * Rb);
  A(&L->phi, N * Rb);
  if (nw) {
    A((void **)&L->wl, nw * sizeof(int));
    A((void **)&L->wl_start, (wall_list_blocks(L->nx, L->ny, L->nz) + 1) * sizeof(int));
  }
  A((void **)&L->diag, 96 * sizeof(double));
  A((void **)&L->err, sizeof(int));
  if (e != cudaSuccess) {
    free_all(L);
    delete L;
    cudaGetLastError();
    return alloc_fail(e, "device allocation failed");
  }
  // Upload geometry.
  std::vector<float> wgeo_f;
  const void *wgeo_src = hg.wgeo.data();
  if (!is_fp64(L)) {
    wgeo_f.assign(hg.wgeo.begin(), hg.wgeo.end());
    wgeo_src = wgeo_f.data();
  }
  // The upload runs on a private stream: the new buffers are not referenced
  // by anything queued on the lattice's stream, so creating a lattice does
  // not wait for the caller's work in flight (e.g. other lattices' steps).
  e = cudaStreamCreateWithFlags(&L->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->ev_init, cudaEventDisableTiming);
  cudaStream_t st = L->aux;
  if (e == cudaSuccess && (N & 3))
    e = cudaMemsetAsync(L->flags + N, 0, ((N + 3) & ~(size_t)3) - N, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L->flags, hg.flags.data(), N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L->widx, hg.widx.data(), N * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nw)
    e = cudaMemcpyAsync(L->wmask, hg.wmask.data(), nw * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nw)
    e = cudaMemcpyAsync(L->wcell, hg.wcell.data(), nw * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nw)
    e = cudaMemcpyAsync(L->wgeo, wgeo_src, 5 * nw * Rb, cudaMemcpyHostToDevice, st);
  std::vector<float> sfrac_f;
  if (!hg.sfrac.empty()) {
    const void *sfrac_src = hg.sfrac.data();
    if (!is_fp64(L)) {
      sfrac_f.assign(hg.sfrac.begin(), hg.sfrac.end());
      sfrac_src = sfrac_f.data();
    }
    if (e == cudaSuccess && nw)
      e = cudaMemcpyAsync(L->wcut, hg.wcut.data(), nw * sizeof(uint32_t), cudaMemcpyHostToDevice,
                          st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L->sfrac, sfrac_src, N * Rb, cudaMemcpyHostToDevice, st);
  }
  void *zero_bufs[] = {L->h[0], L->h[1], L->g, L->wp[0], L->wp[1], L->ghost, L->phi, L->err};
  size_t zero_len[] = {HS * N * E, HS * N * E, 19 * N * E, 18 * nw * E, 18 * nw * E,
                       18 * nw * Rb, N * Rb, sizeof(int)};
  for (int k = 0; k < 8 && e == cudaSuccess; ++k)
    if (zero_len[k]) e = cudaMemsetAsync(zero_bufs[k], 0, zero_len[k], st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_all(L);
    delete L;
    return fail(PFLB_ERR_CUDA, std::string("upload failed: ") + cudaGetErrorString(e));
  }
  make_tmaps(L);
  L->lz = resolve_lz(L);
  L->wcell_h.swap(hg.wcell);
  e = ensure_wall_lists(L, L->aux);  // nothing on the lattice's stream reads them yet
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->aux);
  if (e != cudaSuccess) {
    free_all(L);
    delete L;
    return fail(PFLB_ERR_CUDA, std::string("upload failed: ") + cudaGetErrorString(e));
  }
  *out = L;
  return PFLB_OK;
}

// Initial state from L->phi0, asynchronous on the lattice stream; the
// event marks when phi0 may be overwritten again.
static pflb_status init_from_device_phi(pflb_lattice *L, double P0) {
  CK(L, do_init(L, L->phi0, P0));
  CK(L, cudaEventRecord(L->ev_init, L->stream));
  return PFLB_OK;
}

pflb_status pflb_init_phi(pflb_lattice *L, const double *phi_host, double P0) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!phi_host) return fail(PFLB_ERR_ARG, "null phi");
  if (!L->phi0) {
    cudaError_t e = cudaMalloc((void **)&L->phi0, (size_t)L->N * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      L->phi0 = nullptr;
      return alloc_fail(e, "device allocation failed (init scratch)");
    }
    L->dev_bytes += L->N * 8;
  }
  // The copy runs on the private stream (after any earlier init of this
  // lattice has read phi0) and the host waits for the copy alone, not for
  // the work queued on the lattice stream.
  CK(L, cudaStreamWaitEvent(L->aux, L->ev_init, 0));
  CK(L, cudaMemcpyAsync(L->phi0, phi_host, (size_t)L->N * sizeof(double), cudaMemcpyHostToDevice,
                        L->aux));
  CK(L, cudaStreamSynchronize(L->aux));
  return init_from_device_phi(L, P0);
}

pflb_status pflb_init_tanh(pflb_lattice *L, int shape, const double center[3], double R,
                           const double normal[3], double P0) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!center || shape < 0 || shape > 2) return fail(PFLB_ERR_ARG, "bad shape or center");
  double nv[3] = {1, 0, 0};
  if (shape != 0) {
    if (!normal) return fail(PFLB_ERR_ARG, "shape needs a normal");
    const double nn = std::sqrt(normal[0] * normal[0] + normal[1] * normal[1] + normal[2] * normal[2]);
    if (!(nn > 0)) return fail(PFLB_ERR_ARG, "zero normal");
    for (int a = 0; a < 3; ++a) nv[a] = normal[a] / nn;
  }
  std::vector<double> phi;
  try {
    phi.resize((size_t)L->N);
  } catch (...) {
    return fail(PFLB_ERR_OOM, "host allocation failed");
  }
  const double W = L->p.W;
  const int dims[3] = {L->nx, L->ny, L->nz};
  const long long plane = (long long)L->nx * L->ny;
  parallel_z(L->nz, L->N, [&](int z0, int z1) {
  for (long long c = z0 * plane; c < z1 * plane; ++c) {
    const long long pos[3] = {c % L->nx, (c / L->nx) % L->ny, c / plane};
    double d[3];
    for (int a = 0; a < 3; ++a) {
      double dd = (double)pos[a] - center[a];
      dd -= dims[a] * std::nearbyint(dd / dims[a]);  // minimum image
      d[a] = dd;
    }
    double arg;
    if (shape == 0) {
      arg = R - std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    } else {
      const double sd = d[0] * nv[0] + d[1] * nv[1] + d[2] * nv[2];
      arg = shape == 1 ? -sd : R - std::fabs(sd);
    }
    phi[c] = 0.5 * (1.0 + std::tanh(2.0 * arg / W));  // Eq. 12
  }
  });
  return pflb_init_phi(L, phi.data(), P0);
}

pflb_status pflb_set_force(pflb_lattice *L, const double Fex[3]) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!Fex) return fail(PFLB_ERR_ARG, "null force");
  for (int a = 0; a < 3; ++a) L->p.Fex[a] = Fex[a];
  return PFLB_OK;
}

pflb_status pflb_set_region(pflb_lattice *L, const int box[6]) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!box) return fail(PFLB_ERR_ARG, "null box");
  for (int k = 0; k < 6; ++k) L->reg[k] = box[k];
  return PFLB_OK;
}

pflb_status pflb_set_kernel(pflb_lattice *L, int kind, int bx, int by, int lz) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (kind != PFLB_KERNEL_FUSED && kind != PFLB_KERNEL_TWOPASS && kind != PFLB_KERNEL_FUSED_TMA &&
      kind != PFLB_KERNEL_PIPE)
    return fail(PFLB_ERR_ARG, "unknown kernel");
  if (lz < -1) return fail(PFLB_ERR_ARG, "lz must be > 0, 0 (keep) or -1 (automatic)");
  const int nbx = bx > 0 ? bx : L->bx, nby = by > 0 ? by : L->by;
  if (nbx * nby > 256 || nbx < 1 || nby < 1 || (nbx * nby) % 32)
    return fail(PFLB_ERR_ARG, "bx*by must be a multiple of 32 in [32, 256]");
  if (2 * (nbx + 2) + 2 * nby > nbx * nby)
    return fail(PFLB_ERR_ARG, "tile too thin: halo ring larger than the block");
  L->kernel = kind;
  L->bx = nbx;
  L->by = nby;
  if (lz > 0) L->lz_req = lz;
  if (lz == -1) L->lz_req = 0;
  L->lz = resolve_lz(L);
  CK(L, ensure_wall_lists(L, L->stream));
  return PFLB_OK;
}

pflb_status pflb_set_x_boundaries(pflb_lattice *L, const pflb_xbc *lo, const pflb_xbc *hi) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  const bool on = lo || hi;
  if (on) {
    if (!lo || !hi) return fail(PFLB_ERR_ARG, "open x boundaries need both planes");
    for (const pflb_xbc *b : {lo, hi}) {
      if (b->type != PFLB_XBC_PRESSURE && b->type != PFLB_XBC_VELOCITY)
        return fail(PFLB_ERR_ARG, "boundary type must be PFLB_XBC_PRESSURE or PFLB_XBC_VELOCITY");
      if (!std::isfinite(b->P) || !std::isfinite(b->phi) || !std::isfinite(b->u[0]) ||
          !std::isfinite(b->u[1]) || !std::isfinite(b->u[2]))
        return fail(PFLB_ERR_ARG, "non-finite boundary value");
    }
    if (L->nx < 3) return fail(PFLB_ERR_ARG, "open x boundaries need nx >= 3");
    if (!L->bcm) {
      const size_t bytes = 5 * 2 * (size_t)L->ny * L->nz * compute_bytes(L->p.storage);
      cudaError_t e = cudaMalloc(&L->bcm, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        L->bcm = nullptr;
        return alloc_fail(e, "device allocation failed (boundary states)");
      }
      L->dev_bytes += (int64_t)bytes;
    }
    if (lo->ramp_steps < 0 || hi->ramp_steps < 0 || lo->ramp_steps != hi->ramp_steps)
      return fail(PFLB_ERR_ARG, "ramp_steps must be >= 0 and the same on both planes");
    // ramp start values: those in effect now (same boundary type), else the
    // rest state (P = 0, u = 0; phi at its target)
    const pflb::XbcSpec cur = pflb::xbc_spec(*L, L->step);
    const pflb_xbc *bs[2] = {lo, hi};
    for (int k = 0; k < 2; ++k) {
      const double v[5] = {bs[k]->P, bs[k]->u[0], bs[k]->u[1], bs[k]->u[2], bs[k]->phi};
      const bool same = L->bc_on && L->bc_type[k] == bs[k]->type;
      for (int q = 0; q < 5; ++q) {
        L->bc_from[k][q] = same ? pflb::xbc_value(cur, k, q, L->step) : (q < 4 ? 0.0 : v[4]);
        L->bc_val[k][q] = v[q];
      }
      L->bc_type[k] = bs[k]->type;
    }
    L->bc_t0 = L->step;
    L->bc_ramp = lo->ramp_steps;
  }
  if (on != L->bc_on) {
    CK(L, dispatch(L, [&](auto *s_, auto *r_) {
      PFLB_SR_TYPES
      return pflb::mark_xbc<S, R>(*L, on);
    }));
  }
  L->bc_on = on;
  L->lz = resolve_lz(L);  // the TMA kernel is not used with open boundaries
  CK(L, ensure_wall_lists(L, L->stream));
  return PFLB_OK;
}

pflb_status pflb_tune(pflb_lattice *L, int trial_steps, int *lz_out) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (trial_steps < 1) return fail(PFLB_ERR_ARG, "trial_steps must be >= 1");
  static const int cand[] = {-1, 4, 6, 8, 10, 12, 16, 24, 32};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  CK(L, cudaEventCreate(&t0));
  cudaError_t e = cudaEventCreate(&t1);
  if (e != cudaSuccess) {
    cudaEventDestroy(t0);
    CK(L, e);
  }
  float best_ms = 1e30f;
  int best = -1;
  pflb_status st = PFLB_OK;
  for (int c : cand) {
    if (c > L->nz) continue;
    st = pflb_set_kernel(L, L->kernel, L->bx, L->by, c);
    if (st != PFLB_OK) break;
    st = pflb_step(L, 1);  // the new depth's first launch (attributes, lists)
    if (st != PFLB_OK) break;
    e = cudaEventRecord(t0, L->stream);
    if (e == cudaSuccess) st = pflb_step(L, trial_steps);
    if (e == cudaSuccess && st == PFLB_OK) e = cudaEventRecord(t1, L->stream);
    if (e == cudaSuccess && st == PFLB_OK) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess && st == PFLB_OK) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e != cudaSuccess || st != PFLB_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != PFLB_OK) return st;
  CK(L, e);
  st = pflb_set_kernel(L, L->kernel, L->bx, L->by, best);
  if (st != PFLB_OK) return st;
  if (lz_out) *lz_out = L->lz;
  return PFLB_OK;
}

pflb_status pflb_get_kernel(const pflb_lattice *L, int out[4]) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!out) return fail(PFLB_ERR_ARG, "null output");
  const bool tma = L->kernel == PFLB_KERNEL_FUSED_TMA && L->p.storage == PFLB_STORAGE_FP32 &&
                   L->tma_ok && !L->bc_on;
  const bool pipe = pflb::pipe_kernel_runs(*L);
  // the kind that runs: the pipelined and TMA kernels fall back to the
  // fused one where they do not apply
  out[0] = pipe || tma || L->kernel == PFLB_KERNEL_TWOPASS ? L->kernel : PFLB_KERNEL_FUSED;
  out[1] = tma ? 32 : (pipe ? 32 : L->bx);
  out[2] = tma ? 8 : (pipe ? 4 : L->by);
  out[3] = L->lz;
  return PFLB_OK;
}

pflb_status pflb_step(pflb_lattice *L, int64_t nsteps) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (nsteps < 0) return fail(PFLB_ERR_ARG, "negative step count");
  for (int64_t k = 0; k < nsteps; ++k) {
    const bool d = L->diag_every > 0 && (L->step % L->diag_every) == 0;
    CK(L, do_step(L, d));
  }
  return PFLB_OK;
}

pflb_status pflb_set_diag_every(pflb_lattice *L, int every) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (every < 0) return fail(PFLB_ERR_ARG, "negative diagnostic interval");
  L->diag_every = every;
  return PFLB_OK;
}

// Reads the device error flag (synchronises): a bounded wait inside a
// kernel ran out.
static pflb_status check_device_flag(pflb_lattice *L) {
  int flag = 0;
  CK(L, cudaMemcpyAsync(&flag, L->err, sizeof flag, cudaMemcpyDeviceToHost, L->stream));
  CK(L, cudaStreamSynchronize(L->stream));
  if (flag) {
    L->poisoned = true;
    return fail(PFLB_ERR_TIMEOUT, "a bounded wait in the step kernel ran out; state is invalid");
  }
  return PFLB_OK;
}

// Raw accumulators (32 doubles, see pflb_model.cuh D_*) to the public struct.
static pflb_status decode_diag(const double *d, int64_t step, int nx, pflb_diag_t *out) {
  std::memset(out, 0, sizeof *out);
  out->step = step;
  out->mass = d[pflb::D_MASS];
  out->n_heavy = d[pflb::D_NHEAVY];
  out->n_p_heavy = d[pflb::D_NPH];
  out->n_p_light = d[pflb::D_NPL];
  out->p_heavy = d[pflb::D_NPH] > 0 ? d[pflb::D_PH] / d[pflb::D_NPH] : 0.0;
  out->p_light = d[pflb::D_NPL] > 0 ? d[pflb::D_PL] / d[pflb::D_NPL] : 0.0;
  out->dp = out->p_heavy - out->p_light;
  out->u_max = d[pflb::D_UMAX];
  out->region_mass = d[pflb::D_REGION];
  out->cl_count = d[pflb::D_CLN];
  if (out->cl_count > 0) {
    out->cl_mean[0] = d[pflb::D_CLX] / out->cl_count;
    out->cl_mean[1] = d[pflb::D_CLY] / out->cl_count;
    out->cl_mean[2] = d[pflb::D_CLZ] / out->cl_count;
    out->cl_m2[0] = d[pflb::D_CLXX] / out->cl_count;
    out->cl_m2[1] = d[pflb::D_CLYY] / out->cl_count;
    out->cl_m2[2] = d[pflb::D_CLZZ] / out->cl_count;
  }
  out->kinetic = d[pflb::D_KIN];
  out->nonfinite = d[pflb::D_NONFINITE];
  out->front_x = d[pflb::D_FRONT] > 0 ? d[pflb::D_FRONT] - 1.0 : -1.0;
  out->rear_x = d[pflb::D_REAR] > 0 ? (double)nx - d[pflb::D_REAR] : -1.0;
  if (out->nonfinite > 0 || !std::isfinite(out->mass))
    return fail(PFLB_ERR_NAN, "non-finite values in the fields");
  return PFLB_OK;
}

static pflb_status fetch_diag(pflb_lattice *L, const double *dev, pflb_diag_t *out) {
  double d[32];
  CK(L, cudaMemcpyAsync(d, dev, sizeof d, cudaMemcpyDeviceToHost, L->stream));
  pflb_status fs = check_device_flag(L);
  if (fs != PFLB_OK) return fs;
  return decode_diag(d, L->step, L->nx, out);
}

pflb_status pflb_last_diag_async(pflb_lattice *L, pflb_diag_raw_t *raw, int64_t *ticket) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!raw || !ticket) return fail(PFLB_ERR_ARG, "null output");
  if (L->ndiag == 0) return fail(PFLB_ERR_STATE, "no step has computed diagnostics yet");
  const int k = (int)(L->aticket % pflb::kAsyncReads);
  if (!L->aev[k]) CK(L, cudaEventCreateWithFlags(&L->aev[k], cudaEventDisableTiming));
  raw->step = L->last_diag_step;
  CK(L, cudaMemcpyAsync(raw->acc, L->diag + 32 * ((L->ndiag - 1) & 1), sizeof raw->acc,
                        cudaMemcpyDeviceToHost, L->stream));
  CK(L, cudaMemcpyAsync(&raw->err, L->err, sizeof raw->err, cudaMemcpyDeviceToHost, L->stream));
  CK(L, cudaEventRecord(L->aev[k], L->stream));
  *ticket = L->aticket++;
  return PFLB_OK;
}

pflb_status pflb_diag_wait(pflb_lattice *L, int64_t ticket, const pflb_diag_raw_t *raw,
                           pflb_diag_t *out) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!raw || !out) return fail(PFLB_ERR_ARG, "null argument");
  if (ticket < 0 || ticket >= L->aticket || ticket < L->aticket - pflb::kAsyncReads)
    return fail(PFLB_ERR_ARG, "ticket not outstanding (at most 16 reads in flight)");
  CK(L, cudaEventSynchronize(L->aev[ticket % pflb::kAsyncReads]));
  if (raw->err) {
    L->poisoned = true;
    return fail(PFLB_ERR_TIMEOUT, "a bounded wait in the step kernel ran out; state is invalid");
  }
  return decode_diag(raw->acc, raw->step, L->nx, out);
}

pflb_status pflb_step_ex(pflb_lattice *L, int64_t nsteps, int diag_last) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (nsteps < 0 || (diag_last && nsteps < 1)) return fail(PFLB_ERR_ARG, "bad step count");
  for (int64_t k = 0; k < nsteps; ++k) CK(L, do_step(L, diag_last && k == nsteps - 1));
  return PFLB_OK;
}

pflb_status pflb_step_diag(pflb_lattice *L, int64_t nsteps, pflb_diag_t *out) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (nsteps < 1 || !out) return fail(PFLB_ERR_ARG, "need nsteps >= 1 and an output");
  for (int64_t k = 0; k < nsteps; ++k) CK(L, do_step(L, k == nsteps - 1));
  return pflb_last_diag(L, out);
}

pflb_status pflb_last_diag(pflb_lattice *L, pflb_diag_t *out) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!out) return fail(PFLB_ERR_ARG, "null output");
  if (L->ndiag == 0) return fail(PFLB_ERR_STATE, "no step has computed diagnostics yet");
  pflb_status r = fetch_diag(L, L->diag + 32 * ((L->ndiag - 1) & 1), out);
  out->step = L->last_diag_step;
  return r;
}

pflb_status pflb_diag(pflb_lattice *L, pflb_diag_t *out) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!out) return fail(PFLB_ERR_ARG, "null output");
  CK(L, do_macro(L, false));
  return fetch_diag(L, L->diag + 64, out);
}

pflb_status pflb_read(pflb_lattice *L, int field, double *host_out) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!host_out || field < 0 || field > 5) return fail(PFLB_ERR_ARG, "bad field or output");
  if (!L->out) {
    cudaError_t e = cudaMalloc((void **)&L->out, 6 * (size_t)L->N * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      L->out = nullptr;
      return alloc_fail(e, "device allocation failed (field output)");
    }
    L->dev_bytes += 6 * L->N * 8;
  }
  CK(L, do_macro(L, true));
  CK(L, cudaMemcpyAsync(host_out, L->out + (size_t)field * L->N, (size_t)L->N * sizeof(double),
                        cudaMemcpyDeviceToHost, L->stream));
  return check_device_flag(L);
}

int64_t pflb_get_step(const pflb_lattice *L) { return L ? L->step : -1; }

int64_t pflb_device_bytes(const pflb_lattice *L) { return L ? L->dev_bytes : 0; }

int64_t pflb_estimate_bytes(const pflb_geometry *geom, int storage) {
  if (!geom || !geom->solid || geom->nx < 1 || geom->ny < 1 || geom->nz < 1) return -1;
  const long long N = (long long)geom->nx * geom->ny * geom->nz;
  if (!fractions_ok(geom)) return -1;
  const std::vector<uint32_t> all = link_masks(geom), cut = cut_masks(geom);
  long long nw = 0;
  bool has_cut = false;
  for (long long c = 0; c < N; ++c) {
    nw += (all[(size_t)c] | cut[(size_t)c]) != 0;
    has_cut = has_cut || (geom->solid_frac && !geom->solid[c] && geom->solid_frac[c] > 0.0);
  }
  return bytes_for(geom->nx, geom->ny, geom->nz, nw, storage, has_cut);
}

static const char kMagic[8] = {'P', 'F', 'L', 'B', 'C', 'K', 'P', '1'};

pflb_status pflb_save(pflb_lattice *L, const char *path) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!path) return fail(PFLB_ERR_ARG, "null path");
  const int rd = (int)(L->step & 1);
  const size_t N = (size_t)L->N, nw = (size_t)L->nw, E = L->elem;
  const size_t Rb = compute_bytes(L->p.storage);
  std::vector<char> buf;
  const size_t sizes[4] = {h_slots_of(L->p.storage) * N * E, 19 * N * E, 18 * nw * E,
                           18 * nw * Rb};
  const void *src[4] = {L->h[rd], L->g, L->wp[rd], L->ghost};
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(PFLB_ERR_ARG, std::string("cannot open ") + path);
  int64_t hdr[6] = {L->nx, L->ny, L->nz, L->nw, L->p.storage, L->step};
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof hdr, 1, f) == 1;
  for (int k = 0; k < 4 && ok; ++k) {
    try {
      buf.resize(sizes[k] ? sizes[k] : 1);
    } catch (...) {
      std::fclose(f);
      return fail(PFLB_ERR_OOM, "host allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(buf.data(), src[k], sizes[k], cudaMemcpyDeviceToHost, L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) {
      std::fclose(f);
      return cuda_fail(L, e, "checkpoint copy");
    }
    ok = std::fwrite(buf.data(), 1, sizes[k], f) == sizes[k];
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? PFLB_OK : fail(PFLB_ERR_ARG, "write failed");
}

pflb_status pflb_load(pflb_lattice *L, const char *path) {
  pflb_status s = check_lattice(L);
  if (s != PFLB_OK) return s;
  if (!path) return fail(PFLB_ERR_ARG, "null path");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(PFLB_ERR_ARG, std::string("cannot open ") + path);
  char magic[8];
  int64_t hdr[6];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0 ||
      std::fread(hdr, sizeof hdr, 1, f) != 1) {
    std::fclose(f);
    return fail(PFLB_ERR_ARG, "not a checkpoint");
  }
  if (hdr[0] != L->nx || hdr[1] != L->ny || hdr[2] != L->nz || hdr[3] != L->nw ||
      hdr[4] != L->p.storage) {
    std::fclose(f);
    return fail(PFLB_ERR_ARG, "checkpoint geometry or storage differs");
  }
  if (hdr[5] < 0) {
    std::fclose(f);
    return fail(PFLB_ERR_ARG, "checkpoint step is negative");
  }
  // Everything is read and checked on the host before any device buffer or
  // the step counter changes: a short or oversized file leaves the lattice
  // as it was.
  const int64_t step = hdr[5];
  const int rd = (int)(step & 1);
  const size_t N = (size_t)L->N, nw = (size_t)L->nw, E = L->elem;
  const size_t Rb = compute_bytes(L->p.storage);
  const size_t sizes[4] = {h_slots_of(L->p.storage) * N * E, 19 * N * E, 18 * nw * E,
                           18 * nw * Rb};
  void *dst[4] = {L->h[rd], L->g, L->wp[rd], L->ghost};
  std::vector<char> buf[4];
  for (int k = 0; k < 4; ++k) {
    try {
      buf[k].resize(sizes[k] ? sizes[k] : 1);
    } catch (...) {
      std::fclose(f);
      return fail(PFLB_ERR_OOM, "host allocation failed");
    }
    if (std::fread(buf[k].data(), 1, sizes[k], f) != sizes[k]) {
      std::fclose(f);
      return fail(PFLB_ERR_ARG, "truncated checkpoint");
    }
  }
  char extra;
  const bool trailing = std::fread(&extra, 1, 1, f) == 1;
  std::fclose(f);
  if (trailing) return fail(PFLB_ERR_ARG, "checkpoint longer than its header states");
  for (int k = 0; k < 4; ++k) {
    cudaError_t e = cudaMemcpyAsync(dst[k], buf[k].data(), sizes[k], cudaMemcpyHostToDevice,
                                    L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) return cuda_fail(L, e, "checkpoint upload");  // poisons L
  }
  L->step = step;
  return PFLB_OK;
}

// ------------------------------------------------------------- batches

static pflb_status batch_fail(pflb_batch *b, cudaError_t e, const char *what) {
  if (b) b->poisoned = true;
  return fail(PFLB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define BCK(b, call)                                         \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return batch_fail(b, e_, #call);  \
  } while (0)

static void batch_drop_graph(pflb_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// Which lattices of the batch the pipelined march can run (the others use
// the fused tile march of k_batch).
static std::vector<char> batch_pipe_set(const pflb_batch *b) {
  std::vector<char> on(b->lats.size());
  for (size_t l = 0; l < b->lats.size(); ++l) on[l] = pflb::pipe_layout_ok(*b->lats[l]) ? 1 : 0;
  return on;
}

// Work lists of the pipelined lattices (tile columns of 32 x 4 in chunks of
// plz planes, plz minimising rounds of resident blocks x (plz + 0.6) as for
// a single lattice; wall nodes in chunks of 128), and their grid.
static pflb_status batch_build_pipe_items(pflb_batch *b) {
  BCK(b, cudaStreamSynchronize(b->dev.stream));  // the old lists may still be in use
  std::vector<int4> items;
  std::vector<int2> witems;
  long long cols = 0;
  int maxz = 1;
  for (int l = 0; l < (int)b->lats.size(); ++l) {
    if (!b->pipe_set[l]) continue;
    const Lattice *L = b->lats[l];
    cols += (long long)((L->nx + 31) / 32) * ((L->ny + 3) / 4);
    maxz = std::max(maxz, L->nz);
    for (int r = 0; r < L->nw; r += 128) witems.push_back(make_int2(l, r));
  }
  const int per = dispatch_storage(b->storage, [&](auto *s_, auto *r_) {
    PFLB_SR_TYPES
    return pflb::batch_pipe_blocks_per_sm<S, R>();
  });
  const long long slots = (long long)per * b->nsm;
  int best = 8;
  double best_cost = 1e300;
  for (int lz = std::min(32, maxz); lz >= 2 && cols > 0; --lz) {
    long long blocks = 0;
    for (int l = 0; l < (int)b->lats.size(); ++l)
      if (b->pipe_set[l]) {
        const Lattice *L = b->lats[l];
        blocks += (long long)((L->nx + 31) / 32) * ((L->ny + 3) / 4) * ((L->nz + lz - 1) / lz);
      }
    const double cost = (double)((blocks + slots - 1) / slots) * (lz + 0.6);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = lz;
    }
  }
  b->dev.plz = best;
  std::vector<int4> items8;  // lattices staged in 8-byte chunks
  for (int l = 0; l < (int)b->lats.size(); ++l) {
    if (!b->pipe_set[l]) continue;
    const Lattice *L = b->lats[l];
    std::vector<int4> &dst = pflb::pipe_chunk_bytes(*L) == 8 ? items8 : items;
    for (int z0 = 0; z0 < L->nz; z0 += best)
      for (int y0 = 0; y0 < L->ny; y0 += 4)
        for (int x0 = 0; x0 < L->nx; x0 += 32) dst.push_back(make_int4(l, x0, y0, z0));
  }
  if (b->dev.pitems) cudaFree(b->dev.pitems);
  if (b->dev.pitems8) cudaFree(b->dev.pitems8);
  if (b->dev.witems) cudaFree(b->dev.witems);
  b->dev.pitems = b->dev.pitems8 = b->dev.witems = nullptr;
  b->dev.npitems = (int)items.size();
  b->dev.npitems8 = (int)items8.size();
  b->dev.nwitems = (int)witems.size();
  if (!items.empty()) {
    BCK(b, cudaMalloc(&b->dev.pitems, items.size() * sizeof(int4)));
    BCK(b, cudaMemcpyAsync(b->dev.pitems, items.data(), items.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, b->dev.stream));
  }
  if (!items8.empty()) {
    BCK(b, cudaMalloc(&b->dev.pitems8, items8.size() * sizeof(int4)));
    BCK(b, cudaMemcpyAsync(b->dev.pitems8, items8.data(), items8.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, b->dev.stream));
  }
  if (!witems.empty()) {
    BCK(b, cudaMalloc(&b->dev.witems, witems.size() * sizeof(int2)));
    BCK(b, cudaMemcpyAsync(b->dev.witems, witems.data(), witems.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, b->dev.stream));
  }
  b->dev.pgrid = (int)std::max(
      1LL, std::min<long long>(std::max(b->dev.npitems, b->dev.npitems8), slots));
  return PFLB_OK;
}

// Work list for the current launch shape, and the persistent grid size.
static pflb_status batch_build_items(pflb_batch *b) {
  b->pipe_set = batch_pipe_set(b);
  pflb_status pst = batch_build_pipe_items(b);
  if (pst != PFLB_OK) return pst;
  std::vector<int4> items;
  const int bx = b->dev.bx, by = b->dev.by, lz = b->dev.lz;
  for (int l = 0; l < (int)b->lats.size(); ++l) {
    if (b->pipe_set[l]) continue;
    const Lattice *L = b->lats[l];
    for (int z0 = 0; z0 < L->nz; z0 += lz)
      for (int y0 = 0; y0 < L->ny; y0 += by)
        for (int x0 = 0; x0 < L->nx; x0 += bx) items.push_back(make_int4(l, x0, y0, z0));
  }
  if (items.size() > b->items_cap) {
    if (b->dev.items) cudaFree(b->dev.items);
    b->dev.items = nullptr;
    BCK(b, cudaMalloc(&b->dev.items, items.size() * sizeof(int4)));
    b->items_cap = items.size();
  }
  b->dev.nitems = (int)items.size();
  if (!items.empty())
    BCK(b, cudaMemcpyAsync(b->dev.items, items.data(), items.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, b->dev.stream));
  const int fit = dispatch_storage(b->storage, [&](auto *s_, auto *r_) {
    PFLB_SR_TYPES
    return pflb::batch_max_blocks_per_sm<S, R>(bx, by);
  });
  b->per_sm = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, fit) : std::min(fit, 4);
  b->dev.grid = std::max(1, std::min(b->dev.nitems, b->per_sm * b->nsm));
  batch_drop_graph(b);
  BCK(b, cudaStreamSynchronize(b->dev.stream));
  return PFLB_OK;
}

extern "C" pflb_status pflb_batch_create(pflb_lattice *const *lattices, int count, void *cuda_stream,
                                         pflb_batch **out) {
  if (!out) return fail(PFLB_ERR_ARG, "null out");
  *out = nullptr;
  if (!lattices || count < 1) return fail(PFLB_ERR_ARG, "need at least one lattice");
  for (int l = 0; l < count; ++l) {
    pflb_status st = check_lattice(lattices[l]);
    if (st != PFLB_OK) return st;
    if (lattices[l]->p.storage != lattices[0]->p.storage)
      return fail(PFLB_ERR_ARG, "all lattices of a batch need the same storage");
    for (int k = 0; k < l; ++k)
      if (lattices[k] == lattices[l]) return fail(PFLB_ERR_ARG, "a lattice appears twice");
  }
  pflb_batch *b = new (std::nothrow) pflb_batch();
  if (!b) return fail(PFLB_ERR_OOM, "host allocation failed");
  for (int l = 0; l < count; ++l) b->lats.push_back(lattices[l]);
  b->storage = lattices[0]->p.storage;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (b->nsm < 1) b->nsm = 1;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->dev.stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->dev.stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  b->desc_bytes = dispatch_storage(b->storage, [&](auto *s_, auto *r_) {
    PFLB_SR_TYPES
    return pflb::batch_desc_bytes<S, R>();
  });
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->dev.descs, 2 * (size_t)count * b->desc_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->dev.par0, count * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->dev.counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->dev.pcounter, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->dev.bstep, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->dev.xspecs, count * sizeof(pflb::XbcSpec));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->dev.xlist, count * sizeof(int));
  if (e != cudaSuccess) {
    pflb_batch_destroy(b);
    cudaGetLastError();
    return alloc_fail(e, "batch allocation failed");
  }
  pflb_status st = batch_build_items(b);
  if (st != PFLB_OK) {
    pflb_batch_destroy(b);
    return st;
  }
  *out = b;
  return PFLB_OK;
}

extern "C" pflb_status pflb_batch_set_launch(pflb_batch *b, int bx, int by, int lz,
                                             int blocks_per_sm) {
  if (!b) return fail(PFLB_ERR_ARG, "null batch");
  if (b->poisoned) return fail(PFLB_ERR_STATE, "batch poisoned by an earlier CUDA error");
  const int nbx = bx > 0 ? bx : b->dev.bx, nby = by > 0 ? by : b->dev.by;
  const int nlz = lz > 0 ? lz : b->dev.lz;
  if (nbx < 1 || nby < 1 || nbx * nby > 256 || (nbx * nby) % 32 ||
      2 * (nbx + 2) + 2 * nby > nbx * nby || blocks_per_sm < 0)
    return fail(PFLB_ERR_ARG, "bad launch shape (bx*by a multiple of 32 in [32, 256], halo "
                              "ring no larger than the block)");
  b->dev.bx = nbx;
  b->dev.by = nby;
  b->dev.lz = nlz;
  b->blocks_per_sm = blocks_per_sm;
  return batch_build_items(b);
}

// Runs nsteps on the batch stream (graph replay for the plain steps).
static pflb_status batch_run(pflb_batch *b, int64_t nsteps, bool diag_last) {
  const int n = (int)b->lats.size();
  // open boundaries switched on or off since the work lists were built
  // move a lattice between the pipelined and the fused march
  if (batch_pipe_set(b) != b->pipe_set) {
    pflb_status st = batch_build_items(b);
    if (st != PFLB_OK) return st;
  }
  // order after every lattice's own stream
  for (Lattice *L : b->lats) {
    if (L->stream == b->dev.stream) continue;
    BCK(b, cudaEventRecord(b->ev, L->stream));
    BCK(b, cudaStreamWaitEvent(b->dev.stream, b->ev, 0));
  }
  std::vector<char> host(2 * (size_t)n * b->desc_bytes);
  std::vector<int> par(n);
  dispatch_storage(b->storage, [&](auto *s_, auto *r_) {
    PFLB_SR_TYPES
    pflb::batch_build_descs<S, R>(b->lats.data(), n, host.data());
    return 0;
  });
  for (int l = 0; l < n; ++l) par[l] = (int)(b->lats[l]->step & 1);
  // parities the pipelined lattices start this call at (one march launch
  // per parity present at each step)
  int pmask = 0;
  for (int l = 0; l < n; ++l)
    if (b->pipe_set[l]) pmask |= 1 << par[l];
  b->dev.pmask = pmask;
  if (pmask != b->graph_pmask) batch_drop_graph(b);
  // open x boundaries: specs of every lattice (type 0 = periodic) and the
  // list of those that have them; the values may change between calls
  std::vector<pflb::XbcSpec> specs(n);
  std::vector<int> xlist;
  for (int l = 0; l < n; ++l) {
    const Lattice *L = b->lats[l];
    specs[l] = pflb::xbc_spec(*L, L->step);
    if (L->bc_on) xlist.push_back(l);
  }
  b->dev.nxbc = (int)xlist.size();
  if (b->dev.nxbc != b->graph_nxbc) batch_drop_graph(b);
  BCK(b, cudaMemcpyAsync(b->dev.xspecs, specs.data(), n * sizeof(pflb::XbcSpec),
                         cudaMemcpyHostToDevice, b->dev.stream));
  if (!xlist.empty())
    BCK(b, cudaMemcpyAsync(b->dev.xlist, xlist.data(), xlist.size() * sizeof(int),
                           cudaMemcpyHostToDevice, b->dev.stream));
  BCK(b, cudaMemcpyAsync(b->dev.descs, host.data(), host.size(), cudaMemcpyHostToDevice,
                         b->dev.stream));
  BCK(b, cudaMemcpyAsync(b->dev.par0, par.data(), n * sizeof(int), cudaMemcpyHostToDevice,
                         b->dev.stream));
  BCK(b, cudaMemsetAsync(b->dev.bstep, 0, sizeof(int), b->dev.stream));
  // tpar: parity of the batch step (the device counter bstep starts at 0
  // with each call and advances by one per step)
  auto launch = [&](bool diag, int tpar) {
    return dispatch_storage(b->storage, [&](auto *s_, auto *r_) {
      PFLB_SR_TYPES
      return pflb::batch_launch_step<S, R>(b->dev, diag, tpar);
    });
  };
  int64_t plain = nsteps - (diag_last ? 1 : 0);
  int64_t t = 0;
  if (plain >= kGraphSteps && !b->graph) {
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->dev.stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = launch(false, k & 1);
    cudaError_t e2 = cudaStreamEndCapture(b->dev.stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_fail(b, e, "graph capture");
    b->graph_nxbc = b->dev.nxbc;
    b->graph_pmask = b->dev.pmask;
  }
  // replays come first, so each starts at an even batch step (kGraphSteps
  // is even), as the captured parities assume
  while (plain >= kGraphSteps) {
    BCK(b, cudaGraphLaunch(b->graph, b->dev.stream));
    plain -= kGraphSteps;
    t += kGraphSteps;
  }
  for (; plain > 0; --plain, ++t) BCK(b, launch(false, (int)(t & 1)));
  if (diag_last) BCK(b, launch(true, (int)(t & 1)));
  for (Lattice *L : b->lats) {
    L->step += nsteps;
    if (diag_last) {
      L->last_diag_step = L->step - 1;
      L->ndiag++;
    }
  }
  // later work on each lattice's own stream comes after the batch
  BCK(b, cudaEventRecord(b->ev, b->dev.stream));
  for (Lattice *L : b->lats)
    if (L->stream != b->dev.stream) BCK(b, cudaStreamWaitEvent(L->stream, b->ev, 0));
  return PFLB_OK;
}

extern "C" pflb_status pflb_batch_step(pflb_batch *b, int64_t nsteps, int diag_last) {
  if (!b) return fail(PFLB_ERR_ARG, "null batch");
  if (b->poisoned) return fail(PFLB_ERR_STATE, "batch poisoned by an earlier CUDA error");
  if (nsteps < 0 || (diag_last && nsteps < 1)) return fail(PFLB_ERR_ARG, "bad step count");
  for (Lattice *L : b->lats)
    if (L->poisoned) return fail(PFLB_ERR_STATE, "a lattice of the batch is poisoned");
  if (nsteps == 0) return PFLB_OK;
  return batch_run(b, nsteps, diag_last != 0);
}

extern "C" pflb_status pflb_batch_tune(pflb_batch *b, int trial_steps, int best[4]) {
  if (!b) return fail(PFLB_ERR_ARG, "null batch");
  if (b->poisoned) return fail(PFLB_ERR_STATE, "batch poisoned by an earlier CUDA error");
  if (trial_steps < 1) return fail(PFLB_ERR_ARG, "trial_steps must be >= 1");
  static const int cand[][4] = {{32, 4, 16, 0}, {32, 4, 8, 0}, {32, 8, 16, 2}, {32, 8, 8, 2},
                                {16, 8, 16, 0}, {64, 4, 16, 2}, {32, 4, 32, 0}, {16, 16, 8, 2}};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  BCK(b, cudaEventCreate(&t0));
  BCK(b, cudaEventCreate(&t1));
  float best_ms = 1e30f;
  int bi = 0;
  for (int k = 0; k < (int)(sizeof cand / sizeof cand[0]); ++k) {
    pflb_status st = pflb_batch_set_launch(b, cand[k][0], cand[k][1], cand[k][2], cand[k][3]);
    if (st != PFLB_OK) continue;
    st = batch_run(b, 1, false);  // warm the new shape
    if (st != PFLB_OK) return st;
    BCK(b, cudaEventRecord(t0, b->dev.stream));
    st = batch_run(b, trial_steps, false);
    if (st != PFLB_OK) return st;
    BCK(b, cudaEventRecord(t1, b->dev.stream));
    BCK(b, cudaEventSynchronize(t1));
    float ms = 0;
    BCK(b, cudaEventElapsedTime(&ms, t0, t1));
    if (ms < best_ms) { best_ms = ms; bi = k; }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  pflb_status st = pflb_batch_set_launch(b, cand[bi][0], cand[bi][1], cand[bi][2], cand[bi][3]);
  if (st != PFLB_OK) return st;
  if (best)
    for (int k = 0; k < 4; ++k) best[k] = k < 3 ? cand[bi][k] : b->per_sm;
  return PFLB_OK;
}

extern "C" void pflb_batch_destroy(pflb_batch *b) {
  if (!b) return;
  if (b->dev.stream) cudaStreamSynchronize(b->dev.stream);
  batch_drop_graph(b);
  void *ptrs[] = {b->dev.descs,   b->dev.par0,   b->dev.items,  b->dev.counter,
                  b->dev.bstep,   b->dev.xspecs, b->dev.xlist,  b->dev.pitems,
                  b->dev.pitems8, b->dev.witems, b->dev.pcounter};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->own_stream && b->dev.stream) cudaStreamDestroy(b->dev.stream);
  delete b;
}

void pflb_destroy(pflb_lattice *L) {
  if (!L) return;
  cudaStreamSynchronize(L->stream);
  free_all(L);
  delete L;
}

const char *pflb_last_error(void) { return g_err.c_str(); }

}  // extern "C"
