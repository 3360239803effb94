// pflb_noalloc.cu -- macroscopic fields and diagnostics of caller-owned
// population arrays without any device allocation (pflb_fields_noalloc).
//
// Some callers cannot allocate device memory: their device memory belongs
// to another allocator (a framework's memory pool that must see every
// byte), or they run in a latency-critical loop where cudaMalloc's implicit
// device synchronisation is not acceptable.  This entry point takes the
// populations and the output buffer from the caller and keeps its own
// scratch (the phi field and the FP64 diagnostic accumulators) in
// file-scope device arrays of a fixed maximum size, so it never calls
// cudaMalloc, cudaFree or any allocating library routine.
//
// It is a variant of the field/diagnostic pass of the library (phi pass,
// then the per-cell macroscopic recovery with the FP64 block reductions),
// restricted to wall-free periodic lattices at FP32 storage.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pflb.h"
#include "pflb_kernels.cuh"
#include "pflb_launch.cuh"

namespace {

// Largest lattice the scratch holds: 2^20 cells (4 MiB of phi).  Every GPU
// that loads the library keeps these arrays until the process exits.
constexpr long long kMaxCells = 1LL << 20;

static __device__ __align__(256) float g_phi_scratch[kMaxCells];
static __device__ __align__(256) double g_diag_scratch[32];

// Host-side handles of the scratch arrays.  In host code the array names
// are host stand-ins, not device addresses: the real addresses come from
// cudaGetSymbolAddress, once per device, with that device current.
struct DevScratch {
  float *phi = nullptr;
  double *diag = nullptr;
  bool ready = false;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
DevScratch g_dev[kMaxDevices];
pflb_status na_fail(pflb_status s, const std::string &m) {
  pflb::set_last_error(m.c_str());  // reported by pflb_last_error()
  return s;
}

pflb_status scratch_for_current_device(DevScratch *&out, std::string &err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return PFLB_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device ordinal out of range";
    return PFLB_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  DevScratch &d = g_dev[dev];
  if (!d.ready) {
    e = cudaGetSymbolAddress((void **)&d.phi, g_phi_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&d.diag, g_diag_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return PFLB_ERR_CUDA;
    }
    d.ready = true;
  }
  out = &d;
  return PFLB_OK;
}

// phi = sum_i h_i into the scratch field (wall-free lattice).
__global__ void k_na_phi(const float *__restrict__ h, int N, float *__restrict__ phi) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < pflb::Q; ++i) s += h[(long long)i * N + c];
  phi[c] = s;
}

// Per cell: stencil from the scratch phi, g in natural layout (slot i holds
// the population arriving in direction i), macroscopic recovery, optional
// field output, diagnostics reduced into the scratch accumulators.
__global__ void __launch_bounds__(256)
    k_na_fields(int nx, int ny, int nz, const float *__restrict__ g, const float *__restrict__ phi,
                const pflb::Model<float> m, double *fields, double *diag) {
  using namespace pflb;
  using R = float;
  __shared__ R wacc[DIAG_MAX_WARPS][32];
  diag_block_zero(wacc);
  __syncthreads();
  const int N = nx * ny * nz;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  DiagAcc<R> acc;
  acc.zero();
  if (c < N) {
    const int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
    Nbr nb;
    nb.init(x, y, z, nx, ny, nz);
    R val[Q], gg[Q];
    val[0] = phi[c];
#pragma unroll
    for (int i = 1; i < Q; ++i) val[i] = phi[c + nb.off(i)];
#pragma unroll
    for (int k = 0; k < Q; ++k) gg[k] = g[(long long)k * N + c];
    R gx, gy, gz, lap;
    cd_stencil(val, gx, gy, gz, lap);
    const Macro<R> mc = macros(m, gg, val[0], gx, gy, gz, lap);
    const R p = val[0];
    acc.v[D_MASS] = p;
    acc.v[D_NHEAVY] = p >= R(0.5) ? R(1) : R(0);
    if (p > R(0.95)) { acc.v[D_PH] = mc.P; acc.v[D_NPH] = R(1); }
    if (p < R(0.05)) { acc.v[D_PL] = mc.P; acc.v[D_NPL] = R(1); }
    acc.v[D_REGION] = p;
    const R u2 = mc.ux * mc.ux + mc.uy * mc.uy + mc.uz * mc.uz;
    acc.v[D_KIN] = R(0.5) * mc.rho * u2;
    if (!finite_(p + mc.P + u2)) acc.v[D_NONFINITE] = R(1);
    acc.umax = u2;
    if (fields) {
      fields[c] = (double)p;
      fields[(long long)N + c] = (double)mc.rho;
      fields[2LL * N + c] = (double)mc.P;
      fields[3LL * N + c] = (double)mc.ux;
      fields[4LL * N + c] = (double)mc.uy;
      fields[5LL * N + c] = (double)mc.uz;
    }
  }
  diag_warp_add(wacc[threadIdx.x >> 5], acc);
  diag_block_flush(diag, wacc);
}

}  // namespace

extern "C" pflb_status pflb_fields_noalloc(int nx, int ny, int nz, const float *h_dev,
                                           const float *g_dev, const pflb_params *params,
                                           double *fields_dev, pflb_diag_t *diag_out,
                                           void *cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1) return na_fail(PFLB_ERR_ARG, "dimensions must be >= 1");
  const long long N = (long long)nx * ny * nz;
  if (N > kMaxCells)
    return na_fail(PFLB_ERR_ARG, "lattice has " + std::to_string(N) +
                                     " cells; pflb_fields_noalloc handles at most " +
                                     std::to_string(kMaxCells));
  if (!h_dev || !g_dev || !params) return na_fail(PFLB_ERR_ARG, "null populations or params");
  if (!fields_dev && !diag_out) return na_fail(PFLB_ERR_ARG, "nothing to compute: no output");
  if (!(params->W > 0) || !(params->rho_L > 0) || !(params->rho_H > 0))
    return na_fail(PFLB_ERR_ARG, "need W, rho_L, rho_H > 0");
  if (params->storage != PFLB_STORAGE_FP32)
    return na_fail(PFLB_ERR_ARG, "pflb_fields_noalloc reads FP32 populations only "
                                 "(params->storage must be PFLB_STORAGE_FP32)");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (diag_out) {
    // The diagnostic form copies to pageable host memory and waits for the
    // stream; on a stream under capture that would invalidate the capture,
    // so it is refused before anything is enqueued.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(st, &cs);
    if (ce != cudaSuccess)
      return na_fail(PFLB_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (cs != cudaStreamCaptureStatusNone)
      return na_fail(PFLB_ERR_ARG, "diag_out needs a stream that is not being captured");
  }
  DevScratch *sc = nullptr;
  std::string err;
  pflb_status s = scratch_for_current_device(sc, err);
  if (s != PFLB_OK) return na_fail(s, err);
  // The accumulators keep the previous call's contents: clear them.
  cudaError_t e = cudaMemsetAsync(sc->diag, 0, 32 * sizeof(double), st);
  const pflb::Model<float> m = pflb::make_model<float>(*params);
  const int T = 256;
  const unsigned B = (unsigned)((N + T - 1) / T);
  if (e == cudaSuccess) {
    k_na_phi<<<B, T, 0, st>>>(h_dev, (int)N, sc->phi);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_na_fields<<<B, T, 0, st>>>(nx, ny, nz, g_dev, sc->phi, m, fields_dev, sc->diag);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return na_fail(PFLB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (!diag_out) return PFLB_OK;
  double d[32];
  e = cudaMemcpyAsync(d, sc->diag, sizeof d, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(PFLB_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
  using namespace pflb;
  std::memset(diag_out, 0, sizeof *diag_out);
  diag_out->step = -1;
  diag_out->mass = d[D_MASS];
  diag_out->n_heavy = d[D_NHEAVY];
  diag_out->n_p_heavy = d[D_NPH];
  diag_out->n_p_light = d[D_NPL];
  diag_out->p_heavy = d[D_NPH] > 0 ? d[D_PH] / d[D_NPH] : 0.0;
  diag_out->p_light = d[D_NPL] > 0 ? d[D_PL] / d[D_NPL] : 0.0;
  diag_out->dp = diag_out->p_heavy - diag_out->p_light;
  diag_out->u_max = d[D_UMAX];
  diag_out->region_mass = d[D_REGION];
  diag_out->kinetic = d[D_KIN];
  diag_out->nonfinite = d[D_NONFINITE];
  diag_out->front_x = -1.0;  // not computed by this pass
  diag_out->rear_x = -1.0;
  if (diag_out->nonfinite > 0 || !std::isfinite(diag_out->mass))
    return na_fail(PFLB_ERR_NAN, "non-finite values in the fields");
  return PFLB_OK;
}
