// pflb_batch.cuh -- one persistent kernel advancing many lattices.
//
// Work list: one item per (lattice, tile column, z chunk), as int4
// (lattice, x0, y0, z0).  A grid of (SMs x blocks per SM) blocks pulls items
// from an atomic counter until the list is exhausted; each item copies its
// lattice's step descriptor (Args, both A-A parities precomputed on the
// host) into shared memory and runs the same tile march as the single-lattice
// fused kernel, so every cell sees exactly the arithmetic of a lattice
// stepped alone.  The parity of lattice l at batch step t is
// (par0[l] + t) & 1, with t read from a device counter that a one-thread
// kernel advances after each step, so a captured CUDA graph of several steps
// replays correctly.
#pragma once
#include "pflb_kernels.cuh"

namespace pflb {

__host__ __device__ constexpr size_t batch_align16(size_t b) { return (b + 15) & ~size_t(15); }

// phi ring, per-thread diagnostic slots (diagnostic launches only), step
// descriptor
template <class S, class R>
__host__ __device__ constexpr size_t batch_smem(int BX, int BY, bool diag) {
  return fused_smem_bytes<R>(BX, BY, diag) + sizeof(Args<S, R>);
}

template <class S, class R, bool DIAG, bool XBC = false>
__global__ void __launch_bounds__(256, PFLB_MIN_BLOCKS)
    k_batch(const Args<S, R> *__restrict__ descs, const int *__restrict__ par0,
            const int4 *__restrict__ items, int nitems, int *counter, const int *bstep, int BX,
            int BY, int LZ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sphi = reinterpret_cast<R *>(smem_raw);
  R *tacc = reinterpret_cast<R *>(smem_raw + fused_phi_bytes<R>(BX, BY));
  Args<S, R> *sa = reinterpret_cast<Args<S, R> *>(smem_raw + fused_smem_bytes<R>(BX, BY, DIAG));
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
    const int *src = reinterpret_cast<const int *>(descs + 2 * it.x + p);
    int *dst = reinterpret_cast<int *>(sa);
    for (int k = tid; k < (int)(sizeof(Args<S, R>) / 4); k += blockDim.x) dst[k] = src[k];
    if (DIAG) diag_thread_zero(tacc);
    __syncthreads();
    const Args<S, R> &a = *sa;
    if (DIAG && it.y == 0 && it.z == 0 && it.w == 0 && tid < 32 && a.diag_zero)
      a.diag_zero[tid] = 0.0;
    const int ze = min(it.w + LZ, a.nz);
    if (p)
      march_tile<S, R, true, DIAG, XBC>(a, it.y, it.z, it.w, ze, BX, BY, sphi, tacc);
    else
      march_tile<S, R, false, DIAG, XBC>(a, it.y, it.z, it.w, ze, BX, BY, sphi, tacc);
    if (DIAG) diag_thread_flush(a.diag, tacc, wacc);
    __syncthreads();  // shared descriptor and phi ring are reused by the next item
  }
}

// Boundary states of the open-boundary lattices of a batch (blockIdx.x:
// lattice in xlist; blockIdx.y: a strided share of its boundary cells), for
// the parity each lattice has at this batch step.
template <class S, class R>
__global__ void k_batch_xbc(const Args<S, R> *__restrict__ descs, const int *__restrict__ par0,
                            const int *__restrict__ xlist, const XbcSpec *__restrict__ specs,
                            const int *bstep) {
  const int l = xlist[blockIdx.x];
  const int p = (par0[l] + *bstep) & 1;
  const Args<S, R> &a = descs[2 * l + p];
  const XbcSpec &sp = specs[l];
  const int n = 2 * a.ny * a.nz;
  const int stride = blockDim.x * gridDim.y;
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < n; j += stride) {
    if (p)
      xbc_cell<S, R, true>(a, sp, a.bcm, j, sp.step0 + *bstep);
    else
      xbc_cell<S, R, false>(a, sp, a.bcm, j, sp.step0 + *bstep);
  }
}

// static: the header is included by several translation units.
static __global__ void k_batch_tick(int *bstep) { *bstep += 1; }

}  // namespace pflb
