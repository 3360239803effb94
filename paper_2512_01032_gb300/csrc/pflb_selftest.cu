// pflb_selftest.cu -- exercise of the failure-detection path of the staged
// step kernel without a fault: a one-block kernel waits, through the same
// bounded-wait helper the step kernel uses for its TMA stages, on an
// mbarrier that nothing ever completes.  The wait runs out after the given
// number of polls, raises the lattice's device error flag and returns, so
// the GPU context stays usable; the lattice then reports PFLB_ERR_TIMEOUT
// at its next synchronising call, exactly as after a stalled copy.
#include <cuda_runtime.h>

#include <string>

#include "../../include/pflb.h"
#include "pflb_async.cuh"
#include "pflb_internal.h"

namespace {

__global__ void k_wait_nothing(int *err, unsigned long long polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    pflb::mbar_init(&bar, 1);  // one arrival expected, none will come
    pflb::fence_mbar_init();
    pflb::bounded_wait(&bar, 0, err, polls);
  }
}

}  // namespace

extern "C" pflb_status pflb_selftest_wait_timeout(pflb_lattice *L, int64_t polls) {
  if (!L) {
    pflb::set_last_error("null lattice");
    return PFLB_ERR_ARG;
  }
  if (polls < 1 || polls > (1LL << 20)) {
    pflb::set_last_error("polls must be in [1, 2^20]");
    return PFLB_ERR_ARG;
  }
  k_wait_nothing<<<1, 32, 0, L->stream>>>(L->err, (unsigned long long)polls);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    pflb::set_last_error((std::string("launch: ") + cudaGetErrorString(e)).c_str());
    return PFLB_ERR_CUDA;
  }
  return PFLB_OK;
}
