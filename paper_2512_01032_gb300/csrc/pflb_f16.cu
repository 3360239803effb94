// FP16 storage of scaled population deviations, FP32 arithmetic.
#include "pflb_launch.cuh"
namespace pflb {
PFLB_INSTANTIATE(__half, float)
}
