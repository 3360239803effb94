// FP32 storage and arithmetic.
#include "pflb_launch.cuh"
namespace pflb {
PFLB_INSTANTIATE(float, float)
}
