// BF16 storage of the populations (value itself), FP32 arithmetic.
#include "pflb_launch.cuh"
namespace pflb {
PFLB_INSTANTIATE(__nv_bfloat16, float)
}
