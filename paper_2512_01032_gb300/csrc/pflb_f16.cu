// FP16 storage of the weight-scaled populations (h_i / w_i, g_i / w_i), FP32 arithmetic.
#include "pflb_launch.cuh"
namespace pflb {
PFLB_INSTANTIATE(__half, float)
}
