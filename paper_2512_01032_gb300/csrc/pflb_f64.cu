// FP64 storage and arithmetic (parity path).
#include "pflb_launch.cuh"
namespace pflb {
PFLB_INSTANTIATE(double, double)
}
