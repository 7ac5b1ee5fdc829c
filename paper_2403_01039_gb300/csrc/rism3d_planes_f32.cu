// FP32 instantiation of the plane-pass kernels (fused and split forms; templates in
// rism3d_kernels.cuh).
#include "rism3d_kernels.cuh"

namespace rism {
RISM_INSTANTIATE_PLANES(float)
}  // namespace rism
