// FP32 instantiation of the solver kernels other than the plane passes (the templates are
// in rism3d_kernels.cuh; the plane passes are in rism3d_planes_f32.cu), so that the units
// compile in parallel.
#include "rism3d_kernels.cuh"

namespace rism {
RISM_EXTERN_PLANES(float)
RISM_INSTANTIATE_REST(float)
}  // namespace rism
