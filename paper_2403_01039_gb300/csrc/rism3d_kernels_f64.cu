// FP64 instantiation of the solver kernels (the templates are in rism3d_kernels.cuh); the two
// precisions are separate translation units so that they compile in parallel.
#include "rism3d_kernels.cuh"

namespace rism {
RISM_INSTANTIATE(double)
}  // namespace rism
