// tt_proj_f16.cu -- projector kernels with float arithmetic and __half storage of
// the coefficient volume and of the back-contracted residual.
#include "tt_kernels.cuh"

namespace tt {
TT_INSTANTIATE_PROJECTORS(float, __half)
}  // namespace tt
