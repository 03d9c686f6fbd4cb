// tt_proj_f32.cu -- projector kernels with float arithmetic and float storage of
// the coefficient volume and of the back-contracted residual.
#include "tt_kernels.cuh"

namespace tt {
TT_INSTANTIATE_PROJECTORS(float, float)
}  // namespace tt
