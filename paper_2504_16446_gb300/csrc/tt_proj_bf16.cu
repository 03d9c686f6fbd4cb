// tt_proj_bf16.cu -- projector kernels with float arithmetic and __nv_bfloat16 storage of
// the coefficient volume and of the back-contracted residual.
#include "tt_kernels.cuh"

namespace tt {
TT_INSTANTIATE_PROJECTORS(float, __nv_bfloat16)
}  // namespace tt
