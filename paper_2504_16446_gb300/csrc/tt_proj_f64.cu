// tt_proj_f64.cu -- projector kernels with double arithmetic and double storage of
// the coefficient volume and of the back-contracted residual.
#include "tt_kernels.cuh"

namespace tt {
TT_INSTANTIATE_PROJECTORS(double, double)
}  // namespace tt
