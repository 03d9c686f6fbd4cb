// tt_proj_f32.cu -- float instantiations of the projector kernels.
#include "tt_kernels.cuh"

namespace tt {

template <>
cudaError_t launch_forward<float>(tt_handle *h, float *Iout, const float *I, const float *W, bool grad)
{
#define TT_CALL(L) launch_forward_L<float, L>(h, Iout, I, W, grad)
    TT_DISPATCH_L(h->L, TT_CALL)
#undef TT_CALL
}

template <>
cudaError_t launch_backcontract<float>(tt_handle *h, const float *R, float *G)
{
#define TT_CALL(L) launch_backcontract_L<float, L>(h, R, G)
    TT_DISPATCH_L(h->L, TT_CALL)
#undef TT_CALL
}

template <>
cudaError_t launch_adjoint<float>(tt_handle *h, const float *G, float *g)
{
#define TT_CALL(L) launch_adjoint_L<float, L>(h, G, g)
    TT_DISPATCH_L(h->L, TT_CALL)
#undef TT_CALL
}

}  // namespace tt
