// tt_proj_f64.cu -- double instantiations of the projector kernels.
#include "tt_kernels.cuh"

namespace tt {

template <>
cudaError_t launch_forward<double>(tt_handle *h, double *Iout, const double *I, const double *W, bool grad)
{
#define TT_CALL(L) launch_forward_L<double, L>(h, Iout, I, W, grad)
    TT_DISPATCH_L(h->L, TT_CALL)
#undef TT_CALL
}

template <>
cudaError_t launch_backcontract<double>(tt_handle *h, const double *R, double *G)
{
#define TT_CALL(L) launch_backcontract_L<double, L>(h, R, G)
    TT_DISPATCH_L(h->L, TT_CALL)
#undef TT_CALL
}

template <>
cudaError_t launch_adjoint<double>(tt_handle *h, const double *G, double *g)
{
#define TT_CALL(L) launch_adjoint_L<double, L>(h, G, g)
    TT_DISPATCH_L(h->L, TT_CALL)
#undef TT_CALL
}

}  // namespace tt
