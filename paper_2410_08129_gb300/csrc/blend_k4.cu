// blend_k4.cu -- forward blend with a 4-entry register core (instantiation unit).
#include "blend_impl.cuh"

namespace htgs {

bool blend_fwd_k4(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s) {
    if (ppt == 1) return dispatch_shape_fwd<4, 1>(b, a, s);
    if (ppt == 2) return dispatch_shape_fwd<4, 2>(b, a, s);
    if (ppt == 4) return dispatch_shape_fwd<4, 4>(b, a, s);
    return dispatch_shape_fwd<4, 1>(b, a, s);
}

} // namespace htgs
