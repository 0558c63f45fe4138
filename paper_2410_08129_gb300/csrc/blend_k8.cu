// blend_k8.cu -- forward blend with a 8-entry register core (instantiation unit).
#include "blend_impl.cuh"

namespace htgs {

bool blend_fwd_k8(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s) {
    if (ppt == 1) return dispatch_shape_fwd<8, 1>(b, a, s);
    if (ppt == 2) return dispatch_shape_fwd<8, 2>(b, a, s);
    if (ppt == 4) return dispatch_shape_fwd<8, 4>(b, a, s);
    return dispatch_shape_fwd<8, 1>(b, a, s);
}

} // namespace htgs
