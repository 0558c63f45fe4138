// blend_k32.cu -- forward blend with a 32-entry register core (instantiation unit).
#include "blend_impl.cuh"

namespace htgs {

bool blend_fwd_k32(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s) {
    if (ppt == 1) return dispatch_shape_fwd<32, 1>(b, a, s);
    return dispatch_shape_fwd<32, 1>(b, a, s);
}

} // namespace htgs
