// blend_notail.cu -- forward blend for inference without the tail (the core
// composited over the background; instantiation unit). One pixel per thread:
// the launch's px_per_thread only changes the schedule, not the result.
#include "blend_impl.cuh"

namespace htgs {

bool blend_fwd_notail(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    const int K = a.prm.K;
    if (K <= 4) return dispatch_shape_fwd<4, 1, true>(b, a, s);
    if (K <= 8) return dispatch_shape_fwd<8, 1, true>(b, a, s);
    if (K <= 16) return dispatch_shape_fwd<16, 1, true>(b, a, s);
    if (K <= 32) return dispatch_shape_fwd<32, 1, true>(b, a, s);
    return false;
}

} // namespace htgs
