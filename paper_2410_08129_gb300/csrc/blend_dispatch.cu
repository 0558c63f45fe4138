// blend_dispatch.cu -- picks the compiled core size for the runtime K.
#include "kernels.cuh"

namespace htgs {

bool blend_fwd_k4(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s);
bool blend_fwd_k8(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s);
bool blend_fwd_k16(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s);
bool blend_fwd_k32(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s);
bool blend_fwd_notail(const Batch &b, const BlendFwdArgs &a, cudaStream_t s);

bool launch_blend_fwd(const Batch &b, const BlendFwdArgs &a, int ppt, cudaStream_t s) {
    const int K = a.prm.K;
    if (a.prm.no_tail) return blend_fwd_notail(b, a, s);
    if (K <= 4) return blend_fwd_k4(b, a, ppt, s);
    if (K <= 8) return blend_fwd_k8(b, a, ppt, s);
    if (K <= 16) return blend_fwd_k16(b, a, ppt, s);
    if (K <= 32) return blend_fwd_k32(b, a, ppt, s);
    return false;
}

} // namespace htgs
