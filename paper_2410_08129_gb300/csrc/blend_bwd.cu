// blend_bwd.cu -- the blend adjoint (instantiation unit): one persistent
// kernel per tile shape, core size at run time, per-pixel state in dynamic
// shared memory.
#include "blend_impl.cuh"

namespace htgs {

namespace {

template <int TW, int TH>
bool run_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    const size_t smem = bwd_smem_bytes(TW * TH, a.prm.K);
    if (!allow_dynamic_smem((const void *)blend_bwd_kernel<TW, TH>, bwd_smem_bytes(TW * TH, HTGS_MAX_K)))
        return false;
    const int grid = persistent_grid((const void *)blend_bwd_kernel<TW, TH>, kBwdThreads, smem, a.max_items);
    blend_bwd_kernel<TW, TH><<<grid, kBwdThreads, smem, s>>>(b, a);
    return true;
}

} // namespace

bool launch_blend_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    if (a.prm.K < 0 || a.prm.K > HTGS_MAX_K) return false;
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return run_bwd<16, 16>(b, a, s);
    if (tw == 16 && th == 8) return run_bwd<16, 8>(b, a, s);
    if (tw == 8 && th == 8) return run_bwd<8, 8>(b, a, s);
    return false;
}

} // namespace htgs
