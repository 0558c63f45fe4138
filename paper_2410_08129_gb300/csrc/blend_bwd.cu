// blend_bwd.cu -- the blend adjoint (instantiation unit): one persistent
// kernel per tile shape, core size at run time, per-pixel state in dynamic
// shared memory.
#include "blend_impl.cuh"

namespace htgs {

namespace {

template <int TW, int TH, bool NOTAIL, bool VIS>
bool run_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    const size_t smem = bwd_smem_bytes(TW * TH, a.prm.K);
    const void *fn = (const void *)blend_bwd_kernel<TW, TH, NOTAIL, VIS>;
    if (!allow_dynamic_smem(fn, bwd_smem_bytes(TW * TH, HTGS_MAX_K))) return false;
    const int grid = persistent_grid(fn, kBwdThreads, smem, a.max_items);
    blend_bwd_kernel<TW, TH, NOTAIL, VIS><<<grid, kBwdThreads, smem, s>>>(b, a);
    return true;
}

// The tail-less variant and the visibility statistic are compiled into
// separate instances so that the default adjoint keeps its code.
template <int TW, int TH>
bool run_bwd_mode(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    if (a.vis) return a.prm.no_tail ? run_bwd<TW, TH, true, true>(b, a, s) : run_bwd<TW, TH, false, true>(b, a, s);
    return a.prm.no_tail ? run_bwd<TW, TH, true, false>(b, a, s) : run_bwd<TW, TH, false, false>(b, a, s);
}

} // namespace

bool launch_blend_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    if (a.prm.K < 0 || a.prm.K > HTGS_MAX_K) return false;
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return run_bwd_mode<16, 16>(b, a, s);
    if (tw == 16 && th == 8) return run_bwd_mode<16, 8>(b, a, s);
    if (tw == 8 && th == 8) return run_bwd_mode<8, 8>(b, a, s);
    return false;
}

} // namespace htgs
