// FP32-pipe throughput probe. Not part of the rendering method: the blend
// kernels are bound by the FP32 pipe (plain FMA/ALU work, no tensor cores),
// so their roofline is the rate at which the device retires FP32 FMAs. This
// kernel measures it: every thread runs kChains independent chains
// x <- fma(x, a, b), enough chains per SM to hide the FMA latency, with a
// and b taken from the arguments so that nothing folds at compile time.
#include <cuda_runtime.h>

#include "htgs.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_chain_kernel(float *out, float a, float b, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * threadIdx.x + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" htgs_status htgs_fma_probe(int32_t blocks, int32_t iters, float *out, void *stream,
                                      int64_t *fma_per_launch) {
    if (blocks <= 0 || iters <= 0 || !out || !fma_per_launch) return HTGS_ERR_INVALID_ARG;
    *fma_per_launch = int64_t(blocks) * kThreads * iters * kUnroll * kChains;
    fma_chain_kernel<<<blocks, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(out, 0.99993f, 1e-4f, iters);
    return cudaGetLastError() == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}
