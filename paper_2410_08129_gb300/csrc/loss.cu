// loss.cu -- L1 photometric loss and its gradient for the training step
// (the paper trains with the 3DGS photometric loss, Sec. 4.2; the step here
// uses its L1 term: loss = mean |C - C*|, dL/dC = sign(C - C*) / n).
#include "common.cuh"

namespace htgs {
namespace {

constexpr int kLossThreads = 256;

__global__ void __launch_bounds__(kLossThreads)
l1_kernel(const float4 *__restrict__ img, const float4 *__restrict__ tgt, int64_t n4,
          const float *__restrict__ img_s, const float *__restrict__ tgt_s, int64_t n, float inv_n,
          float4 *__restrict__ dl, float *__restrict__ dl_s, float *loss) {
    dependent_entry();
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * kLossThreads + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * kLossThreads) {
        const float4 a = img[i], b = tgt[i];
        const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
        acc += fabsf(dx) + fabsf(dy) + fabsf(dz) + fabsf(dw);
        auto sg = [](float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); };
        dl[i] = make_float4(sg(dx) * inv_n, sg(dy) * inv_n, sg(dz) * inv_n, sg(dw) * inv_n);
    }
    // Scalar tail (n not a multiple of 4), handled by block 0.
    if (blockIdx.x == 0)
        for (int64_t i = n4 * 4 + threadIdx.x; i < n; i += kLossThreads) {
            const float d = img_s[i] - tgt_s[i];
            acc += fabsf(d);
            dl_s[i] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv_n;
        }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float ws[kLossThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kLossThreads / 32; ++w) s += ws[w];
        atomicAdd(loss, s * inv_n);
    }
}

} // namespace
} // namespace htgs

extern "C" htgs_status htgs_l1_loss_grad(const float *image, const float *target, int64_t n,
                                         float *dl_dimage, float *loss, void *stream) {
    using namespace htgs;
    if (n < 0 || !loss || (n > 0 && (!image || !target || !dl_dimage))) return HTGS_ERR_INVALID_ARG;
    const bool vec_ok = (((uintptr_t)image | (uintptr_t)target | (uintptr_t)dl_dimage) & 15u) == 0;
    if (!vec_ok) return HTGS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return HTGS_ERR_CUDA;
    if (n == 0) return HTGS_OK;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n4 = n / 4;
    int64_t blocks = (n4 + kLossThreads - 1) / kLossThreads;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    l1_kernel<<<(int)blocks, kLossThreads, 0, s>>>(
        reinterpret_cast<const float4 *>(image), reinterpret_cast<const float4 *>(target), n4, image,
        target, n, 1.f / (float)n, reinterpret_cast<float4 *>(dl_dimage), dl_dimage, loss);
    return cudaGetLastError() == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}
