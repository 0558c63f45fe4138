// render_static.cu -- htgs_render_static: the forward render with all of its
// scratch memory in one fixed-size array that the library itself defines,
// for callers that cannot allocate device memory (the paper has no
// counterpart; see include/htgs.h).
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds HTGS_STATIC_SCRATCH_BYTES of it until the process exits. Host
// code cannot use the array's name as a device address: on the first call on
// a device (with that device current) its address is looked up with
// cudaGetSymbolAddress and cached; later calls reuse it.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticBytes = HTGS_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Device address of g_scratch on the current device, looked up once.
htgs_status scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HTGS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HTGS_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HTGS_OK;
}

} // namespace

extern "C" htgs_status htgs_render_static(const htgs_gaussians *gaussians, const htgs_camera *cam,
                                          const htgs_params *params, const htgs_launch *launch,
                                          float *image, void *stream) {
    if (!gaussians || !cam || !params || !image) return HTGS_ERR_INVALID_ARG;
    // Scratch needed without any tile instances; the rest holds instances.
    size_t base = 0;
    htgs_status st = htgs_workspace_size(gaussians->n, cam, params, launch, 0, &base, nullptr);
    if (st != HTGS_OK) return st;
    if (base > kStaticBytes) return HTGS_ERR_WORKSPACE;
    // Largest instance capacity whose workspace fits: the size grows
    // monotonically with the capacity, so bisect (host arithmetic only).
    int64_t lo = 0, hi = (int64_t)(kStaticBytes / 16) + 1;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        size_t need = 0;
        st = htgs_workspace_size(gaussians->n, cam, params, launch, mid, &need, nullptr);
        if (st != HTGS_OK) return st;
        if (need <= kStaticBytes) lo = mid; else hi = mid;
    }
    const int64_t cap = lo;
    void *ws = nullptr;
    st = scratch_address(&ws);
    if (st != HTGS_OK) return st;
    st = htgs_render(gaussians, cam, params, launch, ws, kStaticBytes, cap, nullptr, image, stream);
    if (st != HTGS_OK) return st;
    // Synchronise and report what the device found (an instance overflow
    // means the scene does not fit the static scratch).
    htgs_status device_status = HTGS_OK;
    st = htgs_get_error(ws, kStaticBytes, stream, &device_status, nullptr);
    if (st != HTGS_OK) return st;
    return device_status;
}
