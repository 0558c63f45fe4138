/*
 * htgs.h -- C ABI of the GB300 (sm_103a) renderer for perspective-correct 3D
 * Gaussian splatting with hybrid transparency (arXiv 2410.08129).
 *
 * Problem statement (Sec. 3.1-3.3): given Gaussians (mean, log-scales,
 * quaternion, opacity logit, SH colour), a pinhole camera and the core size
 * K, produce the image C of Eq. (15): each pixel blends the K nearest
 * fragments exactly in depth order and the remaining tail
 * order-independently behind them; render_backward returns dL/dparameters
 * for a given dL/dimage.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller, unless the
 *    entry point says otherwise. The library never allocates device memory
 *    on the render path and never synchronises the stream it is given.
 *  - Arrays are dense, row-major, float32, with the shapes stated below.
 *  - Scratch memory is a caller-allocated workspace whose size comes from
 *    htgs_workspace_size; the workspace must start on a 256-byte boundary.
 *  - Every call returns an htgs_status; nothing throws across the ABI.
 *    Errors found on the device (instance-capacity overflow, a bounded wait
 *    that gave up) are recorded in the workspace and read back with
 *    htgs_get_error after the stream has run.
 *  - Calls sharing one workspace must not overlap on the GPU.
 */
#ifndef HTGS_H
#define HTGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t htgs_status;
#define HTGS_OK 0
#define HTGS_ERR_INVALID_ARG 1   /* a pointer, size or parameter is out of range */
#define HTGS_ERR_WORKSPACE 2     /* the workspace or saved buffer is too small */
#define HTGS_ERR_OVERFLOW 3      /* more tile instances than instance_capacity; see htgs_get_error */
#define HTGS_ERR_CUDA 4          /* a CUDA launch or runtime call failed */
#define HTGS_ERR_TIMEOUT 5       /* a bounded device-side wait gave up */
#define HTGS_ERR_NOT_SUPPORTED 6 /* e.g. K above the largest compiled core size */
#define HTGS_ERR_INTERNAL 7      /* a device-side consistency check failed (the binning's tile
                                    spans disagreed with the instance counts); the blend is
                                    skipped */

/* Largest core size K compiled into the blend kernels. */
#define HTGS_MAX_K 32
/* Largest instance_capacity: instance indices are 32-bit. */
#define HTGS_MAX_CAPACITY 2147483647ll

/* Scene parameters (Sec. 3.1). N Gaussians; n_coeff = (sh_degree + 1)^2.
 *   means          N x 3        world-space mean mu
 *   log_scales     N x 3        log s_u, log s_v, log s_w
 *   quats          N x 4        (w, x, y, z), normalised inside the library
 *   opacity_logits N            o = sigmoid(logit)
 *   sh             N x n_coeff x 3, real SH in 3DGS order, degree <= 3
 * Device pointers; float32; 16-byte aligned base addresses. */
typedef struct {
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logits;
    const float *sh;
    int64_t n;
    int32_t sh_degree;
    /* NULL, or n floats: the variance v of the 3D smoothing filter applied to
     * each Gaussian before rendering (Sec. 4.2, the 3D filter of Yu et al.):
     * scales become sqrt(s^2 + v) and the opacity is scaled by
     * prod s / sqrt(s^2 + v); v is an input, no gradient flows to it. */
    const float *filter_var;
    /* NULL, or n records written by htgs_bake (HTGS_BAKED_FLOATS(sh_degree)
     * floats each, 16-byte aligned): the forward then reads these instead of
     * means .. sh and filter_var (which may be NULL). Forward only: the
     * backward needs the raw parameters and rejects a baked scene. */
    const float *baked;
} htgs_gaussians;

/* Floats per baked Gaussian (App. A "baking": activations folded into the
 * parameters, every coefficient of a Gaussian in one buffer): the unit
 * quaternion, the mean and 2 ln o, the scales (the 3D filter applied) and a
 * pad, then the 3 (deg + 1)^2 SH coefficients; rounded up to a multiple of 4
 * so that every record starts on a 16-byte boundary. 240 bytes at degree 3. */
#define HTGS_BAKED_FLOATS(deg) (4 * ((12 + 3 * ((deg) + 1) * ((deg) + 1) + 3) / 4))

/* Gradient outputs, same shapes as htgs_gaussians. Device pointers.
 * The last three are optional training statistics of the render (NULL to
 * skip; n floats each, caller-initialised, accumulated across calls):
 *   visibility     max(visibility, largest blending weight of the Gaussian in
 *                  any pixel): alpha_i T_i in the core, T_core (1 - T_tail)
 *                  alpha_j / A in the tail (the visibility score of Sec. 4.2,
 *                  after Niemeyer et al.); non-negative
 *   densify_grad   += |dL/dmean| times half the distance from the camera, per
 *                  view whose pixels the Gaussian covers (Sec. 4.2, after
 *                  Moenne-Loccoz et al.)
 *   densify_count  += 1 per such view */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
    float *visibility;
    float *densify_grad;
    float *densify_count;
} htgs_gaussians_grad;

/* Pinhole camera, OpenCV axes (+x right, +y down, +z forward); world_to_cam
 * is the row-major 4x4 model-view matrix M of Eq. (3) (last row 0 0 0 1).
 * Pixel (i, j) has its centre at (i + 0.5, j + 0.5). Host memory (by value). */
typedef struct {
    float world_to_cam[16];
    float fx, fy, cx, cy;
    float z_near; /* a Gaussian whose cutoff ellipsoid reaches z <= z_near is culled */
    int32_t width, height;
} htgs_camera;

/* Method parameters (Sec. 3.2 tau_alpha; Sec. 4.2 K and tau_K). */
typedef struct {
    int32_t K;        /* core size, 0 <= K <= HTGS_MAX_K (K = 0 is fully order-independent) */
    float tau_alpha;  /* minimum fragment alpha; rho_c = 2 ln(o / tau_alpha) */
    float tau_K;      /* minimum alpha for a fragment to enter the core */
    float alpha_max;  /* alpha = min(o e^{-rho^2/2}, alpha_max), alpha_max < 1 */
    float bg[3];      /* background colour c_bg */
    int32_t no_tail;  /* 0: hybrid transparency (Eq. (15)); 1: inference without the tail
                         (Sec. 4.4 ablation): C = sum_core alpha_i T_i c_i + T_{K+1} c_bg */
    int32_t sorted_blend; /* 1: the variant without per-pixel hybrid transparency (Tab. 3):
                         the perspective-correct fragments of a pixel blended front to back
                         (Eq. (2) plus background) in the order of their Gaussians' view-space
                         mean depth (then index), stopping before the fragment that would take
                         the transmittance below 1e-4; K, tau_K and no_tail are ignored */
} htgs_params;

/* Tuning knobs (none changes the result beyond float rounding order),
 * optional timing hooks and a test hook of the failure path. A NULL
 * htgs_launch* or a zero field selects the default.
 *   events  host array of 6 cudaEvent_t handles (created by the caller; any
 *           entry may be NULL). htgs_render records [0]/[1] around the
 *           preprocess, [2]/[3] around binning and sorting and [4]/[5]
 *           around the blend; htgs_render_backward records [0]/[1] around
 *           the blend adjoint and [2]/[3] around the preprocess adjoint.
 *           Without events a call launches each of its kernels as a
 *           programmatic dependent of the one before (its CTAs may be
 *           scheduled while the previous kernel finishes; it waits for that
 *           kernel's completion before touching memory); with any event set
 *           the kernels are launched plainly, so that the events mark the
 *           phase boundaries. The results are the same either way. */
typedef struct {
    int32_t tile_w, tile_h;   /* tile shape in pixels: 16x16 (default), 32x16, 16x8 or 8x8 */
    int32_t px_per_thread;    /* pixels per thread in the forward blend: 1 (default), 2 or 4, a
                                 request the kernels may narrow: 1 when params.no_tail is set or
                                 K > 16, at most 2 when K > 8; 4 needs 16x16 tiles (32x16 runs it
                                 as 2, 16x8 and 8x8 return HTGS_ERR_NOT_SUPPORTED) */
    int32_t depth_bits;       /* reserved; must be 0 (the sort key is the tile id alone) */
    int32_t smem_batch;       /* records the forward blend stages per shared-memory batch:
                                 32, 64, 128 (default, also for 0) or 192 (two staging
                                 buffers instead of three, in the same shared memory; the
                                 variant without per-pixel hybrid transparency takes 128) */
    void *events[6];
    int32_t test_lookback_stall; /* test of the failure path, 0 otherwise: in the tile sort's first
                                    digit pass the first block also waits for a look-back word that
                                    nothing writes; the bounded wait gives up, the sort completes
                                    correctly, the blend is skipped and htgs_get_error reports
                                    HTGS_ERR_TIMEOUT (forces the radix-sort binning) */
    int32_t binning;          /* how tile lists are built; both give the same lists (the records
                                 covering each tile in record order, or in mean-depth order for
                                 sorted blending): 0 (default) or 1 the stable LSD radix sort of
                                 tile keys; 2 a stable counting sort by tile computed from the
                                 records' tile covers, for a single view whose tile rows are
                                 at most 2048 tiles long (HTGS_ERR_NOT_SUPPORTED otherwise) */
    int32_t tile_cover;       /* which tiles a Gaussian is binned to (Sec. 4.3); both give the
                                 same image up to the summation order of split tiles: 0
                                 (default) per tile row of its bounding rectangle the span of
                                 tiles its cutoff ellipse reaches (the ellipse holds every pixel
                                 with rho^2 <= rho_c, so no tile with a fragment is dropped);
                                 1 every tile of the rectangle */
} htgs_launch;

/* Sizes of the caller-owned buffers for one camera.
 *   instance_capacity  maximum number of (Gaussian, tile) instances, 0 .. HTGS_MAX_CAPACITY
 *   fwd_bytes    [out] workspace bytes needed by htgs_render / htgs_render_backward
 *   saved_bytes  [out] per-pixel state htgs_render saves for the backward:
 *                (7 + K) * width * height * 4 bytes
 * Returns HTGS_ERR_INVALID_ARG for a bad size or parameter. */
htgs_status htgs_workspace_size(int64_t n_gaussians, const htgs_camera *cam,
                                const htgs_params *params, const htgs_launch *launch,
                                int64_t instance_capacity, size_t *fwd_bytes, size_t *saved_bytes);

/* Byte offsets of the internal buffers inside a workspace, for inspection by
 * tests and tools; their contents are valid after htgs_render has run.
 *   rec          n x 8 float4: per-Gaussian blend record (128 bytes)
 *   rect         n x uint2: bounding tile rectangle (tx0 | tx1 << 16, ty0 | ty1 << 16)
 *   count        n x uint32: tiles the Gaussian is binned to (htgs_launch.tile_cover)
 *   sorted_keys  capacity x uint32: tile keys after the radix sort
 *   sorted_vals  capacity x uint32: the matching Gaussian ids
 *   ranges       n_tiles x uint2: [start, end) of each tile in the sorted list
 *   acc          n x 16 float: gradient accumulators of the blend adjoint
 *   items        max_items x int4: blend work items (tile, chunk k, chunks m,
 *                first partial-state slot), longest chunks first
 *   n_items      1 x uint32: number of items of the last render
 *   partials     slots x (6 + 2K) x tile pixels float: partial states of split
 *                tiles (sum alpha, sum alpha rgb, prod (1 - alpha), count as
 *                int bits, then K (depth, gid bits) pairs), pixel-minor
 * A tile whose list is longer than max(1024, instances / 2048) is cut into
 * m > 1 chunks processed by different CTAs (at most slots chunks in all);
 * the forward merges their partial states, so the result does not depend
 * on the cut except for the order of floating-point sums.
 * Same argument rules as htgs_workspace_size; out is a host pointer. */
typedef struct {
    uint64_t rec, rect, count, sorted_keys, sorted_vals, ranges, acc;
    int32_t n_tiles, tiles_x, tiles_y, tile_bits;
    uint64_t items, n_items, partials;
    int32_t max_items, slots;
} htgs_layout;

htgs_status htgs_workspace_layout(int64_t n_gaussians, const htgs_camera *cam,
                                  const htgs_params *params, const htgs_launch *launch,
                                  int64_t instance_capacity, htgs_layout *out);

/* Forward render, Sec. 3.2-3.3 and Eq. (15): preprocess (activations,
 * T' = V P M T, tight bounding box, SH colour), tile binning and radix
 * sort by tile key, and the per-pixel blend with a K-core and an
 * order-independent tail.
 *   image   [out] height x width x 3 float32, device
 *   saved   [out] nullable; (7 + K) * width * height floats of per-pixel state
 *           for htgs_render_backward (see htgs_workspace_size)
 * The call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 * stream). If the instances exceed instance_capacity the blend is skipped
 * and htgs_get_error reports HTGS_ERR_OVERFLOW with the required capacity. */
htgs_status htgs_render(const htgs_gaussians *gaussians, const htgs_camera *cam,
                        const htgs_params *params, const htgs_launch *launch,
                        void *workspace, size_t workspace_bytes, int64_t instance_capacity,
                        float *saved, float *image, void *stream);

/* Backward of htgs_render, Sec. 3.3: re-traverses the tile lists of the
 * preceding htgs_render (same workspace, same inputs), using the saved
 * per-pixel core ids and tail accumulators; the tail's partial derivatives
 * are per-pixel constants. Writes dL/d(every parameter) into `grads`
 * (overwritten, not accumulated). dl_dimage: height x width x 3, device.
 * No gradient flows through depth order, tau_alpha, tau_K or the culls. */
htgs_status htgs_render_backward(const htgs_gaussians *gaussians, const htgs_camera *cam,
                                 const htgs_params *params, const htgs_launch *launch,
                                 void *workspace, size_t workspace_bytes, int64_t instance_capacity,
                                 const float *saved, const float *dl_dimage,
                                 const htgs_gaussians_grad *grads, void *stream);

/* ---------------------------------------------------------------------------
 * Batched form: many views (of uneven resolution, of one scene or of several
 * scenes of uneven size) rendered by one launch per phase. The blend is a
 * persistent kernel over a (view, tile) work queue; nothing synchronises
 * the stream, so a batch can be captured in a CUDA graph. Results are those
 * of rendering each view alone. The paper renders one view at a time (Sec.
 * 4); batching is this library's addition.
 * ------------------------------------------------------------------------- */
#define HTGS_MAX_VIEWS 64

/* One view of a batch. All pointers are device pointers except `gaussians`
 * and `grads`, which point to host structs holding device pointers.
 *   gaussians  the scene this view renders; several views may share one
 *   camera     the view's camera (its own resolution)
 *   image      [out] height x width x 3 (htgs_render_batch)
 *   saved      [out/in] (7 + K) * width * height floats; written by
 *              htgs_render_batch when non-NULL, read by the backward
 *   dl_dimage  height x width x 3 (htgs_render_batch_backward only)
 *   grads      [out] (backward only). Views that share a scene must pass
 *              the same grads; their gradients are summed (the buffers are
 *              zeroed by the call). A view with its own grads gets them
 *              overwritten. */
typedef struct {
    const htgs_gaussians *gaussians;
    htgs_camera camera;
    float *image;
    float *saved;
    const float *dl_dimage;
    const htgs_gaussians_grad *grads;
} htgs_view;

/* Workspace bytes for a batch of n_views (1..HTGS_MAX_VIEWS) views sharing
 * one instance_capacity (tile instances over all views). Host pointers. */
htgs_status htgs_batch_workspace_size(int32_t n_views, const htgs_view *views,
                                      const htgs_params *params, const htgs_launch *launch,
                                      int64_t instance_capacity, size_t *workspace_bytes);

/* Offsets of the internal buffers of a batch workspace (see htgs_layout):
 * records of view v start at record sum_{u < v} n_u, tiles of view v at
 * tile sum_{u < v} tiles_x(u) * tiles_y(u); tiles_x and tiles_y describe
 * view 0. Host pointers; nothing is read on the device. */
htgs_status htgs_batch_workspace_layout(int32_t n_views, const htgs_view *views,
                                        const htgs_params *params, const htgs_launch *launch,
                                        int64_t instance_capacity, htgs_layout *out);

/* Forward render of every view of a batch (Eq. (15) per pixel of each view).
 * Errors and overflow as for htgs_render (htgs_get_error on the workspace). */
htgs_status htgs_render_batch(int32_t n_views, const htgs_view *views, const htgs_params *params,
                              const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                              int64_t instance_capacity, void *stream);

/* Backward of htgs_render_batch (same views, workspace and inputs). */
htgs_status htgs_render_batch_backward(int32_t n_views, const htgs_view *views,
                                       const htgs_params *params, const htgs_launch *launch,
                                       void *workspace, size_t workspace_bytes,
                                       int64_t instance_capacity, void *stream);

/* Reads the device status word of a workspace after synchronising `stream`.
 *   status              [out] HTGS_OK, HTGS_ERR_OVERFLOW or HTGS_ERR_TIMEOUT
 *   instances           [out] nullable; tile instances of the last render
 * Host pointers. Clears nothing: the next htgs_render resets the word. */
htgs_status htgs_get_error(void *workspace, size_t workspace_bytes, void *stream,
                           htgs_status *status, int64_t *instances);

/* Work counters of the last htgs_render on a workspace, after synchronising
 * `stream`. counters (host, 4 x uint64):
 *   [0] pixels inside the Gaussians' tight bounding boxes (sum over Gaussians)
 *   [1] kept fragments, rho^2 <= rho_c, over all pixels
 *   [2] kept fragments with alpha >= tau_K (core candidates)
 *   [3] core insertions */
htgs_status htgs_get_counters(void *workspace, size_t workspace_bytes, void *stream,
                              uint64_t *counters);

/* L1 photometric loss of a rendered image against a target (the training
 * step's loss): loss = mean |image - target| over n = H*W*3 values and
 * dl_dimage = sign(image - target) / n with sign(0) = 0.
 *   image, target  n floats, device
 *   dl_dimage      [out] n floats, device
 *   loss           [out] 1 float, device (overwritten)
 * Asynchronous on `stream`. */
htgs_status htgs_l1_loss_grad(const float *image, const float *target, int64_t n, float *dl_dimage,
                              float *loss, void *stream);

/* Size of the scratch array that htgs_render_static keeps on every device. */
#define HTGS_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* Forward render that allocates nothing: the same result as htgs_render
 * (no saved state), with all scratch memory in a fixed 32 MiB array that the
 * library defines on every device that loads it. For callers that must not
 * allocate device memory themselves, e.g. a plugin inside a host
 * application that owns the device heap, or a real-time loop where an
 * allocation (which may synchronise the device) is not allowed. The paper
 * has no counterpart of this entry point.
 *   image   [out] height x width x 3 float32, device (caller-owned)
 * Size limit: the workspace of htgs_workspace_size must fit the array. That
 * is about 240 bytes per Gaussian (the blend record, tile rectangle, tile
 * cover and count, and the per-Gaussian accumulators the layout keeps) plus
 * a small per-tile part, so at most about 139,000 Gaussians even with no tile
 * instances; the rest of the array holds the instances, at about
 * 18 + (6 + 2K) * tile_pixels / 128 bytes each (44 at K = 4 with 16x16
 * tiles). Beyond the first limit the call returns HTGS_ERR_WORKSPACE, beyond
 * the second HTGS_ERR_OVERFLOW.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture. A device reset (cudaDeviceReset) reloads the library's device
 * code, so the cached address must not be used after one: call this entry
 * point only in processes that do not reset the device. The call
 * synchronises `stream` before returning. Every call shares the one array
 * and the render clears what must start at zero; calls that overlap on the
 * GPU (two streams, or two host threads on one device) race on it. */
htgs_status htgs_render_static(const htgs_gaussians *gaussians, const htgs_camera *cam,
                               const htgs_params *params, const htgs_launch *launch, float *image,
                               void *stream);

/* Baking (App. A): writes, for every Gaussian of `gaussians` (raw parameters,
 * and filter_var if set), the record the forward reads when
 * htgs_gaussians.baked points to it: q / |q|, the mean, 2 ln o and the scales
 * after the 3D filter, and the SH coefficients, computed with the same
 * operations as the forward's own activations, so a render of the baked scene
 * equals a render of the raw one bit for bit.
 *   gaussians  raw parameters (gaussians->baked must be NULL)
 *   baked      [out] n x HTGS_BAKED_FLOATS(sh_degree) floats, device,
 *              16-byte aligned (caller-owned)
 * Asynchronous on `stream`. HTGS_ERR_INVALID_ARG for a NULL or misaligned
 * buffer or invalid parameters. */
htgs_status htgs_bake(const htgs_gaussians *gaussians, float *baked, void *stream);

/* FP32-pipe throughput probe (a measurement aid; the paper has no
 * counterpart). Launches `blocks` CTAs of 256 threads; each thread runs 8
 * independent chains of 16 * iters fused multiply-adds, then writes one
 * float to out (blocks * 256 floats, device, caller-owned). Timing the launch
 * with events on `stream` gives the device's FP32 FMA rate, the roofline of
 * the blend kernels (which use no tensor cores).
 *   fma_per_launch  [out] host: FMA instructions per thread-lane summed
 *                   over the launch, blocks * 256 * iters * 128
 * Asynchronous on `stream`. HTGS_ERR_INVALID_ARG for a non-positive size or
 * a NULL pointer; HTGS_ERR_CUDA when the launch fails. */
htgs_status htgs_fma_probe(int32_t blocks, int32_t iters, float *out, void *stream, int64_t *fma_per_launch);

/* Static string for a status code. */
const char *htgs_status_string(htgs_status status);

#ifdef __cplusplus
}
#endif
#endif /* HTGS_H */
