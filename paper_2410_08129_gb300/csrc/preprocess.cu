// preprocess.cu -- per-Gaussian setup and its adjoint (arXiv 2410.08129,
// Sec. 3.1 scene representation, Sec. 3.2 Eq. (3) T' = V P M T, the tight
// screen bounding box and the opacity-aware cutoff).
//
// One thread per Gaussian. The forward writes the 128-byte blend record (see
// common.cuh), the bounding tile rectangle and the instance count (the
// tiles of the rectangle the cutoff ellipse reaches, row by row); the backward
// turns the per-Gaussian gradient accumulators of the blend adjoint into
// gradients of the means, log-scales, quaternions, opacity logits and SH.
#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

namespace {

// Real spherical harmonics up to degree 3 in 3DGS order (m = -l..l), as
// polynomials of the unit direction. Constants are the closed forms
// Y00 = 1/(2 sqrt(pi)), Y1 = sqrt(3/(4 pi)), Y2 = sqrt(15/(4 pi)),
// sqrt(5/(16 pi)), sqrt(15/(16 pi)), Y3 = sqrt(35/(32 pi)), sqrt(105/(4 pi)),
// sqrt(21/(32 pi)), sqrt(7/(16 pi)), sqrt(105/(16 pi)).
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.48860251190291992f;
constexpr float kSH2a = 1.0925484305920792f;
constexpr float kSH2b = 0.31539156525252005f;
constexpr float kSH2c = 0.54627421529603959f;
constexpr float kSH3a = 0.59004358992664352f;
constexpr float kSH3b = 2.8906114426405538f;
constexpr float kSH3c = 0.45704579946446572f;
constexpr float kSH3d = 0.37317633259011546f;
constexpr float kSH3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_eval(float x, float y, float z, int deg, float Y[16]) {
    Y[0] = kSH0;
    if (deg < 1) return;
    Y[1] = -kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = -kSH1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kSH2a * x * y;
    Y[5] = -kSH2a * y * z;
    Y[6] = kSH2b * (2.f * zz - xx - yy);
    Y[7] = -kSH2a * x * z;
    Y[8] = kSH2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kSH3a * y * (3.f * xx - yy);
    Y[10] = kSH3b * x * y * z;
    Y[11] = -kSH3c * y * (4.f * zz - xx - yy);
    Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kSH3c * x * (4.f * zz - xx - yy);
    Y[14] = kSH3e * z * (xx - yy);
    Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Colour of one Gaussian before the clamp: 0.5 + sum_k Y_k(dir) sh_k for
// degree DEG (compile time, so Y stays in registers). Rows whose length
// (3 (DEG+1)^2 floats) is a multiple of 4 are read as float4.
template <int DEG>
__device__ __forceinline__ void sh_colour(const float *__restrict__ sh, float x, float y, float z,
                                          float rgb[3]) {
    constexpr int NC = (DEG + 1) * (DEG + 1);
    float Y[16];
    sh_eval(x, y, z, DEG, Y);
    float c[3 * NC];
    if constexpr ((3 * NC) % 4 == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(sh);
#pragma unroll
        for (int j = 0; j < 3 * NC / 4; ++j) {
            const float4 v = __ldg(s4 + j);
            c[4 * j] = v.x; c[4 * j + 1] = v.y; c[4 * j + 2] = v.z; c[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 3 * NC; ++j) c[j] = __ldg(sh + j);
    }
    rgb[0] = rgb[1] = rgb[2] = 0.5f;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        rgb[0] += Y[k] * c[3 * k + 0];
        rgb[1] += Y[k] * c[3 * k + 1];
        rgb[2] += Y[k] * c[3 * k + 2];
    }
}

// d(sum_k w_k Y_k)/d(x, y, z) for a weight vector w.
__device__ __forceinline__ void sh_grad(float x, float y, float z, int deg, const float w[16],
                                        float g[3]) {
    g[0] = g[1] = g[2] = 0.f;
    if (deg < 1) return;
    g[1] += -kSH1 * w[1];
    g[2] += kSH1 * w[2];
    g[0] += -kSH1 * w[3];
    if (deg < 2) return;
    g[0] += kSH2a * y * w[4];
    g[1] += kSH2a * x * w[4];
    g[1] += -kSH2a * z * w[5];
    g[2] += -kSH2a * y * w[5];
    g[0] += -2.f * kSH2b * x * w[6];
    g[1] += -2.f * kSH2b * y * w[6];
    g[2] += 4.f * kSH2b * z * w[6];
    g[0] += -kSH2a * z * w[7];
    g[2] += -kSH2a * x * w[7];
    g[0] += 2.f * kSH2c * x * w[8];
    g[1] += -2.f * kSH2c * y * w[8];
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += -kSH3a * 6.f * x * y * w[9];
    g[1] += -kSH3a * 3.f * (xx - yy) * w[9];
    g[0] += kSH3b * y * z * w[10];
    g[1] += kSH3b * x * z * w[10];
    g[2] += kSH3b * x * y * w[10];
    g[0] += kSH3c * 2.f * x * y * w[11];
    g[1] += -kSH3c * (4.f * zz - xx - 3.f * yy) * w[11];
    g[2] += -kSH3c * 8.f * y * z * w[11];
    g[0] += -kSH3d * 6.f * x * z * w[12];
    g[1] += -kSH3d * 6.f * y * z * w[12];
    g[2] += kSH3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    g[0] += -kSH3c * (4.f * zz - 3.f * xx - yy) * w[13];
    g[1] += kSH3c * 2.f * x * y * w[13];
    g[2] += -kSH3c * 8.f * x * z * w[13];
    g[0] += kSH3e * 2.f * x * z * w[14];
    g[1] += -kSH3e * 2.f * y * z * w[14];
    g[2] += kSH3e * (xx - yy) * w[14];
    g[0] += -kSH3a * 3.f * (xx - yy) * w[15];
    g[1] += kSH3a * 6.f * x * y * w[15];
}

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Geometry shared by the forward and the backward setup.
struct Setup {
    bool valid;
    float o, rho_c;    // opacity and cutoff of the rendered (filtered) Gaussian
    float two_ln_o;    // 2 ln o of the rendered Gaussian (rho_c + 2 ln tau_alpha)
    float o_raw;       // sigmoid(logit)
    float s[3];        // scales of the rendered Gaussian
    float s_raw[3];    // exp(log-scales)
    float fvar;        // 3D filter variance (0 without a filter)
    float q[4];        // normalised (w, x, y, z)
    float qnorm;
    float R[3][3];
    V3 A[3];           // rows of M_rot R diag(s): the xyz part of (M T) rows 1..3
    float mu[3];       // view-space mean (the w column of M T)
    float dir[3];
    float dist;
};

// Rotation, view transform, cull and view direction from the activated
// parameters in S (q, s, rho_c) and the mean.
__device__ __forceinline__ void setup_view(float mx, float my, float mz, const CamArgs &cam, Setup &S) {
    const float w = S.q[0], x = S.q[1], y = S.q[2], z = S.q[3];
    S.R[0][0] = 1.f - 2.f * (y * y + z * z); S.R[0][1] = 2.f * (x * y - w * z); S.R[0][2] = 2.f * (x * z + w * y);
    S.R[1][0] = 2.f * (x * y + w * z); S.R[1][1] = 1.f - 2.f * (x * x + z * z); S.R[1][2] = 2.f * (y * z - w * x);
    S.R[2][0] = 2.f * (x * z - w * y); S.R[2][1] = 2.f * (y * z + w * x); S.R[2][2] = 1.f - 2.f * (x * x + y * y);
    // A = M_rot R diag(s); mu_view = M_rot mu + t.
    for (int r = 0; r < 3; ++r) {
        float a[3];
        for (int c = 0; c < 3; ++c)
            a[c] = (cam.M[4 * r + 0] * S.R[0][c] + cam.M[4 * r + 1] * S.R[1][c] + cam.M[4 * r + 2] * S.R[2][c]) * S.s[c];
        S.A[r] = v3(a[0], a[1], a[2]);
        S.mu[r] = cam.M[4 * r + 0] * mx + cam.M[4 * r + 1] * my + cam.M[4 * r + 2] * mz + cam.M[4 * r + 3];
    }
    // Cull: rho_c <= 0, or the cutoff ellipsoid reaches z <= z_near.
    const float e2 = dot(S.A[2], S.A[2]);
    S.valid = (S.rho_c > 0.f) && (S.mu[2] - sqrtf(S.rho_c * e2) > cam.z_near);
    const float vx = mx - cam.centre[0], vy = my - cam.centre[1], vz = mz - cam.centre[2];
    S.dist = sqrtf(vx * vx + vy * vy + vz * vz);
    const float id = S.dist > 0.f ? 1.f / S.dist : 0.f;
    S.dir[0] = vx * id; S.dir[1] = vy * id; S.dir[2] = vz * id;
}

// The activations of Gaussian i (Sec. 3.1): unit quaternion, scales and
// 2 ln o, with the 3D smoothing filter applied when it is given. Shared by the
// forward setup and by baking, so both produce the same bits.
__device__ __forceinline__ void activate(const float *__restrict__ log_scales, const float *__restrict__ quats,
                                         const float *__restrict__ logits, const float *__restrict__ filter_var,
                                         int64_t i, Setup &S) {
    const float l = logits[i];
    // o = sigmoid(logit); 2 ln o = -2 ln(1 + e^{-l}), and rho_c = 2 ln o - 2 ln tau_alpha.
    S.o = 1.f / (1.f + __expf(-l));
    S.o_raw = S.o;
    float two_ln_o = -2.f * log1pf(__expf(-l));
    for (int k = 0; k < 3; ++k) S.s[k] = S.s_raw[k] = __expf(log_scales[3 * i + k]);
    // 3D smoothing filter (Sec. 4.2): convolution with an isotropic Gaussian
    // of variance v. Scales become sqrt(s^2 + v) and the opacity is scaled by
    // prod s / sqrt(s^2 + v), so 2 ln o drops by sum ln(1 + v / s^2).
    S.fvar = filter_var ? filter_var[i] : 0.f;
    if (filter_var) {
        for (int k = 0; k < 3; ++k) {
            const float r = S.fvar / (S.s_raw[k] * S.s_raw[k]);
            S.s[k] = S.s_raw[k] * sqrtf(1.f + r);
            S.o *= rsqrtf(1.f + r);
            two_ln_o -= log1pf(r);
        }
    }
    S.two_ln_o = two_ln_o;
    const float4 qr = reinterpret_cast<const float4 *>(quats)[i];
    S.qnorm = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float inv = 1.f / S.qnorm;
    S.q[0] = qr.x * inv; S.q[1] = qr.y * inv; S.q[2] = qr.z * inv; S.q[3] = qr.w * inv;
}

__device__ __forceinline__ void setup_geometry(const float *__restrict__ means,
                                               const float *__restrict__ log_scales,
                                               const float *__restrict__ quats,
                                               const float *__restrict__ logits,
                                               const float *__restrict__ filter_var, int64_t i,
                                               const CamArgs &cam, const ParamArgs &prm,
                                               Setup &S) {
    // (the mean is loaded first, so that all of the Gaussian's loads are in flight together)
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    activate(log_scales, quats, logits, filter_var, i, S);
    S.rho_c = S.two_ln_o - 2.f * __logf(prm.tau_alpha);
    setup_view(mx, my, mz, cam, S);
}

// The same setup from a baked record (App. A): bake_kernel applied activate(),
// so every field the forward uses is identical bit for bit. (The fields only
// the backward uses are not available: a baked scene renders forward only.)
__device__ __forceinline__ void setup_geometry_baked(const float *__restrict__ baked, int stride, int64_t i,
                                                     const CamArgs &cam, const ParamArgs &prm, Setup &S) {
    const float4 *r = reinterpret_cast<const float4 *>(baked + (size_t)i * stride);
    const float4 q = r[0], mo = r[1], sc = r[2];
    S.q[0] = q.x; S.q[1] = q.y; S.q[2] = q.z; S.q[3] = q.w;
    S.two_ln_o = mo.w;
    S.rho_c = mo.w - 2.f * __logf(prm.tau_alpha);
    S.s[0] = sc.x; S.s[1] = sc.y; S.s[2] = sc.z;
    S.o = S.o_raw = 0.f;
    S.s_raw[0] = S.s_raw[1] = S.s_raw[2] = 0.f;
    S.fvar = 0.f;
    S.qnorm = 1.f;
    setup_view(mo.x, mo.y, mo.z, cam, S);
}

// The expansion vectors of the Pluecker moment m and direction d about the
// record centre (xc, yc): m = M0 + x' Mx + y' My, d = D0 + x' Dx + y' Dy.
// a and b are the splat-space planes of the centre pixel's ray,
// a = T'_1 - xc T'_4, b = T'_2 - yc T'_4 (Sec. 3.2, Eq. (9)), written as
// fx (MT)_1 + (cx - xc)(MT)_3 to avoid cancelling large terms.
struct Expansion {
    V3 a, b, r;          // xyz parts of a, b and T'_4
    float aw, bw, rw;    // homogeneous parts
    V3 M0, Mx, My, D0, Dx, Dy;
};

__device__ __forceinline__ void make_expansion(const Setup &S, const CamArgs &cam, float xc,
                                               float yc, Expansion &E) {
    const float ox = cam.cx - xc, oy = cam.cy - yc;
    E.a = cam.fx * S.A[0] + ox * S.A[2];
    E.aw = cam.fx * S.mu[0] + ox * S.mu[2];
    E.b = cam.fy * S.A[1] + oy * S.A[2];
    E.bw = cam.fy * S.mu[1] + oy * S.mu[2];
    E.r = S.A[2];
    E.rw = S.mu[2];
    // m = a^0 b - b^0 a (the moment, (p^{01}, p^{02}, p^{03})), d = a x b.
    E.M0 = E.aw * E.b - E.bw * E.a;
    E.Mx = E.bw * E.r - E.rw * E.b;
    E.My = E.rw * E.a - E.aw * E.r;
    E.D0 = cross(E.a, E.b);
    E.Dx = cross(E.b, E.r);
    E.Dy = cross(E.r, E.a);
}

} // namespace

// The cutoff region Q >= 0 of a record, Q = q0 + x (q1 + q3 x + q4 y) +
// y (q2 + q5 y) about the box centre, as a matrix A = (a, b; b, c) with the
// region inside {p : p^T A p <= 1} (p measured from the box centre): the
// forward blend skips a warp's pixel block when an axis separates the two.
// The ellipse is grown about its own centre to cover the offset between that
// centre and the box centre, the rounding of the box centre (0.02 px), a
// relative 1e-3, and the rounding of A and of the per-pixel FP32 evaluation
// of Q, both of which scale with the condition number kappa of the quadratic
// part (a growth of 4e-6 kappa, far above the ~4e-7 kappa they need). A region
// that is not a bounded, well-conditioned ellipse (kappa > 1e5) gets A = 0,
// which never separates.
__device__ void cutoff_ellipse(const float (&q)[6], float (&A)[3]) {
    A[0] = A[1] = A[2] = 0.f;
    // -H = (m11, m12; m12, m22), positive definite for an ellipse.
    const float m11 = -q[3], m12 = -0.5f * q[4], m22 = -q[5];
    // det(-H) with the rounding of m12^2 compensated (Kahan's 2x2 determinant).
    const float w = m12 * m12;
    const float det = __fmaf_rn(m11, m22, -w) + __fmaf_rn(-m12, m12, w);
    if (!(m11 > 0.f) || !(det > 0.f)) return;
    const float half_tr = 0.5f * (m11 + m22);
    const float disc = sqrtf(0.25f * (m11 - m22) * (m11 - m22) + m12 * m12);
    const float mu_max = half_tr + disc, mu_min = det / mu_max;
    const float kappa = mu_max / mu_min;
    if (!(kappa <= 1e5f)) return;
    // Stationary point of Q (the ellipse centre) and the maximum of Q there:
    // -H c = -(q1, q2) / 2.
    const float cx = 0.5f * (m22 * q[1] - m12 * q[2]) / det;
    const float cy = 0.5f * (m11 * q[2] - m12 * q[1]) / det;
    const float qmax = q[0] + 0.5f * (q[1] * cx + q[2] * cy);
    if (!(qmax > 0.f)) return;
    // Semi-axes of {p : p^T (-H / qmax) p <= 1}: sqrt(qmax / mu).
    const float rmin = sqrtf(qmax / mu_max);
    const float grow = 1.f + 1e-3f + 4e-6f * kappa + (sqrtf(cx * cx + cy * cy) + 0.02f) / rmin;
    const float s = 1.f / (qmax * grow * grow);
    if (!isfinite(s)) return;
    A[0] = m11 * s;
    A[1] = m12 * s;
    A[2] = m22 * s;
}

// ---------------------------------------------------------------------------
// Baking (App. A): one record per Gaussian with the activations applied, in
// the layout setup_geometry_baked reads: [q / |q|][mean, 2 ln o][s, 0][SH..].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPreThreads) bake_kernel(BakeArgs a) {
    dependent_entry();
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    if (i >= a.n) return;
    Setup S;
    activate(a.log_scales, a.quats, a.logits, a.filter_var, i, S);
    const int stride = HTGS_BAKED_FLOATS(a.sh_degree);
    float4 *r = reinterpret_cast<float4 *>(a.baked + (size_t)i * stride);
    r[0] = make_float4(S.q[0], S.q[1], S.q[2], S.q[3]);
    r[1] = make_float4(a.means[3 * i], a.means[3 * i + 1], a.means[3 * i + 2], S.two_ln_o);
    r[2] = make_float4(S.s[0], S.s[1], S.s[2], 0.f);
    const int ncf = 3 * (a.sh_degree + 1) * (a.sh_degree + 1);
    const float *sh = a.sh + (size_t)i * ncf;
    float *dst = a.baked + (size_t)i * stride + 12;
    for (int k = 0; k < ncf; ++k) dst[k] = sh[k];
    for (int k = ncf; k < stride - 12; ++k) dst[k] = 0.f;
}

// ---------------------------------------------------------------------------
// K1: forward setup.
// ---------------------------------------------------------------------------
// BAKED: some view of the batch renders baked records (each view is checked);
// without it the kernel never looks for them.
template <bool BAKED>
__global__ void __launch_bounds__(kPreThreads)
preprocess_kernel(const __grid_constant__ Batch b, PreArgs a) {
    dependent_entry();
    __shared__ float4 s_recs[kPreThreads / 32][32 * kRecF4];
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    uint32_t count = 0;
    unsigned long long box_pixels = 0;
    // The record's cover and its tile rows (none unless it covers a tile).
    RowCover rcov = row_cover(make_uint2(1u, 0u), 0.f, 0.f, 0.f, 0.f, 0.f, false);
    uint32_t row_lo = 1u, row_hi = 0u;
    float mu_z = 0.f;
    if (i < b.n_rec) {
        // Record i is Gaussian g of the scene that view v renders.
        const ViewDesc &V = b.v[view_of_record(b, i)];
        const int64_t g = i - V.rec_off;
        const CamArgs &cam = V.cam;
        // The SH coefficients (most of the bytes read) are used only after the
        // geometry's chain of dependent steps: ask for them now.
        if (BAKED && V.baked)
            prefetch_l2(V.baked + (size_t)g * HTGS_BAKED_FLOATS(V.sh_degree), HTGS_BAKED_FLOATS(V.sh_degree) * 4);
        else
            prefetch_l2(V.sh + (size_t)g * 3 * (V.sh_degree + 1) * (V.sh_degree + 1),
                        12 * (V.sh_degree + 1) * (V.sh_degree + 1));
        Setup S;
        if (BAKED && V.baked)
            setup_geometry_baked(V.baked, HTGS_BAKED_FLOATS(V.sh_degree), g, cam, a.prm, S);
        else
            setup_geometry(V.means, V.log_scales, V.quats, V.logits, V.filter_var, g, cam, a.prm, S);
        uint2 rect = make_uint2(1u, 0u);
        float4 rec[kRecF4];
        for (int k = 0; k < kRecF4; ++k) rec[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (S.valid) {
            // Tight bounding box (Sec. 3.2). With u = fx (MT)_1, w = (MT)_3 and the
            // form B(x, y) = rho_c x_xyz . y_xyz - x_w y_w (the dual quadric
            // diag(rho_c, rho_c, rho_c, -1) mapped by T'), p = B(u, w)/B(w, w) + cx
            // and h^2 = (B(u, w)^2 - B(u, u) B(w, w)) / B(w, w)^2, whose numerator
            // expands to rho_c (|w_w U - u_w W|^2 - rho_c |U x W|^2); this avoids
            // the cancellation of p^2 - <f, T'_i . T'_i> in single precision.
            const float rc = S.rho_c;
            const float sden = rc * dot(S.A[2], S.A[2]) - S.mu[2] * S.mu[2]; // < 0
            float pc[2], hc[2];
            for (int ax = 0; ax < 2; ++ax) {
                const float f = ax == 0 ? cam.fx : cam.fy;
                const float c = ax == 0 ? cam.cx : cam.cy;
                const V3 U = S.A[ax];
                const float uw = S.mu[ax];
                pc[ax] = f * (rc * dot(U, S.A[2]) - uw * S.mu[2]) / sden + c;
                const V3 t = S.mu[2] * U - uw * S.A[2];
                const V3 cr = cross(U, S.A[2]);
                const float num = rc * (dot(t, t) - rc * dot(cr, cr));
                hc[ax] = fabsf(f) * sqrtf(fmaxf(num, 0.f)) / fabsf(sden);
            }
            // Covered pixel rectangle, widened by a small margin against rounding
            // (a wider box only adds work; the per-pixel test decides).
            const float lim[2] = {(float)(cam.width - 1), (float)(cam.height - 1)};
            float lo[2], hi[2], box[4];
            bool ok = true;
            for (int ax = 0; ax < 2; ++ax) {
                const float m = 1e-3f * hc[ax] + 1e-2f;
                box[2 * ax] = pc[ax] - hc[ax] - m;
                box[2 * ax + 1] = pc[ax] + hc[ax] + m;
                lo[ax] = fmaxf(ceilf(pc[ax] - hc[ax] - 0.5f - m), 0.f);
                hi[ax] = fminf(floorf(pc[ax] + hc[ax] - 0.5f + m), lim[ax]);
                ok = ok && (lo[ax] <= hi[ax]);
            }
            if (ok) {
                box_pixels = (unsigned long long)(hi[0] - lo[0] + 1.f) * (unsigned long long)(hi[1] - lo[1] + 1.f);
                const uint32_t tx0 = (uint32_t)lo[0] / a.tiles.tile_w, tx1 = (uint32_t)hi[0] / a.tiles.tile_w;
                const uint32_t ty0 = (uint32_t)lo[1] / a.tiles.tile_h, ty1 = (uint32_t)hi[1] / a.tiles.tile_h;
                rect = make_uint2(tx0 | (tx1 << 16), ty0 | (ty1 << 16));
                // Record: quadratic coefficients about the box centre.
                const float xc = pc[0], yc = pc[1];
                Expansion E;
                make_expansion(S, cam, xc, yc, E);
                float n[6], d[6], zq[6];
                n[0] = dot(E.M0, E.M0); n[1] = 2.f * dot(E.M0, E.Mx); n[2] = 2.f * dot(E.M0, E.My);
                n[3] = dot(E.Mx, E.Mx); n[4] = 2.f * dot(E.Mx, E.My); n[5] = dot(E.My, E.My);
                d[0] = dot(E.D0, E.D0); d[1] = 2.f * dot(E.D0, E.Dx); d[2] = 2.f * dot(E.D0, E.Dy);
                d[3] = dot(E.Dx, E.Dx); d[4] = 2.f * dot(E.Dx, E.Dy); d[5] = dot(E.Dy, E.Dy);
                // z D = T'_4,xyz . (d x m) + T'_4,w D, expanded in (x', y').
                const V3 C0 = cross(E.D0, E.M0);
                const V3 C1 = cross(E.D0, E.Mx) + cross(E.Dx, E.M0);
                const V3 C2 = cross(E.D0, E.My) + cross(E.Dy, E.M0);
                const V3 C3 = cross(E.Dx, E.Mx);
                const V3 C4 = cross(E.Dx, E.My) + cross(E.Dy, E.Mx);
                const V3 C5 = cross(E.Dy, E.My);
                zq[0] = dot(E.r, C0) + E.rw * d[0];
                zq[1] = dot(E.r, C1) + E.rw * d[1];
                zq[2] = dot(E.r, C2) + E.rw * d[2];
                zq[3] = dot(E.r, C3) + E.rw * d[3];
                zq[4] = dot(E.r, C4) + E.rw * d[4];
                zq[5] = dot(E.r, C5) + E.rw * d[5];
                const float hl = 0.72134752044448170f; // log2(e) / 2
                float q[6];
                for (int k = 0; k < 6; ++k) q[k] = hl * (rc * d[k] - n[k]);
                // Colour (Sec. 3.1, identical to 3DGS): max(0, 0.5 + sum Y_k sh_k).
                const int nc = (V.sh_degree + 1) * (V.sh_degree + 1);
                const float *sh = (BAKED && V.baked) ? V.baked + (size_t)g * HTGS_BAKED_FLOATS(V.sh_degree) + 12
                                                     : V.sh + g * nc * 3;
                float rgb[3];
                switch (V.sh_degree) {
                case 0: sh_colour<0>(sh, S.dir[0], S.dir[1], S.dir[2], rgb); break;
                case 1: sh_colour<1>(sh, S.dir[0], S.dir[1], S.dir[2], rgb); break;
                case 2: sh_colour<2>(sh, S.dir[0], S.dir[1], S.dir[2], rgb); break;
                default: sh_colour<3>(sh, S.dir[0], S.dir[1], S.dir[2], rgb); break;
                }
                rec[0] = make_float4(q[0], d[0], q[1], d[1]);
                rec[1] = make_float4(q[2], d[2], q[3], d[3]);
                rec[2] = make_float4(q[4], d[4], q[5], d[5]);
                rec[3] = make_float4(zq[0], zq[1], zq[2], zq[3]);
                rec[4] = make_float4(zq[4], zq[5], xc, yc);
                rec[5] = make_float4(fmaxf(rgb[0], 0.f), fmaxf(rgb[1], 0.f), fmaxf(rgb[2], 0.f), rc);
                rec[6] = make_float4(box[0], box[1], box[2], box[3]);
                // The point of maximum contribution lies inside the cutoff
                // ellipsoid, whose view depth spans mu_z -+ sqrt(rho_c |A_3|^2).
                const float zext = sqrtf(rc * dot(S.A[2], S.A[2]));
                const float zlo = (S.mu[2] - zext) - 1e-3f * zext - 1e-4f * fabsf(S.mu[2]);
                float cull[3];
                cutoff_ellipse(q, cull);
                rec[7] = make_float4(zlo, cull[0], cull[1], cull[2]);
            }
        }
        // Stage the record in the warp's shared-memory slab (float4 slots
        // XOR-swizzled by the lane so that neither side has bank conflicts).
        const int lane = threadIdx.x & 31;
        float4 *slab = s_recs[threadIdx.x >> 5];
#pragma unroll
        for (int k = 0; k < kRecF4; ++k) slab[lane * kRecF4 + (k ^ (lane & 7))] = rec[k];
        a.rect[i] = rect;
        mu_z = S.mu[2];
        if ((rect.x & 0xffffu) <= (rect.x >> 16)) {
            // The cover from the record's words (read back from the slab, so
            // the record's registers are free by now), stored for the binning.
            const float4 w4 = slab[lane * kRecF4 + (4 ^ (lane & 7))];
            const float4 w7 = slab[lane * kRecF4 + (7 ^ (lane & 7))];
            store_cover(a.cover, i, rect, w4.z, w4.w, w7.y, w7.z, w7.w);
            rcov = row_cover(rect, w4.z, w4.w, w7.y, w7.z, w7.w, a.tiles.cover == 0);
            row_lo = rect.y & 0xffffu;
            row_hi = rect.y >> 16;
        }
    }
    // Instances: per tile row of the rectangle, the tiles the ellipse reaches
    // (or the whole row). The warp deals out its (record, row) pairs 32 at a
    // time, so a splat with many rows does not hold up the other lanes.
    {
        __shared__ uint32_t s_cnt[kPreThreads];
        const int lane = threadIdx.x & 31;
        uint32_t *const wc = s_cnt + (threadIdx.x & ~31);
        wc[lane] = 0;
        __syncwarp();
        warp_cover_rows(rcov, row_lo, row_hi, lane, a.tiles.tile_w, a.tiles.tile_h,
                        [&](bool valid, uint32_t owner, uint32_t, uint32_t, uint32_t w) {
                            if (valid && w) atomicAdd(&wc[owner], w);
                        });
        __syncwarp();
        count = wc[lane];
    }
    if (i < b.n_rec) {
        a.count[i] = count;
        // Sorted blending: key = view-space mean depth (positive, so its float
        // bits order like the depth); records that emit nothing go last.
        if (a.dkey) {
            a.dkey[i] = count ? __float_as_uint(mu_z) : 0xffffffffu;
            a.dval[i] = (uint32_t)i;
            if (i == 0) *a.dtotal = (uint32_t)b.n_rec;
        }
    }
    // The warp's 32 records are contiguous in global memory: store them as
    // 4 KB of consecutive float4s.
    {
        const int lane = threadIdx.x & 31;
        const int64_t w0 = (int64_t)blockIdx.x * kPreThreads + (threadIdx.x & ~31);
        const float4 *slab = s_recs[threadIdx.x >> 5];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kRecF4; ++k) {
            const int idx = k * 32 + lane;    // float4 index inside the warp's 32 records
            const int r = idx / kRecF4, f = idx % kRecF4;
            if (w0 + r < b.n_rec) a.rec[w0 * kRecF4 + idx] = slab[r * kRecF4 + (f ^ (r & 7))];
        }
    }
    // Block sum of counts for the instance scan.
    __shared__ uint32_t warp_sums[kPreThreads / 32];
    __shared__ unsigned long long warp_px[kPreThreads / 32];
    uint32_t v = count;
    unsigned long long bp = box_pixels;
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        bp += __shfl_xor_sync(0xffffffffu, bp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        warp_sums[threadIdx.x >> 5] = v;
        warp_px[threadIdx.x >> 5] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        unsigned long long px = 0;
        for (int w = 0; w < kPreThreads / 32; ++w) {
            s += warp_sums[w];
            px += warp_px[w];
        }
        a.block_sums[blockIdx.x] = s;
        if (px) atomicAdd(a.stats + kStatBoxPairs, px);
    }
}

// ---------------------------------------------------------------------------
// K8: backward setup. acc holds per Gaussian 16 floats accumulated by the
// blend adjoint: dL/d(N coefficients)[6], dL/d(D coefficients)[6],
// sum(dL/dalpha * alpha) and dL/d(rgb)[3]. N = ||m||^2 and D = ||d||^2 are
// the quadratics of the Pluecker moment and direction (Eq. (13) gives
// rho^2 = N / D); alpha = o e^{-N/(2D)}, so dL/do = sum(dL/dalpha alpha)/o.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPreThreads)
preprocess_backward_kernel(const __grid_constant__ Batch b, PreBwdArgs a) {
    dependent_entry();
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    if (i >= b.n_rec) return;
    // Record i is Gaussian g of the scene that view v renders.
    const ViewDesc &V = b.v[view_of_record(b, i)];
    const int64_t g = i - V.rec_off;
    const CamArgs &cam = V.cam;
    const int nc = (V.sh_degree + 1) * (V.sh_degree + 1);
    float gmu[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
    float gsh[48];
    for (int k = 0; k < nc * 3; ++k) gsh[k] = 0.f;
    // Several views of one scene add their gradients; a scene of its own
    // view is written (which also zeroes Gaussians outside the view).
    auto emit = [&]() {
        float *pm = V.g_means + 3 * g, *pl = V.g_log_scales + 3 * g, *pq = V.g_quats + 4 * g;
        float *ps = V.g_sh + g * nc * 3;
        if (a.accumulate) {
            for (int k = 0; k < 3; ++k) { atomicAdd(pm + k, gmu[k]); atomicAdd(pl + k, gls[k]); }
            for (int k = 0; k < 4; ++k) atomicAdd(pq + k, gq[k]);
            atomicAdd(V.g_logits + g, glogit);
            for (int k = 0; k < nc * 3; ++k) atomicAdd(ps + k, gsh[k]);
        } else {
            for (int k = 0; k < 3; ++k) { pm[k] = gmu[k]; pl[k] = gls[k]; }
            for (int k = 0; k < 4; ++k) pq[k] = gq[k];
            V.g_logits[g] = glogit;
            for (int k = 0; k < nc * 3; ++k) ps[k] = gsh[k];
        }
    };
    Setup S;
    setup_geometry(V.means, V.log_scales, V.quats, V.logits, V.filter_var, g, cam, a.prm, S);
    const uint2 rect = a.rect[i];
    const bool active = S.valid && ((rect.x & 0xffffu) <= (rect.x >> 16));
    if (!active) {
        if (!a.accumulate) emit();
        return;
    }
    const float4 *acc4 = reinterpret_cast<const float4 *>(a.acc + 16 * i);
    const float4 A0 = acc4[0], A1 = acc4[1], A2 = acc4[2], A3 = acc4[3];
    // Interleaved pairs (dL/dN_k, dL/dD_k), k = 0..5, then the opacity and colour sums.
    const float gN[6] = {A0.x, A0.z, A1.x, A1.z, A2.x, A2.z};
    const float gD[6] = {A0.y, A0.w, A1.y, A1.w, A2.y, A2.w};
    const float g_aa = A3.x;
    const float gc[3] = {A3.y, A3.z, A3.w};

    const float4 r0 = a.rec[i * kRecF4 + 4]; // (z4, z5, xc, yc)
    Expansion E;
    make_expansion(S, cam, r0.z, r0.w, E);
    // N = n0 + n1 x' + ..., n0 = M0.M0, n1 = 2 M0.Mx, n2 = 2 M0.My, n3 = Mx.Mx,
    // n4 = 2 Mx.My, n5 = My.My; the same for D with the d vectors.
    const V3 dM0 = 2.f * (gN[0] * E.M0 + gN[1] * E.Mx + gN[2] * E.My);
    const V3 dMx = 2.f * (gN[1] * E.M0 + gN[3] * E.Mx + gN[4] * E.My);
    const V3 dMy = 2.f * (gN[2] * E.M0 + gN[4] * E.Mx + gN[5] * E.My);
    const V3 dD0 = 2.f * (gD[0] * E.D0 + gD[1] * E.Dx + gD[2] * E.Dy);
    const V3 dDx = 2.f * (gD[1] * E.D0 + gD[3] * E.Dx + gD[4] * E.Dy);
    const V3 dDy = 2.f * (gD[2] * E.D0 + gD[4] * E.Dx + gD[5] * E.Dy);
    V3 da = v3(0.f, 0.f, 0.f), db = da, dr = da;
    float daw = 0.f, dbw = 0.f, drw = 0.f;
    // M0 = aw b - bw a
    daw += dot(dM0, E.b); db = db + E.aw * dM0; dbw -= dot(dM0, E.a); da = da - E.bw * dM0;
    // Mx = bw r - rw b
    dbw += dot(dMx, E.r); dr = dr + E.bw * dMx; drw -= dot(dMx, E.b); db = db - E.rw * dMx;
    // My = rw a - aw r
    drw += dot(dMy, E.a); da = da + E.rw * dMy; daw -= dot(dMy, E.r); dr = dr - E.aw * dMy;
    // D0 = a x b, Dx = b x r, Dy = r x a
    da = da + cross(E.b, dD0); db = db + cross(dD0, E.a);
    db = db + cross(E.r, dDx); dr = dr + cross(dDx, E.b);
    dr = dr + cross(E.a, dDy); da = da + cross(dDy, E.r);
    // a = fx (MT)_1 + (cx - xc)(MT)_3, b = fy (MT)_2 + (cy - yc)(MT)_3, r = (MT)_3.
    const float ox = cam.cx - r0.z, oy = cam.cy - r0.w;
    V3 dA[3];
    float dmuv[3];
    dA[0] = cam.fx * da;             dmuv[0] = cam.fx * daw;
    dA[1] = cam.fy * db;             dmuv[1] = cam.fy * dbw;
    dA[2] = ox * da + oy * db + dr;  dmuv[2] = ox * daw + oy * dbw + drw;
    // A = M_rot B with B = R diag(s); mu_view = M_rot mu + t.
    float dB[3][3];
    for (int k = 0; k < 3; ++k) {
        const float c0 = cam.M[0 + k], c1 = cam.M[4 + k], c2 = cam.M[8 + k];
        dB[k][0] = c0 * dA[0].x + c1 * dA[1].x + c2 * dA[2].x;
        dB[k][1] = c0 * dA[0].y + c1 * dA[1].y + c2 * dA[2].y;
        dB[k][2] = c0 * dA[0].z + c1 * dA[1].z + c2 * dA[2].z;
        gmu[k] = c0 * dmuv[0] + c1 * dmuv[1] + c2 * dmuv[2];
    }
    float dR[3][3];
    for (int j = 0; j < 3; ++j) {
        float ds = 0.f;
        for (int k = 0; k < 3; ++k) {
            ds += dB[k][j] * S.R[k][j];
            dR[k][j] = dB[k][j] * S.s[j];
        }
        // s' = sqrt(s^2 + v): d s'/d log s = s^2 / s'; and the filtered
        // opacity o' = o prod s / s' has d o'/d log s = o' v / s'^2, with
        // dL/do' = g_aa / o'.
        gls[j] = ds * S.s_raw[j] * S.s_raw[j] / S.s[j] + A3.x * S.fvar / (S.s[j] * S.s[j]);
    }
    const float w = S.q[0], x = S.q[1], y = S.q[2], z = S.q[3];
    float dq[4];
    dq[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    dq[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                   z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    dq[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                   w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    dq[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                   y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float pdot = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
    const float iq = 1.f / S.qnorm;
    for (int k = 0; k < 4; ++k) gq[k] = (dq[k] - S.q[k] * pdot) * iq;
    // o' = sigmoid(l) prod s / s': dL/dl = (sum dL/dalpha alpha / o') o' (1 - sigmoid(l)).
    glogit = g_aa * (1.f - S.o_raw);
    // Colour: channels clamped at zero pass no gradient.
    float Y[16];
    sh_eval(S.dir[0], S.dir[1], S.dir[2], V.sh_degree, Y);
    const float *sh = V.sh + g * nc * 3;
    float raw[3] = {0.5f, 0.5f, 0.5f};
    for (int k = 0; k < nc; ++k)
        for (int ch = 0; ch < 3; ++ch) raw[ch] += Y[k] * sh[3 * k + ch];
    float gce[3];
    for (int ch = 0; ch < 3; ++ch) gce[ch] = raw[ch] > 0.f ? gc[ch] : 0.f;
    float wdir[16];
    for (int k = 0; k < 16; ++k) wdir[k] = 0.f;
    for (int k = 0; k < nc; ++k) {
        for (int ch = 0; ch < 3; ++ch) gsh[3 * k + ch] = gce[ch] * Y[k];
        wdir[k] = gce[0] * sh[3 * k] + gce[1] * sh[3 * k + 1] + gce[2] * sh[3 * k + 2];
    }
    float gd[3];
    sh_grad(S.dir[0], S.dir[1], S.dir[2], V.sh_degree, wdir, gd);
    if (S.dist > 0.f) {
        const float pd = gd[0] * S.dir[0] + gd[1] * S.dir[1] + gd[2] * S.dir[2];
        const float id = 1.f / S.dist;
        for (int k = 0; k < 3; ++k) gmu[k] += (gd[k] - S.dir[k] * pd) * id;
    }
    // Training statistics of this view (Sec. 4.2): the mean's gradient times
    // half the camera distance, the view count and the largest blending weight.
    if (V.g_dgrad)
        atomicAdd(V.g_dgrad + g, 0.5f * S.dist * sqrtf(gmu[0] * gmu[0] + gmu[1] * gmu[1] + gmu[2] * gmu[2]));
    if (V.g_dcount) atomicAdd(V.g_dcount + g, 1.f);
    if (V.g_vis && a.vis) {
        const float w = a.vis[i];
        if (w > 0.f) atomicMax(reinterpret_cast<int *>(V.g_vis) + g, __float_as_int(w));
    }
    emit();
}

void launch_preprocess(bool any_baked, int blocks, const Batch &b, const PreArgs &a, cudaStream_t s) {
    if (any_baked)
        launch_k(preprocess_kernel<true>, blocks, kPreThreads, 0, s, b, a);
    else
        launch_k(preprocess_kernel<false>, blocks, kPreThreads, 0, s, b, a);
}

} // namespace htgs
