/*
 * htgs_oracle.c -- FP64 brute-force reference renderer for perspective-correct
 * 3D Gaussian splatting with hybrid transparency (arXiv 2410.08129).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it. It shares no code with the CUDA path.
 *
 * Every quantity is computed in double precision, in the order and notation
 * of the paper:
 *   - Sec. 3.1: scene representation (sigmoid opacity, log-scales, normalised
 *     quaternion, SH colour identical to 3DGS) and Eq. (1)/(2) alpha blending.
 *   - Sec. 3.2, Eq. (3): T = [s_u t_u, s_v t_v, s_w t_w, mu; 0 0 0 1],
 *     T' = V P M T; the tight screen bounding box (p_i, h_i) with the
 *     opacity-aware cutoff rho_c = 2 ln(o / tau_alpha).
 *   - Sec. 3.2, Eq. (9)-(13): the pixel ray as the planes pi_x, pi_y mapped
 *     by T'^T, the Pluecker coordinates p^{ij} and
 *     rho^2 = ||(p^{01}, p^{02}, p^{03})||^2 / ||(p^{23}, p^{31}, p^{12})||^2.
 *   - Sec. 3.3, Eq. (14)-(16): the per-pixel view-space depth of the point of
 *     maximum contribution and the hybrid-transparency colour
 *     C = sum_{i<=K} alpha_i T_i c_i + T_{K+1}((1 - T_tail) c_tail + T_tail c_bg).
 *   - Sec. 4.2: K and the core admission threshold tau_K.
 * Every pixel is tested against every Gaussian (no bounding boxes, no tiles).
 *
 * Readings where the paper is silent (they are stated again in the design
 * notes): pixel centres at (i + 0.5, j + 0.5); a fragment is kept iff
 * rho^2 <= rho_c; alpha is clamped to alpha_max; a Gaussian is culled when
 * rho_c <= 0 or when its cutoff ellipsoid reaches z <= z_near; core ties are
 * broken by (z, gid); an empty tail has c_tail = 0; the colour is
 * max(0, 0.5 + sum_lm Y_lm(dir) k_lm) with dir from the camera centre to the
 * mean.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Interface types (mirrored by ctypes in oracle/__init__.py)               */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *means;      /* N x 3 */
    const double *log_scales; /* N x 3 */
    const double *quats;      /* N x 4, (w, x, y, z) */
    const double *logits;     /* N */
    const double *sh;         /* N x (deg+1)^2 x 3 */
    int64_t n;
    int32_t sh_degree;
    const double *filter_var; /* N or NULL: variance of the 3D smoothing filter */
} og_gaussians;

typedef struct {
    double world_to_cam[16]; /* row-major; OpenCV axes */
    double fx, fy, cx, cy, z_near;
    int32_t width, height;
} og_camera;

typedef struct {
    int32_t K;
    double tau_alpha, tau_K, alpha_max;
    double bg[3];
    int32_t no_tail; /* 1: inference without the tail (Sec. 4.4): C = core + T_{K+1} bg */
    int32_t sorted_blend; /* 1: Tab. 3 "w/o per-pixel HT": fragments in order of their Gaussian's
                             view-space mean depth, sorted alpha blending, early termination */
} og_params;

typedef struct {
    int32_t x0, y0, w, h; /* pixel window [x0, x0+w) x [y0, y0+h) */
} og_window;

/* Per-Gaussian setup (Sec. 3.2). */
typedef struct {
    int32_t valid;       /* 1 = rendered, 0 = culled */
    int32_t cull_reason; /* 0 none, 1 rho_c <= 0, 2 near plane */
    double cull_margin;  /* signed distance of the deciding quantity to its threshold */
    double o, rho_c;
    double s[3];         /* exp(log-scales) */
    double q[4];         /* normalised quaternion (w, x, y, z) */
    double R[3][3];      /* columns t_u, t_v, t_w */
    double MT[4][4];     /* M T */
    double r1[4], r2[4], r4[4]; /* rows 1, 2, 4 of T' = V P M T */
    double p[2], h[2];   /* bounding-box centre and half extent in x and y */
    int32_t rect[4];     /* covered pixel rectangle: x_min, x_max, y_min, y_max (inclusive) */
    double dir[3];       /* unit direction camera centre -> mean */
    double dist;         /* |mean - camera centre| */
    double rgb_raw[3];   /* 0.5 + SH sum, before the clamp */
    double rgb[3];       /* colour */
    double o_raw;        /* sigmoid(logit) before the 3D filter (o = o_raw without one) */
    double s_raw[3];     /* exp(log-scales) before the 3D filter */
    double filter_var;   /* the 3D filter's variance (0 without one) */
} og_splat;

/* Optional per-pixel diagnostics of og_render (each pointer may be NULL). */
typedef struct {
    int32_t *n_frag;       /* w*h: fragments with rho^2 <= rho_c */
    int32_t *n_core;       /* w*h */
    int32_t *core_gid;     /* w*h*K, depth order, -1 padded */
    double *T_core;        /* w*h: T_{K+1} (transmittance behind the core) */
    double *T_tail;        /* w*h */
    double *A_tail;        /* w*h: sum of tail alphas */
    double *c_tail;        /* w*h*3 */
    int32_t *ambiguous;    /* w*h: near-decisions whose flip moves the colour by > 2e-5 */
    uint64_t *frag_hash;   /* w*h: order-independent hash of the fragment gid set */
    int32_t *near_decision;/* w*h: every near-decision, whatever its effect on the colour */
    double *amb_effect;    /* w*h: sum over the pixel's near-decisions of the largest channel
                              change that flipping that one decision alone makes to the colour */
} og_pixel_diag;

/* Near-decision flags. A discrete decision that single precision may take
   the other way: the cutoff rho^2 <= rho_c, core admission alpha >= tau_K,
   the alpha clamp, and the depth order at and inside the core. Bits of
   og_pixel_diag.near_decision mark every such event; bits of
   og_pixel_diag.ambiguous mark those whose flip changes the pixel colour by
   more than OG_EFFECT_TOL (found by blending the pixel again with the
   decision flipped). */
enum {
    OG_AMB_CUTOFF = 1,   /* |rho^2 - rho_c| <= 4e-6 max(1, rho_c) */
    OG_AMB_TAUK = 2,     /* |alpha - tau_K| <= 2e-6 */
    OG_AMB_AMAX = 4,     /* |o e^{-rho^2/2} - alpha_max| <= 1e-6 */
    OG_AMB_CORE_EDGE = 8,/* K-th and (K+1)-th candidate depths within 1e-6 |z| */
    OG_AMB_CORE_TIE = 16,/* two adjacent core depths within 1e-6 |z| */
    OG_AMB_DEN = 32,     /* ray nearly parallel to a flat splat: den tiny relative to its scale */
    OG_AMB_TERM = 64,    /* sorted blending: T (1 - alpha) within 1e-6 relative of the termination threshold */
    OG_AMB_ORDER = 128   /* sorted blending: two used fragments' mean depths within 1e-6 |z| */
};
/* Sorted blending stops before the fragment that would take T below this. */
#define OG_SORTED_TMIN 1e-4
#define OG_CUTOFF_REL 4e-6
#define OG_TAUK_ABS 2e-6
#define OG_AMAX_ABS 1e-6
#define OG_DEPTH_REL 1e-6
#define OG_EFFECT_TOL 2e-5

/* ------------------------------------------------------------------------ */
/* Threading                                                                */
/* ------------------------------------------------------------------------ */

static int og_threads_override = 0;

void og_set_threads(int n) { og_threads_override = n; }

int og_get_threads(void) {
    if (og_threads_override > 0) return og_threads_override;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

typedef void (*og_task_fn)(void *ctx, int64_t begin, int64_t end);

typedef struct {
    og_task_fn fn;
    void *ctx;
    int64_t count;
    int64_t chunk;
    int64_t next;
    pthread_mutex_t lock;
} og_pool_job;

static void *og_worker(void *arg) {
    og_pool_job *job = (og_pool_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t b = job->next;
        job->next += job->chunk;
        pthread_mutex_unlock(&job->lock);
        if (b >= job->count) break;
        int64_t e = b + job->chunk < job->count ? b + job->chunk : job->count;
        job->fn(job->ctx, b, e);
    }
    return NULL;
}

static void og_parallel_for(int64_t count, int64_t chunk, og_task_fn fn, void *ctx) {
    int nt = og_get_threads();
    if (nt > 256) nt = 256;
    og_pool_job job;
    job.fn = fn;
    job.ctx = ctx;
    job.count = count;
    job.chunk = chunk > 0 ? chunk : 1;
    job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (nt <= 1 || count <= job.chunk) {
        og_worker(&job);
    } else {
        pthread_t th[256];
        int started = 0;
        for (int i = 0; i < nt - 1; ++i)
            if (pthread_create(&th[i], NULL, og_worker, &job) == 0) ++started;
        og_worker(&job);
        for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    }
    pthread_mutex_destroy(&job.lock);
}

/* ------------------------------------------------------------------------ */
/* Spherical harmonics (Sec. 3.1: "identical to 3DGS")                      */
/* ------------------------------------------------------------------------ */
/*
 * Real spherical harmonics up to degree 3 in the order m = -l..l, built from
 * the complex Y_l^m (Condon-Shortley phase included) as
 * Y_{l,-|m|} = sqrt(2) Im Y_l^{|m|}, Y_{l,0} = Y_l^0, Y_{l,|m|} = sqrt(2) Re Y_l^{|m|},
 * written as polynomials in the unit direction (x, y, z). The normalisation
 * constants are the closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times
 * the Legendre factors.
 */
void og_sh_basis(const double dir[3], int degree, double Y[16], double dY[16][3]) {
    const double pi = 3.14159265358979323846;
    const double x = dir[0], y = dir[1], z = dir[2];
    const double c0 = 0.5 / sqrt(pi);              /* 1/(2 sqrt(pi)) */
    const double c1 = sqrt(3.0 / (4.0 * pi));
    const double c2a = sqrt(15.0 / (4.0 * pi));
    const double c2b = sqrt(5.0 / (16.0 * pi));
    const double c2c = sqrt(15.0 / (16.0 * pi));
    const double c3a = sqrt(35.0 / (32.0 * pi));
    const double c3b = sqrt(105.0 / (4.0 * pi));
    const double c3c = sqrt(21.0 / (32.0 * pi));
    const double c3d = sqrt(7.0 / (16.0 * pi));
    const double c3e = sqrt(105.0 / (16.0 * pi));
    double Yl[16] = {0};
    double G[16][3] = {{0}};
    Yl[0] = c0;
    if (degree >= 1) {
        Yl[1] = -c1 * y;  G[1][1] = -c1;
        Yl[2] = c1 * z;   G[2][2] = c1;
        Yl[3] = -c1 * x;  G[3][0] = -c1;
    }
    if (degree >= 2) {
        Yl[4] = c2a * x * y;                  G[4][0] = c2a * y; G[4][1] = c2a * x;
        Yl[5] = -c2a * y * z;                 G[5][1] = -c2a * z; G[5][2] = -c2a * y;
        Yl[6] = c2b * (2 * z * z - x * x - y * y);
        G[6][0] = -2 * c2b * x; G[6][1] = -2 * c2b * y; G[6][2] = 4 * c2b * z;
        Yl[7] = -c2a * x * z;                 G[7][0] = -c2a * z; G[7][2] = -c2a * x;
        Yl[8] = c2c * (x * x - y * y);        G[8][0] = 2 * c2c * x; G[8][1] = -2 * c2c * y;
    }
    if (degree >= 3) {
        Yl[9] = -c3a * y * (3 * x * x - y * y);
        G[9][0] = -c3a * 6 * x * y; G[9][1] = -c3a * (3 * x * x - 3 * y * y);
        Yl[10] = c3b * x * y * z;
        G[10][0] = c3b * y * z; G[10][1] = c3b * x * z; G[10][2] = c3b * x * y;
        Yl[11] = -c3c * y * (4 * z * z - x * x - y * y);
        G[11][0] = -c3c * (-2 * x * y); G[11][1] = -c3c * (4 * z * z - x * x - 3 * y * y);
        G[11][2] = -c3c * 8 * y * z;
        Yl[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
        G[12][0] = c3d * (-6 * x * z); G[12][1] = c3d * (-6 * y * z);
        G[12][2] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
        Yl[13] = -c3c * x * (4 * z * z - x * x - y * y);
        G[13][0] = -c3c * (4 * z * z - 3 * x * x - y * y); G[13][1] = -c3c * (-2 * x * y);
        G[13][2] = -c3c * 8 * x * z;
        Yl[14] = c3e * z * (x * x - y * y);
        G[14][0] = c3e * 2 * x * z; G[14][1] = -c3e * 2 * y * z; G[14][2] = c3e * (x * x - y * y);
        Yl[15] = -c3a * x * (x * x - 3 * y * y);
        G[15][0] = -c3a * (3 * x * x - 3 * y * y); G[15][1] = -c3a * (-6 * x * y);
    }
    for (int k = 0; k < 16; ++k) {
        if (Y) Y[k] = Yl[k];
        if (dY)
            for (int j = 0; j < 3; ++j) dY[k][j] = G[k][j];
    }
}

/* ------------------------------------------------------------------------ */
/* Per-Gaussian setup (Sec. 3.1, Sec. 3.2 Eq. (3) and the bounding box)     */
/* ------------------------------------------------------------------------ */

static void og_camera_centre(const og_camera *cam, double c[3]) {
    /* world_to_cam = [Rwc | t]; the centre is -Rwc^T t. */
    const double *M = cam->world_to_cam;
    for (int i = 0; i < 3; ++i)
        c[i] = -(M[0 * 4 + i] * M[3] + M[1 * 4 + i] * M[7] + M[2 * 4 + i] * M[11]);
}

static void og_setup_one(const og_gaussians *g, const og_camera *cam, const og_params *prm,
                         int64_t i, og_splat *out) {
    memset(out, 0, sizeof(*out));
    const double *mu = g->means + 3 * i;
    /* Sec. 3.1: sigmoid opacity, log-space scales, normalised quaternion. */
    out->o = 1.0 / (1.0 + exp(-g->logits[i]));
    for (int k = 0; k < 3; ++k) out->s[k] = exp(g->log_scales[3 * i + k]);
    /* 3D smoothing filter (Sec. 4.2, after Yu et al.): the Gaussian is
       convolved with an isotropic Gaussian of variance v, Sigma + v I =
       R diag(s^2 + v) R^T, and its opacity is scaled by
       sqrt(det Sigma / det (Sigma + v I)) so that its integral is kept. */
    out->o_raw = out->o;
    for (int k = 0; k < 3; ++k) out->s_raw[k] = out->s[k];
    out->filter_var = g->filter_var ? g->filter_var[i] : 0.0;
    if (g->filter_var) {
        for (int k = 0; k < 3; ++k) {
            const double sf = sqrt(out->s_raw[k] * out->s_raw[k] + out->filter_var);
            out->o *= out->s_raw[k] / sf;
            out->s[k] = sf;
        }
    }
    const double *qr = g->quats + 4 * i;
    double qn = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    for (int k = 0; k < 4; ++k) out->q[k] = qr[k] / qn;
    const double w = out->q[0], x = out->q[1], y = out->q[2], z = out->q[3];
    /* Rotation of the unit quaternion; its columns are t_u, t_v, t_w. */
    out->R[0][0] = 1 - 2 * (y * y + z * z); out->R[0][1] = 2 * (x * y - w * z); out->R[0][2] = 2 * (x * z + w * y);
    out->R[1][0] = 2 * (x * y + w * z); out->R[1][1] = 1 - 2 * (x * x + z * z); out->R[1][2] = 2 * (y * z - w * x);
    out->R[2][0] = 2 * (x * z - w * y); out->R[2][1] = 2 * (y * z + w * x); out->R[2][2] = 1 - 2 * (x * x + y * y);

    /* Eq. (3): T = [s_u t_u, s_v t_v, s_w t_w, mu; 0 0 0 1]. */
    double T[4][4] = {{0}};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) T[r][c] = out->s[c] * out->R[r][c];
        T[r][3] = mu[r];
    }
    T[3][3] = 1.0;
    /* M T with the model-view matrix M = world_to_cam. */
    const double *M = cam->world_to_cam;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0;
            for (int k = 0; k < 4; ++k) acc += M[r * 4 + k] * T[k][c];
            out->MT[r][c] = acc;
        }
    /* V P for a pinhole camera in window coordinates: screen x w = fx X + cx Z,
       y w = fy Y + cy Z, w = Z. Only rows 1, 2 and 4 of T' enter the bounding
       box in x, y and the ray planes (whose z coefficient is 0). */
    for (int c = 0; c < 4; ++c) {
        out->r1[c] = cam->fx * out->MT[0][c] + cam->cx * out->MT[2][c];
        out->r2[c] = cam->fy * out->MT[1][c] + cam->cy * out->MT[2][c];
        out->r4[c] = out->MT[2][c];
    }

    /* Opacity-aware cutoff (Sec. 3.2, after Radl et al.). */
    out->rho_c = 2.0 * log(out->o / prm->tau_alpha);
    out->valid = 1;
    if (!(out->rho_c > 0.0)) {
        out->valid = 0;
        out->cull_reason = 1;
        out->cull_margin = out->rho_c;
    } else {
        /* Near plane: cull when the cutoff ellipsoid reaches z <= z_near. Its
           view-z extent is mu_z +- sqrt(rho_c * sum_k (MT)_{3k}^2). */
        double e2 = 0;
        for (int k = 0; k < 3; ++k) e2 += out->MT[2][k] * out->MT[2][k];
        double zmin = out->MT[2][3] - sqrt(out->rho_c * e2);
        out->cull_margin = zmin - cam->z_near;
        if (!(zmin > cam->z_near)) {
            out->valid = 0;
            out->cull_reason = 2;
        }
    }

    /* Tight bounding box (Sec. 3.2): s = <(rc, rc, rc, -1), T'_4 . T'_4>,
       f = (rc, rc, rc, -1)/s, p_i = <f, T'_i . T'_4>, h_i = sqrt(p_i^2 - <f, T'_i . T'_i>). */
    if (out->valid) {
        const double rc = out->rho_c;
        const double fv[4] = {rc, rc, rc, -1.0};
        double sd = 0;
        for (int k = 0; k < 4; ++k) sd += fv[k] * out->r4[k] * out->r4[k];
        double f[4];
        for (int k = 0; k < 4; ++k) f[k] = fv[k] / sd;
        const double *rows[2] = {out->r1, out->r2};
        for (int a = 0; a < 2; ++a) {
            double pi = 0, qi = 0;
            for (int k = 0; k < 4; ++k) {
                pi += f[k] * rows[a][k] * out->r4[k];
                qi += f[k] * rows[a][k] * rows[a][k];
            }
            double disc = pi * pi - qi;
            out->p[a] = pi;
            out->h[a] = disc > 0 ? sqrt(disc) : 0.0;
        }
        /* Pixel (i, j) has its centre at (i + 0.5, j + 0.5); it is covered
           iff the centre lies in [p - h, p + h]. */
        int lim[2] = {cam->width, cam->height};
        for (int a = 0; a < 2; ++a) {
            double lo = ceil(out->p[a] - out->h[a] - 0.5);
            double hi = floor(out->p[a] + out->h[a] - 0.5);
            if (lo < 0) lo = 0;
            if (hi > lim[a] - 1) hi = lim[a] - 1;
            out->rect[2 * a] = (int32_t)(lo > 1e9 ? 1e9 : lo);
            out->rect[2 * a + 1] = (int32_t)(hi < -1e9 ? -1e9 : hi);
        }
    } else {
        out->rect[0] = 0; out->rect[1] = -1; out->rect[2] = 0; out->rect[3] = -1;
    }

    /* View-dependent colour: dir from the camera centre to the mean. */
    double cc[3];
    og_camera_centre(cam, cc);
    double v[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    out->dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) out->dir[k] = out->dist > 0 ? v[k] / out->dist : 0.0;
    double Y[16];
    og_sh_basis(out->dir, g->sh_degree, Y, NULL);
    const int nc = (g->sh_degree + 1) * (g->sh_degree + 1);
    const double *shc = g->sh + (int64_t)i * nc * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < nc; ++k) acc += Y[k] * shc[k * 3 + ch];
        out->rgb_raw[ch] = acc;
        out->rgb[ch] = acc > 0 ? acc : 0.0;
    }
}

typedef struct {
    const og_gaussians *g;
    const og_camera *cam;
    const og_params *prm;
    og_splat *out;
} og_setup_ctx;

static void og_setup_task(void *vctx, int64_t b, int64_t e) {
    og_setup_ctx *c = (og_setup_ctx *)vctx;
    for (int64_t i = b; i < e; ++i) og_setup_one(c->g, c->cam, c->prm, i, &c->out[i]);
}

int og_preprocess(const og_gaussians *g, const og_camera *cam, const og_params *prm, og_splat *out) {
    if (!g || !cam || !prm || !out || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return 1;
    og_setup_ctx c = {g, cam, prm, out};
    og_parallel_for(g->n, 4096, og_setup_task, &c);
    return 0;
}

int og_splat_size(void) { return (int)sizeof(og_splat); }

/* ------------------------------------------------------------------------ */
/* Ray-splat evaluation (Sec. 3.2, Eq. (9)-(13); Sec. 3.3, Eq. (14))        */
/* ------------------------------------------------------------------------ */

typedef struct {
    double a[4], b[4];      /* splat-space planes; index 0..2 = a^1..a^3, index 3 = a^0 */
    double d[3], m[3];      /* Pluecker direction and moment */
    double num, den, rho2;
    double xmax[3];         /* point of maximum contribution in splat space */
    double z;               /* its view-space depth */
} og_eval;

/* Returns 1 when the ray meets the splat (den != 0), filling ev. */
static int og_evaluate(const og_splat *sp, double xs, double ys, og_eval *ev) {
    /* pi^s = T'^T pi with pi_x = (1, 0, 0, -xs), pi_y = (0, 1, 0, -ys):
       a = T'_1 - xs T'_4, b = T'_2 - ys T'_4. */
    for (int k = 0; k < 4; ++k) {
        ev->a[k] = sp->r1[k] - xs * sp->r4[k];
        ev->b[k] = sp->r2[k] - ys * sp->r4[k];
    }
    /* Coefficients in the paper's naming: (a^1 : a^2 : a^3 : a^0). */
    const double a0 = ev->a[3], a1 = ev->a[0], a2 = ev->a[1], a3 = ev->a[2];
    const double b0 = ev->b[3], b1 = ev->b[0], b2 = ev->b[1], b3 = ev->b[2];
    /* p^{ij} = a^i b^j - a^j b^i. */
    const double p23 = a2 * b3 - a3 * b2;
    const double p31 = a3 * b1 - a1 * b3;
    const double p12 = a1 * b2 - a2 * b1;
    const double p01 = a0 * b1 - a1 * b0;
    const double p02 = a0 * b2 - a2 * b0;
    const double p03 = a0 * b3 - a3 * b0;
    /* (d : m) = (p^{23}, p^{31}, p^{12} : p^{01}, p^{02}, p^{03}) up to a common scale. */
    ev->d[0] = p23; ev->d[1] = p31; ev->d[2] = p12;
    ev->m[0] = p01; ev->m[1] = p02; ev->m[2] = p03;
    ev->den = p23 * p23 + p31 * p31 + p12 * p12;
    ev->num = p01 * p01 + p02 * p02 + p03 * p03;
    if (ev->den == 0.0) return 0; /* the ray misses the splat */
    ev->rho2 = ev->num / ev->den;
    /* Closest point of the line to the origin: (d x m) / ||d||^2; its view
       depth is row 3 of M T applied to (x, 1), which is T'_4 for a pinhole. */
    const double *d = ev->d, *m = ev->m;
    ev->xmax[0] = (d[1] * m[2] - d[2] * m[1]) / ev->den;
    ev->xmax[1] = (d[2] * m[0] - d[0] * m[2]) / ev->den;
    ev->xmax[2] = (d[0] * m[1] - d[1] * m[0]) / ev->den;
    ev->z = sp->MT[2][0] * ev->xmax[0] + sp->MT[2][1] * ev->xmax[1] + sp->MT[2][2] * ev->xmax[2] + sp->MT[2][3];
    return 1;
}

/* Evaluate one (Gaussian, pixel) pair for external pin tests. Returns 1 on a
   hit, and writes rho2, z, the unclamped alpha o e^{-rho^2/2}, den, num. */
int og_eval_pair(const og_splat *sp, double xs, double ys, double out[5]) {
    og_eval ev;
    int hit = og_evaluate(sp, xs, ys, &ev);
    out[0] = hit ? ev.rho2 : INFINITY;
    out[1] = hit ? ev.z : NAN;
    out[2] = hit ? sp->o * exp(-0.5 * ev.rho2) : 0.0;
    out[3] = ev.den;
    out[4] = ev.num;
    return hit;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel hybrid transparency (Sec. 3.3, Eq. (15)-(16); Sec. 4.2)        */
/* ------------------------------------------------------------------------ */

typedef struct {
    double z, alpha, a_raw, rho2;
    double c[3];
    int64_t gid;
    int32_t force; /* hybrid: 0 core admission by alpha >= tau_K, +1 / -1 forced in / out;
                      sorted blending: +1 never stop at this fragment, -1 stop before it */
    double zmean;  /* view-space depth of the Gaussian's mean (sorted blending) */
} og_frag;

static int og_frag_cmp(const void *pa, const void *pb) {
    const og_frag *a = (const og_frag *)pa, *b = (const og_frag *)pb;
    if (a->z < b->z) return -1;
    if (a->z > b->z) return 1;
    return (a->gid > b->gid) - (a->gid < b->gid);
}

typedef struct {
    og_frag *f;
    int64_t n, cap;
} og_fragvec;

static int og_push(og_fragvec *v, const og_frag *x) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 64;
        og_frag *p = (og_frag *)realloc(v->f, (size_t)nc * sizeof(og_frag));
        if (!p) return 1;
        v->f = p;
        v->cap = nc;
    }
    v->f[v->n++] = *x;
    return 0;
}

/* Fragment decision for one pair: kept iff the ray meets the splat and
   rho^2 <= rho_c (equivalently o e^{-rho^2/2} >= tau_alpha). Returns 1 when
   kept; *border is set when rho^2 lies within OG_CUTOFF_REL of rho_c (then fr
   is filled even for a rejected pair, so that the flip can be evaluated). */
static int og_fragment(const og_splat *sp, int64_t gid, double xs, double ys, const og_params *prm,
                       og_frag *fr, int32_t *amb, int *border) {
    og_eval ev;
    if (border) *border = 0;
    if (!og_evaluate(sp, xs, ys, &ev)) return 0;
    const double rc = sp->rho_c;
    const int near_cut = fabs(ev.rho2 - rc) <= OG_CUTOFF_REL * (rc > 1 ? rc : 1);
    if (border) *border = near_cut;
    const int kept = ev.rho2 <= rc;
    if (!kept && !near_cut) return 0;
    fr->z = ev.z;
    fr->zmean = sp->MT[2][3];
    fr->rho2 = ev.rho2;
    fr->a_raw = sp->o * exp(-0.5 * ev.rho2);
    fr->alpha = fr->a_raw < prm->alpha_max ? fr->a_raw : prm->alpha_max;
    fr->force = 0;
    for (int ch = 0; ch < 3; ++ch) fr->c[ch] = sp->rgb[ch];
    fr->gid = gid;
    if (kept && amb) {
        if (fabs(fr->alpha - prm->tau_K) <= OG_TAUK_ABS) *amb |= OG_AMB_TAUK;
        if (fabs(fr->a_raw - prm->alpha_max) <= OG_AMAX_ABS) *amb |= OG_AMB_AMAX;
        /* A kept pair whose den is tiny compared with |a||b| is a ray almost
           parallel to a flat splat; FP32 evaluation cannot resolve it. */
        double na = 0, nb = 0;
        for (int k = 0; k < 3; ++k) { na += ev.a[k] * ev.a[k]; nb += ev.b[k] * ev.b[k]; }
        if (ev.den <= 1e-8 * na * nb) *amb |= OG_AMB_DEN;
    }
    return kept;
}

/* Result of blending one pixel; the core is sorted by (z, gid). */
typedef struct {
    double C[3];
    int64_t n_frag, n_core;
    double T_core;        /* T_{n_core + 1} */
    double T_tail, A_tail, c_tail[3];
    int32_t amb;
    uint64_t hash;
} og_pixel_result;

static uint64_t og_mix(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

static int og_frag_cmp_mean(const void *pa, const void *pb) {
    const og_frag *a = (const og_frag *)pa, *b = (const og_frag *)pb;
    if (a->zmean < b->zmean) return -1;
    if (a->zmean > b->zmean) return 1;
    return (a->gid > b->gid) - (a->gid < b->gid);
}

/* Tab. 3 "w/o per-pixel HT": the perspective-correct fragments blended front
   to back in the order of their Gaussians' view-space mean depth (then gid),
   Eq. (2) plus background, stopping before the fragment that would take the
   transmittance below OG_SORTED_TMIN. On return F->f[0 .. n_core) holds the
   blended fragments in order (the "core"; there is no tail). */
static void og_blend_sorted(og_fragvec *F, const og_params *prm, og_pixel_result *res) {
    res->n_frag = F->n;
    res->hash = 0;
    for (int64_t i = 0; i < F->n; ++i) res->hash += og_mix((uint64_t)F->f[i].gid + 0x9e3779b97f4a7c15ULL);
    qsort(F->f, (size_t)F->n, sizeof(og_frag), og_frag_cmp_mean);
    double C[3] = {0, 0, 0}, T = 1.0;
    int64_t used = 0;
    for (int64_t i = 0; i < F->n; ++i) {
        const og_frag *f = &F->f[i];
        const double Tn = T * (1.0 - f->alpha);
        /* The order of the last blended fragment and the first one left out
           also decides the result, so that pair is checked before the stop. */
        if (i > 0 && fabs(f->zmean - F->f[i - 1].zmean) <= OG_DEPTH_REL * fabs(f->zmean)) res->amb |= OG_AMB_ORDER;
        if (fabs(Tn - OG_SORTED_TMIN) <= 1e-6 * OG_SORTED_TMIN + 1e-7 * T) res->amb |= OG_AMB_TERM;
        if (f->force < 0 || (Tn < OG_SORTED_TMIN && f->force <= 0)) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += f->alpha * T * f->c[ch];
        T = Tn;
        ++used;
    }
    res->n_core = used;
    res->T_core = T;
    res->T_tail = 1.0;
    res->A_tail = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        res->c_tail[ch] = 0.0;
        res->C[ch] = C[ch] + T * prm->bg[ch];
    }
}

/* Splits the fragment list F into core and tail and composites, Eq. (15)-(16).
   On return F->f[0 .. n_core) holds the core in depth order. */
static void og_blend(og_fragvec *F, const og_params *prm, og_pixel_result *res) {
    if (prm->sorted_blend) {
        og_blend_sorted(F, prm, res);
        return;
    }
    const int K = prm->K;
    res->n_frag = F->n;
    res->hash = 0;
    for (int64_t i = 0; i < F->n; ++i) res->hash += og_mix((uint64_t)F->f[i].gid + 0x9e3779b97f4a7c15ULL);
    /* Candidates for the core: alpha >= tau_K; sorted by (z, gid). Move them
       to the front (keeping the rest as the tail). */
    int64_t nc = 0;
    for (int64_t i = 0; i < F->n; ++i)
        if (F->f[i].force > 0 || (F->f[i].force == 0 && F->f[i].alpha >= prm->tau_K)) {
            og_frag t = F->f[nc]; F->f[nc] = F->f[i]; F->f[i] = t;
            ++nc;
        }
    qsort(F->f, (size_t)nc, sizeof(og_frag), og_frag_cmp);
    int64_t n_core = nc < K ? nc : K;
    if (nc > K && K > 0) {
        double zk = F->f[K - 1].z, zk1 = F->f[K].z;
        if (fabs(zk1 - zk) <= OG_DEPTH_REL * fabs(zk)) res->amb |= OG_AMB_CORE_EDGE;
    }
    for (int64_t i = 0; i + 1 < n_core; ++i)
        if (fabs(F->f[i + 1].z - F->f[i].z) <= OG_DEPTH_REL * fabs(F->f[i].z)) res->amb |= OG_AMB_CORE_TIE;
    res->n_core = n_core;

    /* Core: sorted alpha blending, T_1 = 1, T_{i+1} = T_i (1 - alpha_i). */
    double C[3] = {0, 0, 0};
    double T = 1.0;
    for (int64_t i = 0; i < n_core; ++i) {
        const og_frag *f = &F->f[i];
        for (int ch = 0; ch < 3; ++ch) C[ch] += f->alpha * T * f->c[ch];
        T *= 1.0 - f->alpha;
    }
    res->T_core = T;
    /* Tail: every other fragment, in any order (none when it is omitted). */
    double A = 0, S[3] = {0, 0, 0}, Tt = 1.0;
    for (int64_t i = n_core; i < F->n && !prm->no_tail; ++i) {
        const og_frag *f = &F->f[i];
        A += f->alpha;
        for (int ch = 0; ch < 3; ++ch) S[ch] += f->alpha * f->c[ch];
        Tt *= 1.0 - f->alpha;
    }
    res->A_tail = A;
    res->T_tail = Tt;
    for (int ch = 0; ch < 3; ++ch) {
        res->c_tail[ch] = A > 0 ? S[ch] / A : 0.0;
        res->C[ch] = C[ch] + T * ((1.0 - Tt) * res->c_tail[ch] + Tt * prm->bg[ch]);
    }
}

typedef struct {
    const og_splat *sp;
    int64_t n;
    const og_camera *cam;
    const og_params *prm;
    og_window win;
    double *image;
    og_pixel_diag *diag;
    int err;
    const int64_t *idx;   /* NULL: every Gaussian; else the n_idx Gaussians to test */
    int64_t n_idx;
    const int64_t *grown; /* with idx: per tested Gaussian its grown pixel rectangle
                             (x0, x1, y0, y1); pixels outside it are not tested */
} og_render_ctx;

/* Blends a copy of src[0..n) (og_blend reorders its input). */
static void og_blend_copy(const og_frag *src, int64_t n, og_fragvec *scratch, const og_params *prm,
                          og_pixel_result *res) {
    scratch->n = 0;
    for (int64_t i = 0; i < n; ++i) og_push(scratch, &src[i]);
    memset(res, 0, sizeof(*res));
    og_blend(scratch, prm, res);
}

/* Largest channel change between two blends of the same pixel. */
static double og_move(const og_pixel_result *a, const og_pixel_result *b) {
    double m = 0;
    for (int ch = 0; ch < 3; ++ch) {
        const double e = fabs(a->C[ch] - b->C[ch]);
        if (e > m) m = e;
    }
    return m;
}

/* Re-blends with each near-decision flipped, one at a time; returns the bits
   whose flip moves the colour by more than OG_EFFECT_TOL and adds every
   flip's move to *budget. */
static int32_t og_effects(const og_fragvec *F0, const og_fragvec *Bd, const og_fragvec *Fs,
                          const og_pixel_result *res, const og_params *prm, og_fragvec *work,
                          og_fragvec *scratch, double *budget) {
    /* (Sorted blending has no core: only its cutoff flips are evaluated here.) */
    const int hybrid = !prm->sorted_blend;
    int32_t amb = 0;
    double sum = 0, mv;
    og_pixel_result alt;
    /* Cutoff: drop a kept borderline fragment, or add a rejected one. */
    for (int64_t b = 0; b < Bd->n; ++b) {
        const og_frag *x = &Bd->f[b];
        work->n = 0;
        int present = 0;
        for (int64_t i = 0; i < F0->n; ++i) {
            if (F0->f[i].gid == x->gid) { present = 1; continue; }
            og_push(work, &F0->f[i]);
        }
        if (!present) og_push(work, x);
        og_blend_copy(work->f, work->n, scratch, prm, &alt);
        sum += (mv = og_move(&alt, res));
        if (mv > OG_EFFECT_TOL) amb |= OG_AMB_CUTOFF;
    }
    /* Core admission: force the opposite side of tau_K. */
    for (int64_t i = 0; i < F0->n && hybrid; ++i) {
        if (fabs(F0->f[i].alpha - prm->tau_K) > OG_TAUK_ABS) continue;
        work->n = 0;
        for (int64_t k = 0; k < F0->n; ++k) og_push(work, &F0->f[k]);
        work->f[i].force = F0->f[i].alpha >= prm->tau_K ? -1 : 1;
        og_blend_copy(work->f, work->n, scratch, prm, &alt);
        sum += (mv = og_move(&alt, res));
        if (mv > OG_EFFECT_TOL) amb |= OG_AMB_TAUK;
    }
    /* Depth order: swap the depths of close neighbours among the sorted
       candidates Fs (core and first excluded candidate). */
    const int64_t K = prm->K;
    for (int64_t i = 0; hybrid && i + 1 < Fs->n && i < K; ++i) {
        const og_frag *a = &Fs->f[i], *b = &Fs->f[i + 1];
        if (fabs(b->z - a->z) > OG_DEPTH_REL * fabs(a->z)) continue;
        const int32_t bit = (i + 1 == K) ? OG_AMB_CORE_EDGE : OG_AMB_CORE_TIE;
        work->n = 0;
        for (int64_t k = 0; k < F0->n; ++k) {
            og_frag f = F0->f[k];
            if (f.gid == a->gid) f.z = b->z;
            else if (f.gid == b->gid) f.z = a->z;
            og_push(work, &f);
        }
        og_blend_copy(work->f, work->n, scratch, prm, &alt);
        sum += (mv = og_move(&alt, res));
        if (mv > OG_EFFECT_TOL) amb |= bit;
    }
    if (budget) *budget = sum;
    return amb;
}

/* Sorted blending (Tab. 3 variant): re-blends with each near-decision
   flipped alone, the stop at a fragment whose T (1 - alpha) lies within
   rounding of the threshold, and the order of two fragments (among the
   blended ones and the first one left out) whose mean depths are within
   OG_DEPTH_REL. Fs holds the fragments in blending order. */
static int32_t og_effects_sorted(const og_fragvec *F0, const og_fragvec *Fs, int64_t used,
                                 const og_pixel_result *res, const og_params *prm, og_fragvec *work,
                                 og_fragvec *scratch, double *budget) {
    int32_t amb = 0;
    double sum = 0, mv;
    og_pixel_result alt;
    double T = 1.0;
    const int64_t last = used < Fs->n ? used : Fs->n - 1;
    for (int64_t i = 0; i <= last; ++i) {
        const og_frag *f = &Fs->f[i];
        const double Tn = T * (1.0 - f->alpha);
        if (fabs(Tn - OG_SORTED_TMIN) <= 1e-6 * OG_SORTED_TMIN + 1e-7 * T) {
            work->n = 0;
            for (int64_t k = 0; k < F0->n; ++k) {
                og_frag g = F0->f[k];
                if (g.gid == f->gid) g.force = i < used ? -1 : 1;
                og_push(work, &g);
            }
            og_blend_copy(work->f, work->n, scratch, prm, &alt);
            sum += (mv = og_move(&alt, res));
            if (mv > OG_EFFECT_TOL) amb |= OG_AMB_TERM;
        }
        if (i > 0 && fabs(f->zmean - Fs->f[i - 1].zmean) <= OG_DEPTH_REL * fabs(f->zmean)) {
            const og_frag *a = &Fs->f[i - 1];
            work->n = 0;
            for (int64_t k = 0; k < F0->n; ++k) {
                og_frag g = F0->f[k];
                /* Swap the two mean depths; equal ones would fall back to the
                   gid order, so the swap is made strict by the gids too. */
                if (g.gid == a->gid) { g.zmean = f->zmean; g.gid = f->gid; }
                else if (g.gid == f->gid) { g.zmean = a->zmean; g.gid = a->gid; }
                og_push(work, &g);
            }
            og_blend_copy(work->f, work->n, scratch, prm, &alt);
            sum += (mv = og_move(&alt, res));
            if (mv > OG_EFFECT_TOL) amb |= OG_AMB_ORDER;
        }
        T = Tn;
    }
    if (budget) *budget = sum;
    return amb;
}

static void og_render_task(void *vctx, int64_t b, int64_t e) {
    og_render_ctx *c = (og_render_ctx *)vctx;
    og_fragvec F = {0}, F0 = {0}, Bd = {0}, work = {0}, scratch = {0};
    const int K = c->prm->K;
    for (int64_t pix = b; pix < e; ++pix) {
        int64_t li = pix % c->win.w, lj = pix / c->win.w;
        double xs = (double)(c->win.x0 + li) + 0.5;
        double ys = (double)(c->win.y0 + lj) + 0.5;
        og_pixel_result res;
        memset(&res, 0, sizeof(res));
        F.n = 0;
        Bd.n = 0;
        const int64_t n_test = c->idx ? c->n_idx : c->n;
        for (int64_t t = 0; t < n_test; ++t) {
            const int64_t g = c->idx ? c->idx[t] : t;
            if (!c->sp[g].valid) continue;
            if (c->grown) {
                const int64_t *q = c->grown + 4 * t;
                const int64_t px = c->win.x0 + li, py = c->win.y0 + lj;
                if (px < q[0] || px > q[1] || py < q[2] || py > q[3]) continue;
            }
            og_frag fr;
            int border = 0;
            int kept = og_fragment(&c->sp[g], g, xs, ys, c->prm, &fr, &res.amb, &border);
            if (kept && og_push(&F, &fr)) { c->err = 1; goto out; }
            if (border && c->diag && og_push(&Bd, &fr)) { c->err = 1; goto out; }
        }
        F0.n = 0;
        if (c->diag)
            for (int64_t i = 0; i < F.n; ++i) og_push(&F0, &F.f[i]);
        og_blend(&F, c->prm, &res);
        for (int ch = 0; ch < 3; ++ch) c->image[pix * 3 + ch] = res.C[ch];
        og_pixel_diag *d = c->diag;
        if (d) {
            int32_t near = res.amb | (Bd.n ? OG_AMB_CUTOFF : 0);
            /* Sorted candidates = the front of F after og_blend. */
            og_fragvec Fs = {F.f, 0, 0};
            int64_t nc = 0;
            while (nc < F.n && (F.f[nc].force > 0 || (F.f[nc].force == 0 && F.f[nc].alpha >= c->prm->tau_K))) ++nc;
            Fs.n = nc < K + 1 ? nc : K + 1;
            int32_t amb = near & OG_AMB_DEN;
            double budget = 0, b2 = 0;
            if (c->prm->sorted_blend) {
                /* Blending order = the front of F after og_blend; the cutoff
                   flips are evaluated like the hybrid ones. */
                og_fragvec Fo = {F.f, F.n, 0};
                if (near & (OG_AMB_TERM | OG_AMB_ORDER))
                    amb |= og_effects_sorted(&F0, &Fo, res.n_core, &res, c->prm, &work, &scratch, &b2);
                if (near & OG_AMB_CUTOFF) {
                    og_fragvec none = {NULL, 0, 0};
                    amb |= og_effects(&F0, &Bd, &none, &res, c->prm, &work, &scratch, &budget);
                }
                budget += b2;
            } else if (near & (OG_AMB_CUTOFF | OG_AMB_TAUK | OG_AMB_CORE_EDGE | OG_AMB_CORE_TIE)) {
                amb |= og_effects(&F0, &Bd, &Fs, &res, c->prm, &work, &scratch, &budget);
            }
            if (d->amb_effect) d->amb_effect[pix] = budget;
            if (d->n_frag) d->n_frag[pix] = (int32_t)res.n_frag;
            if (d->n_core) d->n_core[pix] = (int32_t)res.n_core;
            if (d->core_gid)
                for (int k = 0; k < K; ++k)
                    d->core_gid[pix * K + k] = k < res.n_core ? (int32_t)F.f[k].gid : -1;
            if (d->T_core) d->T_core[pix] = res.T_core;
            if (d->T_tail) d->T_tail[pix] = res.T_tail;
            if (d->A_tail) d->A_tail[pix] = res.A_tail;
            if (d->c_tail)
                for (int ch = 0; ch < 3; ++ch) d->c_tail[pix * 3 + ch] = res.c_tail[ch];
            if (d->ambiguous) d->ambiguous[pix] = amb;
            if (d->near_decision) d->near_decision[pix] = near;
            if (d->frag_hash) d->frag_hash[pix] = res.hash;
        }
    }
out:
    free(F.f);
    free(F0.f);
    free(Bd.f);
    free(work.f);
    free(scratch.f);
}

static int og_check(const og_camera *cam, const og_params *prm, const og_window *win) {
    if (!cam || !prm || !win) return 1;
    if (prm->K < 0 || win->w < 0 || win->h < 0) return 1;
    if (cam->width <= 0 || cam->height <= 0) return 1;
    return 0;
}

/* Renders the pixel window (image: w*h*3, row-major, HWC) given the
   per-Gaussian setup from og_preprocess. */
int og_render_splats(const og_splat *sp, int64_t n, const og_camera *cam, const og_params *prm,
                     const og_window *win, double *image, og_pixel_diag *diag) {
    if (og_check(cam, prm, win) || !image || (n > 0 && !sp)) return 1;
    og_render_ctx c = {sp, n, cam, prm, *win, image, diag, 0, NULL, 0, NULL};
    og_parallel_for((int64_t)win->w * win->h, 4, og_render_task, &c);
    return c.err ? 2 : 0;
}

int og_render(const og_gaussians *g, const og_camera *cam, const og_params *prm,
              const og_window *win, double *image, og_pixel_diag *diag) {
    if (!g || og_check(cam, prm, win)) return 1;
    og_splat *sp = (og_splat *)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(og_splat));
    if (!sp) return 2;
    int rc = og_preprocess(g, cam, prm, sp);
    if (!rc) rc = og_render_splats(sp, g->n, cam, prm, win, image, diag);
    free(sp);
    return rc;
}

/* og_render restricted to the Gaussians whose covered pixel rectangle, grown
   by `margin` pixels on every side, meets the window. The tight box of
   Sec. 3.2 contains every pixel centre with rho^2 <= rho_c, so the result
   equals og_render's whenever the margin also covers the band of rejected
   pairs within OG_CUTOFF_REL of the cutoff (a relative width of 1e-5 in
   rho, i.e. less than a pixel for splats under 10^5 pixels across). Gids
   keep their numbering in the full array. This only skips pairs that the
   brute force would reject; the test suite checks equality with og_render. */
int og_render_boxed(const og_gaussians *g, const og_camera *cam, const og_params *prm,
                    const og_window *win, int32_t margin, double *image, og_pixel_diag *diag,
                    int64_t *n_tested) {
    if (!g || og_check(cam, prm, win) || !image || margin < 0) return 1;
    og_splat *sp = (og_splat *)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(og_splat));
    int64_t *idx = (int64_t *)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int64_t));
    int64_t *grown = (int64_t *)malloc((size_t)(g->n > 0 ? g->n : 1) * 4 * sizeof(int64_t));
    if (!sp || !idx || !grown) { free(sp); free(idx); free(grown); return 2; }
    int rc = og_preprocess(g, cam, prm, sp);
    int64_t m = 0;
    if (!rc) {
        const int64_t wx0 = win->x0, wx1 = (int64_t)win->x0 + win->w - 1;
        const int64_t wy0 = win->y0, wy1 = (int64_t)win->y0 + win->h - 1;
        for (int64_t i = 0; i < g->n; ++i) {
            const og_splat *q = &sp[i];
            if (!q->valid) continue;
            /* The rectangle is clamped to the image; a splat whose box lies
               off-image has an empty one but may still border the window
               across the image edge, so the clamped sides are widened too. */
            int64_t x0 = q->rect[0], x1 = q->rect[1], y0 = q->rect[2], y1 = q->rect[3];
            const double bx0 = floor(q->p[0] - q->h[0] - 0.5), bx1 = ceil(q->p[0] + q->h[0] - 0.5);
            const double by0 = floor(q->p[1] - q->h[1] - 0.5), by1 = ceil(q->p[1] + q->h[1] - 0.5);
            if (x0 > x1) { x0 = bx0 < -1e9 ? -1000000000 : (int64_t)bx0; x1 = bx1 > 1e9 ? 1000000000 : (int64_t)bx1; }
            if (y0 > y1) { y0 = by0 < -1e9 ? -1000000000 : (int64_t)by0; y1 = by1 > 1e9 ? 1000000000 : (int64_t)by1; }
            if (x1 + margin < wx0 || x0 - margin > wx1 || y1 + margin < wy0 || y0 - margin > wy1) continue;
            grown[4 * m + 0] = x0 - margin; grown[4 * m + 1] = x1 + margin;
            grown[4 * m + 2] = y0 - margin; grown[4 * m + 3] = y1 + margin;
            idx[m++] = i;
        }
        og_render_ctx c = {sp, g->n, cam, prm, *win, image, diag, 0, idx, m, grown};
        og_parallel_for((int64_t)win->w * win->h, 4, og_render_task, &c);
        rc = c.err ? 2 : 0;
    }
    if (n_tested) *n_tested = m;
    free(sp);
    free(idx);
    free(grown);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Backward (Sec. 3.3: the tail's partial derivative is shared per pixel)   */
/* ------------------------------------------------------------------------ */
/*
 * For a pixel with dL/dC = g, core fragments i = 1..n (depth order) and
 * B' = (1 - T_tail) c_tail + T_tail bg, let G_n = B' and
 * G_{i-1} = alpha_i c_i + (1 - alpha_i) G_i (the colour seen behind i-1).
 * Then dC/dc_i = alpha_i T_i and dC/dalpha_i = T_i (c_i - G_i).
 * Every tail fragment j shares the per-pixel constants T_core, T_tail, A and
 * c_tail: dC/dc_j = T_core (1 - T_tail) alpha_j / A and
 * dC/dalpha_j = T_core [(1 - T_tail)(c_j - c_tail)/A + T_tail (c_tail - bg)/(1 - alpha_j)].
 * Depth ranks, the cutoff, tau_K and culling are piecewise constant: no
 * gradient flows through them.
 */

typedef struct {
    int32_t n_core;
    double T_core, T_tail, A_tail, c_tail[3];
    double g[3];          /* dL/dC */
} og_pix_state;

typedef struct {
    int64_t gid;
    double dalpha_coef;   /* dL/dalpha_i = g . T_i (c_i - G_i) */
    double dc_coef;       /* dL/dc_i = g * alpha_i T_i */
} og_core_entry;

typedef struct {
    const og_splat *sp;
    int64_t n;
    const og_camera *cam;
    const og_params *prm;
    og_window win;
    const double *dl_dimg;
    og_pix_state *pix;
    og_core_entry *core;  /* w*h*K */
    double *rec_grad;     /* n x 16: dr1[4], dr2[4], dr4[4], do, dc[3] */
    int err;
    double *visibility;   /* n or NULL: largest blending weight over the window's pixels */
    int64_t kcap;         /* per-pixel entries of core: K, or n for sorted blending */
} og_bwd_ctx;

static void og_bwd_pixel_task(void *vctx, int64_t b, int64_t e) {
    og_bwd_ctx *c = (og_bwd_ctx *)vctx;
    og_fragvec F = {0};
    const int64_t K = c->kcap;
    double *Ti = (double *)malloc((size_t)(K > 0 ? K : 1) * sizeof(double));
    if (!Ti) { c->err = 1; return; }
    for (int64_t pix = b; pix < e; ++pix) {
        int64_t li = pix % c->win.w, lj = pix / c->win.w;
        double xs = (double)(c->win.x0 + li) + 0.5;
        double ys = (double)(c->win.y0 + lj) + 0.5;
        og_pixel_result res;
        memset(&res, 0, sizeof(res));
        F.n = 0;
        for (int64_t g = 0; g < c->n; ++g) {
            if (!c->sp[g].valid) continue;
            og_frag fr;
            if (og_fragment(&c->sp[g], g, xs, ys, c->prm, &fr, NULL, NULL))
                if (og_push(&F, &fr)) { c->err = 1; free(F.f); return; }
        }
        og_blend(&F, c->prm, &res);
        og_pix_state *st = &c->pix[pix];
        st->n_core = (int32_t)res.n_core;
        st->T_core = res.T_core;
        st->T_tail = res.T_tail;
        st->A_tail = res.A_tail;
        for (int ch = 0; ch < 3; ++ch) {
            st->c_tail[ch] = res.c_tail[ch];
            st->g[ch] = c->dl_dimg[pix * 3 + ch];
        }
        /* G_n = B', then walk the core back to front. */
        double G[3];
        for (int ch = 0; ch < 3; ++ch)
            G[ch] = (1.0 - res.T_tail) * res.c_tail[ch] + res.T_tail * c->prm->bg[ch];
        double T = 1.0;
        for (int64_t i = 0; i < res.n_core; ++i) { Ti[i] = T; T *= 1.0 - F.f[i].alpha; }
        for (int64_t i = res.n_core - 1; i >= 0; --i) {
            const og_frag *f = &F.f[i];
            double da = 0;
            for (int ch = 0; ch < 3; ++ch) da += st->g[ch] * Ti[i] * (f->c[ch] - G[ch]);
            og_core_entry *ce = &c->core[pix * K + i];
            ce->gid = f->gid;
            ce->dalpha_coef = da;
            ce->dc_coef = f->alpha * Ti[i];
            for (int ch = 0; ch < 3; ++ch) G[ch] = f->alpha * f->c[ch] + (1.0 - f->alpha) * G[ch];
        }
        for (int64_t i = res.n_core; i < K; ++i) c->core[pix * K + i].gid = -1;
    }
    free(F.f);
    free(Ti);
}

static void og_bwd_gauss_task(void *vctx, int64_t b, int64_t e) {
    og_bwd_ctx *c = (og_bwd_ctx *)vctx;
    const int64_t K = c->kcap;
    const int64_t npix = (int64_t)c->win.w * c->win.h;
    for (int64_t g = b; g < e; ++g) {
        const og_splat *sp = &c->sp[g];
        double *rg = c->rec_grad + g * 16;
        memset(rg, 0, 16 * sizeof(double));
        if (c->visibility) c->visibility[g] = 0.0;
        if (!sp->valid) continue;
        for (int64_t pix = 0; pix < npix; ++pix) {
            int64_t li = pix % c->win.w, lj = pix / c->win.w;
            double xs = (double)(c->win.x0 + li) + 0.5;
            double ys = (double)(c->win.y0 + lj) + 0.5;
            og_eval ev;
            if (!og_evaluate(sp, xs, ys, &ev)) continue;
            if (!(ev.rho2 <= sp->rho_c)) continue;
            const og_pix_state *st = &c->pix[pix];
            const double a_raw = sp->o * exp(-0.5 * ev.rho2);
            const double alpha = a_raw < c->prm->alpha_max ? a_raw : c->prm->alpha_max;
            /* dL/dalpha and dL/dc for this fragment. */
            double dL_dalpha = 0, dL_dc[3] = {0, 0, 0};
            int in_core = 0;
            for (int k = 0; k < st->n_core && k < K; ++k) {
                const og_core_entry *ce = &c->core[pix * K + k];
                if (ce->gid == g) {
                    in_core = 1;
                    dL_dalpha = ce->dalpha_coef;
                    for (int ch = 0; ch < 3; ++ch) dL_dc[ch] = st->g[ch] * ce->dc_coef;
                    break;
                }
            }
            /* Blending weight of the fragment in the pixel colour: alpha_i T_i in
               the core, T_core (1 - T_tail) alpha_j / A in the tail. */
            if (c->visibility) {
                double w = 0.0;
                if (in_core) {
                    for (int k = 0; k < st->n_core && k < K; ++k)
                        if (c->core[pix * K + k].gid == g) w = c->core[pix * K + k].dc_coef;
                } else if (!c->prm->no_tail && !c->prm->sorted_blend && st->A_tail > 0) {
                    w = st->T_core * (1.0 - st->T_tail) * alpha / st->A_tail;
                }
                if (w > c->visibility[g]) c->visibility[g] = w;
            }
            /* An omitted tail, or fragments behind the early termination, have no gradient. */
            if (!in_core && (c->prm->no_tail || c->prm->sorted_blend)) continue;
            if (!in_core) {
                const double Tc = st->T_core, Tt = st->T_tail, A = st->A_tail;
                for (int ch = 0; ch < 3; ++ch) {
                    double dCda = Tc * ((1.0 - Tt) * (sp->rgb[ch] - st->c_tail[ch]) / A +
                                        Tt * (st->c_tail[ch] - c->prm->bg[ch]) / (1.0 - alpha));
                    dL_dalpha += st->g[ch] * dCda;
                    dL_dc[ch] = st->g[ch] * Tc * (1.0 - Tt) * alpha / A;
                }
            }
            for (int ch = 0; ch < 3; ++ch) rg[13 + ch] += dL_dc[ch];
            /* alpha = min(o e^{-rho^2/2}, alpha_max). */
            if (a_raw >= c->prm->alpha_max) continue;
            const double e_ = exp(-0.5 * ev.rho2);
            rg[12] += dL_dalpha * e_;                        /* d/do */
            const double dL_drho2 = dL_dalpha * (-0.5 * a_raw);
            /* rho^2 = num/den, num = ||m||^2, den = ||d||^2. */
            double dm[3], dd[3];
            for (int k = 0; k < 3; ++k) {
                dm[k] = dL_drho2 * 2.0 * ev.m[k] / ev.den;
                dd[k] = -dL_drho2 * 2.0 * ev.rho2 * ev.d[k] / ev.den;
            }
            /* m = (p^{01}, p^{02}, p^{03}) = a^0 b_xyz - b^0 a_xyz;
               d = (p^{23}, p^{31}, p^{12}) = a_xyz x b_xyz. */
            double da[4] = {0, 0, 0, 0}, db[4] = {0, 0, 0, 0};
            const double *A4 = ev.a, *B4 = ev.b;
            for (int k = 0; k < 3; ++k) {
                da[3] += dm[k] * B4[k];
                db[k] += A4[3] * dm[k];
                db[3] -= dm[k] * A4[k];
                da[k] -= B4[3] * dm[k];
            }
            /* d(a x b)/da . dd = b x dd ; d(a x b)/db . dd = dd x a. */
            da[0] += B4[1] * dd[2] - B4[2] * dd[1];
            da[1] += B4[2] * dd[0] - B4[0] * dd[2];
            da[2] += B4[0] * dd[1] - B4[1] * dd[0];
            db[0] += dd[1] * A4[2] - dd[2] * A4[1];
            db[1] += dd[2] * A4[0] - dd[0] * A4[2];
            db[2] += dd[0] * A4[1] - dd[1] * A4[0];
            /* a = T'_1 - xs T'_4, b = T'_2 - ys T'_4. */
            for (int k = 0; k < 4; ++k) {
                rg[0 + k] += da[k];
                rg[4 + k] += db[k];
                rg[8 + k] += -xs * da[k] - ys * db[k];
            }
        }
    }
}

typedef struct {
    const og_gaussians *gs;
    const og_splat *sp;
    const og_camera *cam;
    const double *rec_grad;
    double *d_means, *d_log_scales, *d_quats, *d_logits, *d_sh;
    double *densify_grad, *densify_count; /* n or NULL */
} og_chain_ctx;

/* Chain rule from (dT'_1, dT'_2, dT'_4, do, dc) to the parameters. */
static void og_chain_task(void *vctx, int64_t b, int64_t e) {
    og_chain_ctx *c = (og_chain_ctx *)vctx;
    const og_camera *cam = c->cam;
    const int nc = (c->gs->sh_degree + 1) * (c->gs->sh_degree + 1);
    for (int64_t i = b; i < e; ++i) {
        const og_splat *sp = &c->sp[i];
        const double *rg = c->rec_grad + i * 16;
        double *dmu = c->d_means + 3 * i, *dls = c->d_log_scales + 3 * i, *dq = c->d_quats + 4 * i;
        double *dsh = c->d_sh + i * nc * 3;
        memset(dmu, 0, 3 * sizeof(double));
        memset(dls, 0, 3 * sizeof(double));
        memset(dq, 0, 4 * sizeof(double));
        memset(dsh, 0, (size_t)nc * 3 * sizeof(double));
        c->d_logits[i] = 0;
        if (!sp->valid) continue;
        /* Rows of M T: T'_1 = fx (MT)_1 + cx (MT)_3, T'_2 = fy (MT)_2 + cy (MT)_3, T'_4 = (MT)_3. */
        double dMT[3][4];
        for (int k = 0; k < 4; ++k) {
            dMT[0][k] = cam->fx * rg[0 + k];
            dMT[1][k] = cam->fy * rg[4 + k];
            dMT[2][k] = cam->cx * rg[0 + k] + cam->cy * rg[4 + k] + rg[8 + k];
        }
        /* M T = M T; rows 1..3 of M T depend on rows 1..3 of T through the
           upper-left 3x3 block of M (row 4 of T is constant). */
        const double *M = cam->world_to_cam;
        double dT[3][4];
        for (int k = 0; k < 3; ++k)
            for (int cc = 0; cc < 4; ++cc) {
                double acc = 0;
                for (int r = 0; r < 3; ++r) acc += M[r * 4 + k] * dMT[r][cc];
                dT[k][cc] = acc;
            }
        /* T columns: s_j t_j (j < 3) and mu. */
        for (int k = 0; k < 3; ++k) dmu[k] += dT[k][3];
        double dR[3][3];
        for (int j = 0; j < 3; ++j) {
            double ds = 0;
            for (int k = 0; k < 3; ++k) {
                ds += sp->R[k][j] * dT[k][j];
                dR[k][j] = sp->s[j] * dT[k][j];
            }
            /* s = exp(log s); with the 3D filter s' = sqrt(s^2 + v) and
               o' = o prod_k s_k / s'_k, so d s'_j / d log s_j = s_j^2 / s'_j
               and d o' / d log s_j = o' v / s'_j^2 (rg[12] = dL/do'). */
            dls[j] = ds * sp->s_raw[j] * sp->s_raw[j] / sp->s[j] +
                     rg[12] * sp->o * sp->filter_var / (sp->s[j] * sp->s[j]);
        }
        /* R(q) of the unit quaternion q = (w, x, y, z). */
        const double w = sp->q[0], x = sp->q[1], y = sp->q[2], z = sp->q[3];
        double dqn[4];
        dqn[0] = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
        dqn[1] = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2] +
                      z * dR[2][0] + w * dR[2][1] - 2 * x * dR[2][2]);
        dqn[2] = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                      w * dR[2][0] + z * dR[2][1] - 2 * y * dR[2][2]);
        dqn[3] = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1] +
                      y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        /* q_hat = q / |q|: dq = (dq_hat - q_hat (q_hat . dq_hat)) / |q|. */
        const double *qr = c->gs->quats + 4 * i;
        double qn = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
        double dot = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
        for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - sp->q[k] * dot) / qn;
        /* o' = o prod_k s_k / s'_k with o = sigmoid(logit): d o'/d logit = o' (1 - o). */
        c->d_logits[i] = rg[12] * sp->o * (1.0 - sp->o_raw);
        /* colour = max(0, 0.5 + sum_k Y_k(dir) k_k); dir = (mu - centre)/|mu - centre|. */
        double Y[16], dY[16][3];
        og_sh_basis(sp->dir, c->gs->sh_degree, Y, dY);
        const double *shc = c->gs->sh + i * nc * 3;
        double ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(sp->rgb_raw[ch] > 0)) continue;
            double dc = rg[13 + ch];
            for (int k = 0; k < nc; ++k) {
                dsh[k * 3 + ch] += dc * Y[k];
                for (int j = 0; j < 3; ++j) ddir[j] += dc * shc[k * 3 + ch] * dY[k][j];
            }
        }
        if (sp->dist > 0) {
            double pd = ddir[0] * sp->dir[0] + ddir[1] * sp->dir[1] + ddir[2] * sp->dir[2];
            for (int j = 0; j < 3; ++j) dmu[j] += (ddir[j] - sp->dir[j] * pd) / sp->dist;
        }
        /* Densification statistic (Sec. 4.2, after Moenne-Loccoz et al.): the
           norm of the mean's gradient times half the distance to the camera,
           for a Gaussian that covers pixels of this view. */
        if (sp->rect[0] <= sp->rect[1] && sp->rect[2] <= sp->rect[3]) {
            if (c->densify_grad)
                c->densify_grad[i] = 0.5 * sp->dist * sqrt(dmu[0] * dmu[0] + dmu[1] * dmu[1] + dmu[2] * dmu[2]);
            if (c->densify_count) c->densify_count[i] = 1.0;
        }
    }
}

/* Analytic gradient of L = sum(dl_dimg * image) over the pixel window with
   respect to every parameter (each output array shaped like its input). */
int og_render_backward(const og_gaussians *g, const og_camera *cam, const og_params *prm,
                       const og_window *win, const double *dl_dimg,
                       double *d_means, double *d_log_scales, double *d_quats,
                       double *d_logits, double *d_sh,
                       double *visibility, double *densify_grad, double *densify_count) {
    if (!g || og_check(cam, prm, win) || !dl_dimg) return 1;
    if (!d_means || !d_log_scales || !d_quats || !d_logits || !d_sh) return 1;
    if (!prm->sorted_blend && prm->K > 64) return 1;
    const int64_t kcap = prm->sorted_blend ? (g->n > 0 ? g->n : 1) : (prm->K > 0 ? prm->K : 1);
    if ((double)win->w * win->h * kcap > 2e8) return 1;
    const int64_t n = g->n;
    const int64_t npix = (int64_t)win->w * win->h;
    og_splat *sp = (og_splat *)malloc((size_t)(n > 0 ? n : 1) * sizeof(og_splat));
    og_pix_state *pix = (og_pix_state *)calloc((size_t)(npix > 0 ? npix : 1), sizeof(og_pix_state));
    og_core_entry *core = (og_core_entry *)calloc((size_t)(npix * kcap + 1),
                                                  sizeof(og_core_entry));
    double *rec = (double *)calloc((size_t)(n > 0 ? n : 1) * 16, sizeof(double));
    int rc = 0;
    if (!sp || !pix || !core || !rec) rc = 2;
    if (!rc) rc = og_preprocess(g, cam, prm, sp);
    if (!rc) {
        og_bwd_ctx c = {sp, n, cam, prm, *win, dl_dimg, pix, core, rec, 0, visibility, kcap};
        og_parallel_for(npix, 4, og_bwd_pixel_task, &c);
        if (c.err) rc = 2;
        if (!rc) og_parallel_for(n, 8, og_bwd_gauss_task, &c);
    }
    if (!rc) {
        if (densify_grad) memset(densify_grad, 0, (size_t)n * sizeof(double));
        if (densify_count) memset(densify_count, 0, (size_t)n * sizeof(double));
        og_chain_ctx cc = {g, sp, cam, rec, d_means, d_log_scales, d_quats, d_logits, d_sh,
                           densify_grad, densify_count};
        og_parallel_for(n, 1024, og_chain_task, &cc);
    }
    free(sp);
    free(pix);
    free(core);
    free(rec);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Tile binning by bounding box (Sec. 4.3: per-tile instance lists keyed by */
/* the tile id only, no global depth sort)                                  */
/* ------------------------------------------------------------------------ */

/* For pixel rectangles rect[n][4] = (x_min, x_max, y_min, y_max), inclusive,
   counts the instances per tile (tile_count: tiles_x*tiles_y) and, when lists
   is non-NULL, writes each tile's gids in ascending order at offsets given by
   the exclusive prefix sum of tile_count. Returns the total instance count. */
int64_t og_bin(const int32_t *rect, int64_t n, int32_t width, int32_t height, int32_t tile_w,
               int32_t tile_h, int64_t *tile_count, int32_t *lists) {
    const int64_t tx = (width + tile_w - 1) / tile_w, ty = (height + tile_h - 1) / tile_h;
    for (int64_t t = 0; t < tx * ty; ++t) tile_count[t] = 0;
    int64_t total = 0;
    for (int64_t g = 0; g < n; ++g) {
        const int32_t *r = rect + 4 * g;
        if (r[1] < r[0] || r[3] < r[2]) continue;
        for (int32_t j = r[2] / tile_h; j <= r[3] / tile_h; ++j)
            for (int32_t i = r[0] / tile_w; i <= r[1] / tile_w; ++i) {
                tile_count[(int64_t)j * tx + i]++;
                ++total;
            }
    }
    if (lists) {
        int64_t *cursor = (int64_t *)malloc((size_t)(tx * ty > 0 ? tx * ty : 1) * sizeof(int64_t));
        if (!cursor) return -1;
        int64_t acc = 0;
        for (int64_t t = 0; t < tx * ty; ++t) { cursor[t] = acc; acc += tile_count[t]; }
        for (int64_t g = 0; g < n; ++g) {
            const int32_t *r = rect + 4 * g;
            if (r[1] < r[0] || r[3] < r[2]) continue;
            for (int32_t j = r[2] / tile_h; j <= r[3] / tile_h; ++j)
                for (int32_t i = r[0] / tile_w; i <= r[1] / tile_w; ++i)
                    lists[cursor[(int64_t)j * tx + i]++] = (int32_t)g;
        }
        free(cursor);
    }
    return total;
}
