/*
 * gs_oracle.c -- FP64 CPU oracle of the differentiable tile-based Gaussian
 * rasterizer used by every tracking and mapping iteration of RTGS
 * (arXiv 2510.06644, "RTGS: Real-Time 3D Gaussian Splatting SLAM via
 * Multi-Level Redundancy Reduction", MICRO '25).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Everything is double precision except where the method turns a floating
 * value into an integer decision that the GPU path takes in FP32: the sort
 * key uses the float32 bits of the depth, and the pruning score is formed in
 * float32 (see or_prune_select).
 *
 * Sections of the paper followed:
 *   Sec. 2.1, Eq. 1   3D Gaussian scene representation (mean, covariance,
 *                     opacity, colour).
 *   Sec. 2.1 Step 1   projection to 2D Gaussians and tile intersection
 *                     (16x16 tiles, footnote of Step 1-2).
 *   Sec. 2.1 Step 2   depth sort of each tile's fragments.
 *   Sec. 2.1 Eq. 2    alpha of a fragment.
 *   Sec. 2.1 Eq. 3    front-to-back blending with transmittance and early
 *                     termination.
 *   Sec. 2.2 Step 4   rendering backpropagation; Eq. 4 and Eq. 5 describe the
 *                     alpha gradient and the reverse transmittance recovery.
 *                     The oracle differentiates Eq. 3 directly instead of
 *                     using the printed Eq. 4, which drops T and 1/(1-alpha).
 *   Sec. 2.2 Step 5   preprocessing backpropagation to 3D Gaussian gradients
 *                     and the per-Gaussian camera pose gradient summed into
 *                     dL/dP.
 *   Sec. 4.1 Eq. 6    tracking loss (photometric + geometric residual).
 *   Sec. 4.1 Eq. 7    Gaussian importance score and the mask-prune interval K.
 *   Sec. 4.2          keyframe-driven dynamic downsampling schedule.
 *   Sec. 6.1          hyper-parameters lambda = 0.8, K0 = 5, m = 2.
 *
 * Readings where the paper is silent (pixel centre, near plane, low-pass
 * dilation, Jacobian clamp, 3-sigma radius, thresholds, loss normalisation,
 * pose parameterisation) are listed with the projection and render functions
 * below; each one is a plain statement of the formula, not a transcription.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Camera and configuration                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    double R[9];      /* world -> camera rotation, row-major */
    double t[3];      /* world -> camera translation */
    double fx, fy, cx, cy;
    int32_t W, H;     /* full-resolution image */
    int32_t sx, sy;   /* sampling strides (Sec. 4.2); (1,1) = full resolution */
} or_cam;

typedef struct {
    double near_z;    /* cull if camera-frame z < near_z */
    double dilation;  /* low-pass term added to the 2D covariance diagonal */
    double alpha_min; /* fragments with alpha below this are skipped */
    double alpha_max; /* alpha is clamped to this value */
    double t_eps;     /* early-termination threshold on transmittance */
    double bg[3];     /* background colour */
} or_cfg;

#define TILE 16

static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}
static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }
static int64_t clamp_i64(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Tile side in sampled pixels for stride s: 16 / p2(s), at least 4, with
 * p2(s) the smallest power of two >= s, so that a tile keeps the 16-pixel
 * full-resolution footprint of the paper's tile (Sec. 2.1 Step 1-2 footnote)
 * when the frame is point-sampled at stride s (Sec. 4.2). */
static int64_t tile_dim(int64_t s) {
    int64_t p = 1;
    while (p < s && p < TILE) p *= 2;
    int64_t t = TILE / p;
    return t < 4 ? 4 : t;
}

/* Sampled image size and tile grid for the camera's strides (Sec. 4.2). */
static void grid_dims(const or_cam* c, int64_t* Ws, int64_t* Hs, int64_t* TX, int64_t* TY) {
    *Ws = ceil_div(c->W, c->sx);
    *Hs = ceil_div(c->H, c->sy);
    *TX = ceil_div(*Ws, tile_dim(c->sx));
    *TY = ceil_div(*Hs, tile_dim(c->sy));
}

/* Half extents of the pixel box where alpha = op exp(-d^T Q d / 2) can reach
 * alpha_min (Q = conic; fragments below alpha_min are skipped, Sec. 2.1):
 * |d_x| <= sqrt(2 ln(op / alpha_min) (Q^-1)_xx), (Q^-1)_xx = c / det.  ln is
 * bounded above by 64 (x^(1/64) - 1) (e^t >= 1 + t), plus 1e-3, and the
 * extent is widened by 1.002 and 2e-3 px.  This bound decides integers (which
 * tiles hold the Gaussian), so it is evaluated in float32 with correctly
 * rounded operations only (products, quotients, six square roots), no
 * contraction: the same numbers on every IEEE machine.  Returns 0 when no
 * pixel can reach alpha_min (op < alpha_min); the extents are +inf when the
 * conic is degenerate. */
static int alpha_extent_f(float ca, float cb, float cc, float op, float amin, float* ex, float* ey) {
    if (!(op >= amin)) return 0;
    *ex = INFINITY;
    *ey = INFINITY;
    float det = ca * cc - cb * cb;
    if (!(det > 0.f)) return 1;
    float q = op / amin;
    for (int i = 0; i < 6; ++i) q = sqrtf(q);
    float L = 64.f * (q - 1.f);
    float t2 = 2.f * ((L > 0.f ? L : 0.f) + 1e-3f);
    *ex = sqrtf(t2 * cc / det) * 1.002f + 2e-3f;
    *ey = sqrtf(t2 * ca / det) * 1.002f + 2e-3f;
    return 1;
}

/* Tile rectangle of a 2D Gaussian (Sec. 2.1, Step 1-2).  The Gaussian covers
 * the integer pixel box [floor(u)-r, floor(u)+r] x [floor(v)-r, floor(v)+r]
 * of the full-resolution image (returned in `box`); this box contains every
 * pixel whose centre (p+0.5) lies within r of the mean on each axis.  Its
 * tiles are those holding a sampled pixel of the box that can also reach
 * alpha_min: |p + 0.5 - u| <= ex (alpha_extent_f, from the float32 values of
 * u, v, the conic and the opacity).  With strides (sx, sy) the sampled pixel
 * i sits at full-resolution column sx*i, so the covered sampled columns are
 * ceil(b0/sx) .. floor(b1/sx) for the shrunk box [b0, b1], clipped to the
 * sampled image and divided by the tile side (16 at full resolution, see
 * tile_dim).  Returns the rect [x0,x1) x [y0,y1) in tile units (empty when no
 * such pixel lies in the image). */
static void tile_rect(const or_cam* c, double u, double v, int64_t r, const double* conic, double opacity,
                      double alpha_min, int64_t rect[4], int64_t box[4]) {
    int64_t Ws, Hs, TX, TY;
    grid_dims(c, &Ws, &Hs, &TX, &TY);
    double uc = u < -1e9 ? -1e9 : (u > 1e9 ? 1e9 : u);
    double vc = v < -1e9 ? -1e9 : (v > 1e9 ? 1e9 : v);
    int64_t xi = (int64_t)floor(uc), yi = (int64_t)floor(vc);
    box[0] = xi - r; box[1] = xi + r; box[2] = yi - r; box[3] = yi + r;
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    float ex, ey;
    if (!alpha_extent_f((float)conic[0], (float)conic[1], (float)conic[2], (float)opacity, (float)alpha_min,
                        &ex, &ey))
        return;
    int64_t b0 = box[0], b1 = box[1], b2 = box[2], b3 = box[3];
    const float uf = (float)u, vf = (float)v;
    if (ex < 1e8f && fabsf(uf) < 1e8f) {
        int64_t lo = (int64_t)ceilf((uf - ex) - 0.5f), hi = (int64_t)floorf((uf + ex) - 0.5f);
        if (lo > b0) b0 = lo;
        if (hi < b1) b1 = hi;
    }
    if (ey < 1e8f && fabsf(vf) < 1e8f) {
        int64_t lo = (int64_t)ceilf((vf - ey) - 0.5f), hi = (int64_t)floorf((vf + ey) - 0.5f);
        if (lo > b2) b2 = lo;
        if (hi < b3) b3 = hi;
    }
    if (b1 < b0 || b3 < b2) return;
    int64_t i0 = ceil_div(b0, c->sx), i1 = floor_div(b1, c->sx);
    int64_t j0 = ceil_div(b2, c->sy), j1 = floor_div(b3, c->sy);
    /* only sampled pixels inside the image count */
    i0 = clamp_i64(i0, 0, Ws); i1 = clamp_i64(i1, -1, Ws - 1);
    j0 = clamp_i64(j0, 0, Hs); j1 = clamp_i64(j1, -1, Hs - 1);
    if (i0 > i1 || j0 > j1) return;
    rect[0] = i0 / tile_dim(c->sx);
    rect[1] = i1 / tile_dim(c->sx) + 1;
    rect[2] = j0 / tile_dim(c->sy);
    rect[3] = j1 / tile_dim(c->sy) + 1;
    (void)TX; (void)TY;
}

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra (row-major)                                    */
/* ------------------------------------------------------------------------ */

static void mat3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
static void mat3_T(const double* A, double* B) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * j + i] = A[3 * i + j];
}

/* Rotation of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double Rq[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z);     Rq[2] = 2 * (x * z + w * y);
    Rq[3] = 2 * (x * y + w * z);     Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
    Rq[6] = 2 * (x * z - w * y);     Rq[7] = 2 * (y * z + w * x);     Rq[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 2.1, Step 1-1)                                           */
/* ------------------------------------------------------------------------ */

/* Intermediate quantities of the projection of one Gaussian, shared by the
 * forward projection and its backward pass. */
typedef struct {
    int visible;          /* passed the near-plane and determinant tests */
    double p[3];          /* camera-frame mean */
    double qn[4];         /* normalised quaternion */
    double qlen;          /* |q| */
    double Rq[9];         /* rotation of qn */
    double scale[3];      /* exp(log_scale) */
    double M[9];          /* Rq * diag(scale) */
    double Sigma[9];      /* world-frame 3D covariance  M M^T (Eq. 1) */
    double Sc[9];         /* camera-frame covariance R Sigma R^T */
    double tx, ty;        /* clamped x, y used by the Jacobian */
    int clamp_x, clamp_y; /* which of x/z, y/z hit the clamp */
    double limx, limy;    /* signed clamp values when clamped */
    double J[6];          /* 2x3 Jacobian of the perspective map */
    double a, b, c;       /* 2D covariance J Sc J^T plus dilation */
    double det;
    double conic[3];      /* inverse 2D covariance (A, B, C) */
    double u, v;          /* 2D mean in pixels */
    double r3;            /* 3 * sqrt(lambda_max), before ceil */
    int64_t radius;
    double opacity;
} or_proj1;

/* Projection of Gaussian k.  Readings (the paper only says that Step 1-1
 * projects each Gaussian with the camera pose):
 *   - mean: p = R mu + t; u = fx x/z + cx, v = fy y/z + cy;
 *   - culled when z < near_z;
 *   - 3D covariance Sigma = Rq S S^T Rq^T, S = diag(exp(log_scale)) (Eq. 1);
 *   - EWA local affine approximation: Sigma2 = J (R Sigma R^T) J^T with
 *     J = [[fx/z, 0, -fx tx/z^2], [0, fy/z, -fy ty/z^2]] where tx = z *
 *     clamp(x/z, +-1.3 (W/2)/fx) and likewise ty;
 *   - low-pass dilation: Sigma2 += dilation * I;
 *   - culled when det(Sigma2) <= 0;
 *   - conic = Sigma2^{-1};
 *   - radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1,
 *     mid^2 - det)), mid = (a + c)/2;
 *   - opacity = sigmoid(logit). */
static void project_one(const double* mu, const double* ls, const double* q, double ologit,
                        const or_cam* cam, const or_cfg* cfg, or_proj1* o) {
    memset(o, 0, sizeof(*o));
    const double* R = cam->R;
    for (int i = 0; i < 3; ++i)
        o->p[i] = R[3 * i] * mu[0] + R[3 * i + 1] * mu[1] + R[3 * i + 2] * mu[2] + cam->t[i];
    double x = o->p[0], y = o->p[1], z = o->p[2];
    if (!(z >= cfg->near_z)) return;

    o->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) o->qn[i] = q[i] / o->qlen;
    quat_to_rot(o->qn, o->Rq);
    for (int i = 0; i < 3; ++i) o->scale[i] = exp(ls[i]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) o->M[3 * i + j] = o->Rq[3 * i + j] * o->scale[j];
    double MT[9];
    mat3_T(o->M, MT);
    mat3_mul(o->M, MT, o->Sigma);
    double RT[9], tmp[9];
    mat3_T(R, RT);
    mat3_mul(R, o->Sigma, tmp);
    mat3_mul(tmp, RT, o->Sc);

    double limx = 1.3 * (0.5 * cam->W) / cam->fx;
    double limy = 1.3 * (0.5 * cam->H) / cam->fy;
    double xz = x / z, yz = y / z;
    o->clamp_x = 0; o->clamp_y = 0;
    if (xz > limx) { xz = limx; o->clamp_x = 1; o->limx = limx; }
    else if (xz < -limx) { xz = -limx; o->clamp_x = 1; o->limx = -limx; }
    if (yz > limy) { yz = limy; o->clamp_y = 1; o->limy = limy; }
    else if (yz < -limy) { yz = -limy; o->clamp_y = 1; o->limy = -limy; }
    o->tx = xz * z;
    o->ty = yz * z;
    double* J = o->J;
    J[0] = cam->fx / z; J[1] = 0;              J[2] = -cam->fx * o->tx / (z * z);
    J[3] = 0;           J[4] = cam->fy / z;    J[5] = -cam->fy * o->ty / (z * z);

    /* Sigma2 = J Sc J^T */
    double JS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += J[3 * i + k] * o->Sc[3 * k + j];
            JS[3 * i + j] = s;
        }
    double S2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += JS[3 * i + k] * J[3 * j + k];
            S2[2 * i + j] = s;
        }
    o->a = S2[0] + cfg->dilation;
    o->b = S2[1];
    o->c = S2[3] + cfg->dilation;
    o->det = o->a * o->c - o->b * o->b;
    if (!(o->det > 0)) return;
    o->conic[0] = o->c / o->det;
    o->conic[1] = -o->b / o->det;
    o->conic[2] = o->a / o->det;
    double mid = 0.5 * (o->a + o->c);
    double disc = mid * mid - o->det;
    if (disc < 0.1) disc = 0.1;
    double lmax = mid + sqrt(disc);
    o->r3 = 3.0 * sqrt(lmax);
    o->radius = (int64_t)ceil(o->r3);
    o->u = cam->fx * x / z + cam->cx;
    o->v = cam->fy * y / z + cam->cy;
    o->opacity = 1.0 / (1.0 + exp(-ologit));
    o->visible = 1;
}

/* Forward projection of n Gaussians.
 * Outputs (all length n, row-major):
 *   uv[2n], conic[3n], depth[n], opacity[n], radius[n] (0 = culled or
 *   masked), rect[4n] = tile rect (x0, x1, y0, y1), touched[n] = number of
 *   tiles in the rect, r3[n] = 3 sqrt(lambda_max) before rounding (for the
 *   tests' boundary accounting). */
void or_project(int64_t n, const double* means, const double* log_scales, const double* quats,
                const double* opacity_logit, const uint8_t* mask, const or_cam* cam,
                const or_cfg* cfg, double* uv, double* conic, double* depth, double* opacity,
                int64_t* radius, int64_t* rect, int64_t* touched, double* r3) {
    for (int64_t k = 0; k < n; ++k) {
        uv[2 * k] = uv[2 * k + 1] = 0;
        conic[3 * k] = conic[3 * k + 1] = conic[3 * k + 2] = 0;
        depth[k] = 0; opacity[k] = 0; radius[k] = 0; touched[k] = 0; r3[k] = 0;
        rect[4 * k] = rect[4 * k + 1] = rect[4 * k + 2] = rect[4 * k + 3] = 0;
        if (mask && mask[k]) continue;
        or_proj1 o;
        project_one(means + 3 * k, log_scales + 3 * k, quats + 4 * k, opacity_logit[k], cam, cfg, &o);
        if (!o.visible) continue;
        uv[2 * k] = o.u; uv[2 * k + 1] = o.v;
        conic[3 * k] = o.conic[0]; conic[3 * k + 1] = o.conic[1]; conic[3 * k + 2] = o.conic[2];
        depth[k] = o.p[2];
        opacity[k] = o.opacity;
        radius[k] = o.radius;
        r3[k] = o.r3;
        int64_t box[4];
        tile_rect(cam, o.u, o.v, o.radius, o.conic, o.opacity, cfg->alpha_min, rect + 4 * k, box);
        touched[k] = (rect[4 * k + 1] - rect[4 * k]) * (rect[4 * k + 3] - rect[4 * k + 2]);
    }
}

/* ------------------------------------------------------------------------ */
/* Tile intersection and depth sort (Sec. 2.1, Steps 1-2 and 2)              */
/* ------------------------------------------------------------------------ */

static uint32_t f32_bits(double d) {
    float f = (float)d;
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

typedef struct { uint64_t key; uint32_t val; } or_kv;

static int cmp_kv(const void* pa, const void* pb) {
    const or_kv* a = (const or_kv*)pa;
    const or_kv* b = (const or_kv*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

/* Number of (tile, Gaussian) pairs: the sum of tiles touched (tile_rect with
 * the given conics, opacities and alpha_min). */
int64_t or_bin_count(int64_t n, const double* uv, const int64_t* radius, const double* conic,
                     const double* opacity, double alpha_min, const or_cam* cam) {
    int64_t total = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (radius[k] <= 0) continue;
        int64_t rect[4], box[4];
        tile_rect(cam, uv[2 * k], uv[2 * k + 1], radius[k], conic + 3 * k, opacity[k], alpha_min, rect, box);
        total += (rect[1] - rect[0]) * (rect[3] - rect[2]);
    }
    return total;
}

/* Keys, values and per-tile ranges.  For every Gaussian with radius > 0 and
 * every tile of its rect, one pair: key = tile_id << 32 | float32 bits of the
 * depth (depth > 0 so the bits order like the values), value = Gaussian id.
 * The pairs are sorted by (key, id) with the C library sort, so equal depths
 * inside a tile keep id order.  ranges[2t], ranges[2t+1] = first and one past
 * the last sorted index of tile t ([0,0) for an empty tile).  Buffers must
 * hold or_bin_count() pairs and 2*TX*TY range words. */
void or_bin_sort(int64_t n, const double* uv, const double* depth, const int64_t* radius, const double* conic,
                 const double* opacity, double alpha_min, const or_cam* cam, uint64_t* keys, uint32_t* vals,
                 uint32_t* ranges) {
    int64_t Ws, Hs, TX, TY;
    grid_dims(cam, &Ws, &Hs, &TX, &TY);
    int64_t total = or_bin_count(n, uv, radius, conic, opacity, alpha_min, cam);
    or_kv* kv = (or_kv*)malloc(sizeof(or_kv) * (size_t)(total > 0 ? total : 1));
    int64_t w = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (radius[k] <= 0) continue;
        int64_t rect[4], box[4];
        tile_rect(cam, uv[2 * k], uv[2 * k + 1], radius[k], conic + 3 * k, opacity[k], alpha_min, rect, box);
        for (int64_t ty = rect[2]; ty < rect[3]; ++ty)
            for (int64_t tx = rect[0]; tx < rect[1]; ++tx) {
                uint64_t tile = (uint64_t)(ty * TX + tx);
                kv[w].key = (tile << 32) | (uint64_t)f32_bits(depth[k]);
                kv[w].val = (uint32_t)k;
                ++w;
            }
    }
    qsort(kv, (size_t)total, sizeof(or_kv), cmp_kv);
    for (int64_t t = 0; t < TX * TY; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t i = 0; i < total; ++i) {
        keys[i] = kv[i].key;
        vals[i] = kv[i].val;
        uint64_t t = kv[i].key >> 32;
        if (i == 0 || (kv[i - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)i;
        if (i == total - 1 || (kv[i + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
    free(kv);
}

/* ------------------------------------------------------------------------ */
/* Rendering (Sec. 2.1, Step 3: Eq. 2 and Eq. 3)                             */
/* ------------------------------------------------------------------------ */

/* Inputs of the renderer: the projected 2D Gaussians. */
typedef struct {
    int64_t n;
    const double* uv;       /* [n,2] */
    const double* conic;    /* [n,3] (A, B, C) of [[A,B],[B,C]] */
    const double* opacity;  /* [n] */
    const double* rgb;      /* [n,3] */
    const double* depth;    /* [n] */
    const int64_t* radius;  /* [n] */
} or_splats;

/* One fragment f_{P,k} as the compositing visits it. */
typedef struct {
    int64_t k;        /* Gaussian id */
    int64_t list_pos; /* index inside the tile list (tiled variant) */
    double dx, dy;    /* pixel centre minus 2D mean */
    double G;         /* exp(power) */
    double alpha;     /* min(alpha_max, o G) */
    int clamped;      /* o G exceeded alpha_max */
    double T;         /* transmittance before this fragment */
} or_frag;

/* Integer box test of reading new-1: is pixel (px, py) inside
 * [floor(u) - r, floor(u) + r] x [floor(v) - r, floor(v) + r]?  The floors
 * are integer decisions that a float32 mean can take the other way when u or
 * v lies within its rounding of an integer: box_window gives that window,
 * d = 1e-5 max(1, |u|) (likewise for v), and box_float_decided says whether
 * flooring u -+ d or v -+ d moves a floor.  For such a Gaussian in_box sets
 * *amb when the four combinations of those floors do not decide the pixel's
 * inclusion the same way (decided = 0: *amb = 0). */
static double box_window(double u) { return 1e-5 * fmax(1.0, fabs(u)); }

static double clamp_coord(double u) { return u < -1e9 ? -1e9 : (u > 1e9 ? 1e9 : u); }

static int box_float_decided(double u, double v) {
    u = clamp_coord(u);
    v = clamp_coord(v);
    const double du = box_window(u), dv = box_window(v);
    return floor(u - du) != floor(u + du) || floor(v - dv) != floor(v + dv);
}

static int in_box(double u, double v, int64_t r, int64_t px, int64_t py, int decided, int* amb) {
    u = clamp_coord(u);
    v = clamp_coord(v);
    const int64_t xi = (int64_t)floor(u), yi = (int64_t)floor(v);
    const int in = !(px < xi - r || px > xi + r || py < yi - r || py > yi + r);
    *amb = 0;
    if (!decided) return in;
    const double du = box_window(u), dv = box_window(v);
    const int64_t xs[2] = {(int64_t)floor(u - du), (int64_t)floor(u + du)};
    const int64_t ys[2] = {(int64_t)floor(v - dv), (int64_t)floor(v + dv)};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int ib = !(px < xs[a] - r || px > xs[a] + r || py < ys[b] - r || py > ys[b] + r);
            if (ib != in) *amb = 1;
        }
    return in;
}

/* box_float_decided of every Gaussian (malloc'ed; the caller frees it). */
static uint8_t* float_decided_boxes(const or_splats* s) {
    uint8_t* f = (uint8_t*)calloc((size_t)(s->n + 1), 1);
    for (int64_t k = 0; k < s->n; ++k) f[k] = (uint8_t)box_float_decided(s->uv[2 * k], s->uv[2 * k + 1]);
    return f;
}

/* Per-pixel compositing of an ordered candidate list (Eq. 2, Eq. 3).
 * Readings: the pixel centre is (px + 0.5, py + 0.5) in full-resolution
 * pixels; a candidate outside the Gaussian's integer box is not a fragment
 * of this pixel; power = -1/2 (A dx^2 + C dy^2) - B dx dy; power > 0 is
 * skipped; alpha = min(alpha_max, o exp(power)); alpha < alpha_min is
 * skipped; if T (1 - alpha) < t_eps the ray stops before this fragment is
 * blended (early termination, Eq. 3 note); colour and depth blend with the
 * same weights T alpha; the background enters with weight T_final.
 * A candidate whose box inclusion is float-decided (in_box's *amb, for the
 * Gaussians flagged in fdec by box_float_decided) marks the pixel marginal
 * if it would blend there (power <= 0, alpha within the margin of alpha_min
 * or above); the float64 floors decide the fragment.
 * Writes the composited fragments to frags (if not NULL) and returns their
 * count.  *last_pos = list position + 1 of the last composited fragment.
 * margin accumulates whether any predicate was within a relative 1e-4 of its
 * threshold (a pixel where FP32 and FP64 may legitimately disagree). */
static int64_t composite_pixel(const or_splats* s, const uint8_t* fdec, const or_cfg* cfg, int64_t px,
                               int64_t py, const int64_t* cand, int64_t ncand, or_frag* frags,
                               double out_rgb[3], double* out_depth, double* out_T,
                               int64_t* last_pos, int* margin) {
    double T = 1.0, C[3] = {0, 0, 0}, D = 0;
    int64_t nf = 0;
    *last_pos = 0;
    const double rel = 1e-4;
    double pxc = (double)px + 0.5, pyc = (double)py + 0.5;
    for (int64_t i = 0; i < ncand; ++i) {
        int64_t k = cand[i];
        int64_t r = s->radius[k];
        if (r <= 0) continue;
        double u = s->uv[2 * k], v = s->uv[2 * k + 1];
        int amb;
        const int in = in_box(u, v, r, px, py, fdec[k], &amb);
        if (!in && !amb) continue;
        double dx = pxc - u, dy = pyc - v;
        double A = s->conic[3 * k], B = s->conic[3 * k + 1], Cc = s->conic[3 * k + 2];
        double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        if (amb && power <= 0 && s->opacity[k] * exp(power) >= (1.0 - rel) * cfg->alpha_min)
            *margin = 1;
        if (!in) continue;
        if (fabs(power) < 1e-6) *margin = 1;
        if (power > 0) continue;
        double G = exp(power);
        double a = s->opacity[k] * G;
        int clamped = 0;
        if (fabs(a - cfg->alpha_max) < rel * cfg->alpha_max) *margin = 1;
        if (a > cfg->alpha_max) { a = cfg->alpha_max; clamped = 1; }
        if (fabs(a - cfg->alpha_min) < rel * cfg->alpha_min) *margin = 1;
        if (a < cfg->alpha_min) continue;
        double Tn = T * (1.0 - a);
        if (fabs(Tn - cfg->t_eps) < rel * cfg->t_eps) *margin = 1;
        if (Tn < cfg->t_eps) break;
        if (frags) {
            or_frag* f = &frags[nf];
            f->k = k; f->list_pos = i; f->dx = dx; f->dy = dy; f->G = G;
            f->alpha = a; f->clamped = clamped; f->T = T;
        }
        ++nf;
        for (int c = 0; c < 3; ++c) C[c] += T * a * s->rgb[3 * k + c];
        D += T * a * s->depth[k];
        T = Tn;
        *last_pos = i + 1;
    }
    for (int c = 0; c < 3; ++c) out_rgb[c] = C[c] + T * cfg->bg[c];
    *out_depth = D;
    *out_T = T;
    return nf;
}

/* Candidate list of a sampled pixel from the per-tile sorted lists. */
static int64_t tile_candidates(const or_cam* cam, int64_t i, int64_t j, const uint32_t* vals,
                               const uint32_t* ranges, int64_t* cand) {
    int64_t Ws, Hs, TX, TY;
    grid_dims(cam, &Ws, &Hs, &TX, &TY);
    int64_t t = (j / tile_dim(cam->sy)) * TX + (i / tile_dim(cam->sx));
    int64_t b = ranges[2 * t], e = ranges[2 * t + 1];
    for (int64_t q = b; q < e; ++q) cand[q - b] = vals[q];
    return e - b;
}

typedef struct { uint32_t dbits; int64_t k; } or_dk;
static int cmp_dk(const void* pa, const void* pb) {
    const or_dk* a = (const or_dk*)pa;
    const or_dk* b = (const or_dk*)pb;
    if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
    return a->k < b->k ? -1 : (a->k > b->k);
}

/* Candidate list of a pixel by brute force: every Gaussian with radius > 0
 * whose integer box contains the pixel (or may, in float32: in_box's *amb),
 * ordered by (float32 depth bits, id). */
static int64_t brute_candidates(const or_splats* s, const uint8_t* fdec, int64_t px, int64_t py, int64_t* cand,
                                or_dk* scratch) {
    int64_t m = 0;
    for (int64_t k = 0; k < s->n; ++k) {
        int64_t r = s->radius[k];
        if (r <= 0) continue;
        int amb;
        if (!in_box(s->uv[2 * k], s->uv[2 * k + 1], r, px, py, fdec[k], &amb) && !amb) continue;
        scratch[m].dbits = f32_bits(s->depth[k]);
        scratch[m].k = k;
        ++m;
    }
    qsort(scratch, (size_t)m, sizeof(or_dk), cmp_dk);
    for (int64_t q = 0; q < m; ++q) cand[q] = scratch[q].k;
    return m;
}

/* Forward render of the sampled image (Ws x Hs).  vals/ranges = the tile
 * lists from or_bin_sort, or NULL for the brute-force variant.
 * Outputs: rgb [3,Hs,Ws] (planar), depth [Hs,Ws], T_final [Hs,Ws],
 * last [Hs,Ws] (tile-list position + 1 of the last composited fragment;
 * count of candidates up to it in the brute-force variant), nfrag [Hs,Ws]
 * (composited fragments), margin [Hs,Ws] (1 if any predicate was marginal).
 * Returns the sum over pixels of a fragment signature used by the finite
 * difference tests to detect a change of the composited set. */
double or_render_fwd(const or_splats* s, const or_cam* cam, const or_cfg* cfg,
                     const uint32_t* vals, const uint32_t* ranges, double* rgb, double* depth,
                     double* T_final, int64_t* last, int64_t* nfrag, uint8_t* margin) {
    int64_t Ws, Hs, TX, TY;
    grid_dims(cam, &Ws, &Hs, &TX, &TY);
    int64_t P = Ws * Hs;
    int64_t maxc = s->n;
    if (vals) {
        maxc = 0;
        for (int64_t t = 0; t < TX * TY; ++t)
            if (ranges[2 * t + 1] - ranges[2 * t] > maxc) maxc = ranges[2 * t + 1] - ranges[2 * t];
    }
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxc + 1));
    or_dk* scratch = vals ? NULL : (or_dk*)malloc(sizeof(or_dk) * (size_t)(s->n + 1));
    or_frag* frags = (or_frag*)malloc(sizeof(or_frag) * (size_t)(maxc + 1));
    uint8_t* fdec = float_decided_boxes(s);
    double sig = 0;
    for (int64_t j = 0; j < Hs; ++j)
        for (int64_t i = 0; i < Ws; ++i) {
            int64_t px = i * cam->sx, py = j * cam->sy;
            int64_t nc = vals ? tile_candidates(cam, i, j, vals, ranges, cand)
                              : brute_candidates(s, fdec, px, py, cand, scratch);
            double c3[3], d, T;
            int64_t lp;
            int mg = 0;
            int64_t nf = composite_pixel(s, fdec, cfg, px, py, cand, nc, frags, c3, &d, &T, &lp, &mg);
            int64_t pix = j * Ws + i;
            for (int c = 0; c < 3; ++c) rgb[c * P + pix] = c3[c];
            depth[pix] = d;
            T_final[pix] = T;
            last[pix] = lp;
            nfrag[pix] = nf;
            margin[pix] = (uint8_t)mg;
            for (int64_t q = 0; q < nf; ++q)
                sig += (double)((frags[q].k + 1) % 1000003) * (double)((pix % 997) + 1);
        }
    free(cand);
    free(scratch);
    free(frags);
    free(fdec);
    return sig;
}

/* ------------------------------------------------------------------------ */
/* Loss (Sec. 4.1, Eq. 6)                                                    */
/* ------------------------------------------------------------------------ */

/* L = w_rgb * mean_{3P} |C - C_hat| + w_depth * mean_{P} |D - D_hat|, the
 * depth term only where the target depth is non-zero (zero marks an invalid
 * depth measurement).  With w_rgb = lambda_pho and w_depth = 1 - lambda_pho
 * this is Eq. 6 with L1 residuals; the tracking workload uses w_rgb = 1,
 * w_depth = 0.5.  sign(0) = 0.  Writes dL/dC [3,P] and dL/dD [P]. */
double or_loss_l1(int64_t P, const double* rgb, const double* depth, const double* trgb,
                  const double* tdepth, double w_rgb, double w_depth, double* d_rgb,
                  double* d_depth) {
    double L = 0;
    for (int64_t q = 0; q < 3 * P; ++q) {
        double r = rgb[q] - trgb[q];
        L += w_rgb * fabs(r) / (3.0 * (double)P);
        d_rgb[q] = w_rgb * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (3.0 * (double)P);
    }
    for (int64_t q = 0; q < P; ++q) {
        d_depth[q] = 0;
        if (tdepth[q] == 0) continue;
        double r = depth[q] - tdepth[q];
        L += w_depth * fabs(r) / (double)P;
        d_depth[q] = w_depth * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)P;
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Rendering backpropagation (Sec. 2.2, Step 4)                              */
/* ------------------------------------------------------------------------ */

/* Gradients of L with respect to the 2D Gaussian attributes, given dL/dC
 * [3,P] and dL/dD [P].  Layout of grad2d, 12 doubles per Gaussian:
 *   [0] dL/du  [1] dL/dv  [2] dL/dA  [3] dL/dB  [4] dL/dC (conic)
 *   [5] dL/dopacity  [6] dL/ddepth  [7] 0  [8..10] dL/drgb  [11] 0.
 * For each pixel the composited fragments are re-derived exactly as in the
 * forward pass, and Eq. 3 is differentiated directly:
 *   C = sum_k T_k a_k c_k + T_final bg,  T_k = prod_{n<k} (1 - a_n),
 *   dC/dc_k = T_k a_k,
 *   dC/da_k = T_k c_k - S_k / (1 - a_k),  S_k = sum_{n>k} T_n a_n c_n + T_final bg,
 * and the same for depth with d_k and no background.  The paper's Eq. 4 is
 * this expression without T_k and 1/(1-a_k); Eq. 5 is the reverse recovery
 * of T_k, which the oracle does not need because it keeps T_k from the
 * forward products.  Through a = o G (G = exp(power)), unless clamped:
 *   dL/do = G dL/da,  dL/dpower = a dL/da,
 *   power = -1/2 (A dx^2 + C dy^2) - B dx dy,  dx = px + 0.5 - u. */
void or_render_bwd(const or_splats* s, const or_cam* cam, const or_cfg* cfg,
                   const uint32_t* vals, const uint32_t* ranges, const double* d_rgb,
                   const double* d_depth, double* grad2d) {
    int64_t Ws, Hs, TX, TY;
    grid_dims(cam, &Ws, &Hs, &TX, &TY);
    int64_t P = Ws * Hs;
    memset(grad2d, 0, sizeof(double) * 12 * (size_t)s->n);
    int64_t maxc = s->n;
    if (vals) {
        maxc = 0;
        for (int64_t t = 0; t < TX * TY; ++t)
            if (ranges[2 * t + 1] - ranges[2 * t] > maxc) maxc = ranges[2 * t + 1] - ranges[2 * t];
    }
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxc + 1));
    or_dk* scratch = vals ? NULL : (or_dk*)malloc(sizeof(or_dk) * (size_t)(s->n + 1));
    or_frag* f = (or_frag*)malloc(sizeof(or_frag) * (size_t)(maxc + 1));
    uint8_t* fdec = float_decided_boxes(s);
    double* SC = (double*)malloc(sizeof(double) * 3 * (size_t)(maxc + 1));
    double* SD = (double*)malloc(sizeof(double) * (size_t)(maxc + 1));
    for (int64_t j = 0; j < Hs; ++j)
        for (int64_t i = 0; i < Ws; ++i) {
            int64_t px = i * cam->sx, py = j * cam->sy;
            int64_t nc = vals ? tile_candidates(cam, i, j, vals, ranges, cand)
                              : brute_candidates(s, fdec, px, py, cand, scratch);
            double c3[3], d, Tf;
            int64_t lp;
            int mg = 0;
            int64_t nf = composite_pixel(s, fdec, cfg, px, py, cand, nc, f, c3, &d, &Tf, &lp, &mg);
            int64_t pix = j * Ws + i;
            double gC[3] = {d_rgb[pix], d_rgb[P + pix], d_rgb[2 * P + pix]};
            double gD = d_depth[pix];
            /* suffix sums S_k (exclusive of k), background included */
            double accC[3] = {Tf * cfg->bg[0], Tf * cfg->bg[1], Tf * cfg->bg[2]};
            double accD = 0;
            for (int64_t q = nf - 1; q >= 0; --q) {
                for (int c = 0; c < 3; ++c) SC[3 * q + c] = accC[c];
                SD[q] = accD;
                int64_t k = f[q].k;
                double w = f[q].T * f[q].alpha;
                for (int c = 0; c < 3; ++c) accC[c] += w * s->rgb[3 * k + c];
                accD += w * s->depth[k];
            }
            for (int64_t q = 0; q < nf; ++q) {
                int64_t k = f[q].k;
                double a = f[q].alpha, T = f[q].T;
                double* g = grad2d + 12 * k;
                double dLda = 0;
                for (int c = 0; c < 3; ++c) {
                    g[8 + c] += T * a * gC[c];
                    dLda += gC[c] * (T * s->rgb[3 * k + c] - SC[3 * q + c] / (1.0 - a));
                }
                g[6] += T * a * gD;
                dLda += gD * (T * s->depth[k] - SD[q] / (1.0 - a));
                if (f[q].clamped) continue;
                double G = f[q].G;
                g[5] += G * dLda;
                double dpow = a * dLda;
                double dx = f[q].dx, dy = f[q].dy;
                double A = s->conic[3 * k], B = s->conic[3 * k + 1], Cc = s->conic[3 * k + 2];
                g[2] += -0.5 * dx * dx * dpow;
                g[3] += -dx * dy * dpow;
                g[4] += -0.5 * dy * dy * dpow;
                g[0] += (A * dx + B * dy) * dpow;
                g[1] += (B * dx + Cc * dy) * dpow;
            }
        }
    free(cand);
    free(scratch);
    free(f);
    free(fdec);
    free(SC);
    free(SD);
}

/* ------------------------------------------------------------------------ */
/* Preprocessing backpropagation and camera pose (Sec. 2.2, Step 5)          */
/* ------------------------------------------------------------------------ */

/* Chain the 2D gradients back through the projection of each Gaussian.
 * Outputs (any may be NULL):
 *   d_means[3n], d_log_scales[3n], d_quats[4n] (w.r.t. the unnormalised
 *   quaternion), d_opacity_logit[n], d_rgb[3n];
 *   d_pcam[3n] = dL/dp (camera-frame mean), d_Sc[9n] = dL/dSigma_c;
 *   pose_grad[6] = dL/dxi summed over Gaussians for the left perturbation
 *   T_cw <- exp(xi^) T_cw, xi = (rho, phi): dL/drho = sum_k dL/dp_k,
 *   dL/dphi = sum_k [p_k x dL/dp_k + (<G_k, [e_i]x Sc_k - Sc_k [e_i]x>)_i],
 *   G_k = dL/dSc_k (Sec. 2.2: per-Gaussian dL/dP_k aggregated into dL/dP);
 *   score_terms[2n] = (||dL/dmu||_2, ||dL/dSigma||_F) for Eq. 7. */
void or_project_bwd(int64_t n, const double* means, const double* log_scales, const double* quats,
                    const double* opacity_logit, const uint8_t* mask, const or_cam* cam,
                    const or_cfg* cfg, const double* grad2d, double* d_means,
                    double* d_log_scales, double* d_quats, double* d_opacity_logit,
                    double* d_rgb, double* d_pcam, double* d_Sc, double* pose_grad,
                    double* score_terms) {
    if (pose_grad) for (int i = 0; i < 6; ++i) pose_grad[i] = 0;
    const double* R = cam->R;
    for (int64_t k = 0; k < n; ++k) {
        if (d_means) for (int i = 0; i < 3; ++i) d_means[3 * k + i] = 0;
        if (d_log_scales) for (int i = 0; i < 3; ++i) d_log_scales[3 * k + i] = 0;
        if (d_quats) for (int i = 0; i < 4; ++i) d_quats[4 * k + i] = 0;
        if (d_opacity_logit) d_opacity_logit[k] = 0;
        if (d_rgb) for (int i = 0; i < 3; ++i) d_rgb[3 * k + i] = 0;
        if (d_pcam) for (int i = 0; i < 3; ++i) d_pcam[3 * k + i] = 0;
        if (d_Sc) for (int i = 0; i < 9; ++i) d_Sc[9 * k + i] = 0;
        if (score_terms) { score_terms[2 * k] = 0; score_terms[2 * k + 1] = 0; }
        if (mask && mask[k]) continue;
        or_proj1 o;
        project_one(means + 3 * k, log_scales + 3 * k, quats + 4 * k, opacity_logit[k], cam, cfg, &o);
        if (!o.visible) continue;
        const double* g2 = grad2d + 12 * k;
        double x = o.p[0], y = o.p[1], z = o.p[2];
        double fx = cam->fx, fy = cam->fy;

        /* conic Q = S2^{-1}: dL/dS2 = -Q Gq Q, Gq = [[gA, gB/2], [gB/2, gC]] */
        double Q[4] = {o.conic[0], o.conic[1], o.conic[1], o.conic[2]};
        double Gq[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
        double QG[4], G2[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                QG[2 * i + j] = Q[2 * i] * Gq[j] + Q[2 * i + 1] * Gq[2 + j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                G2[2 * i + j] = -(QG[2 * i] * Q[j] + QG[2 * i + 1] * Q[2 + j]);

        /* S2 = J Sc J^T (+ dilation): dL/dSc = J^T G2 J, dL/dJ = 2 G2 J Sc */
        const double* J = o.J;
        double Gc[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) s += J[3 * a + i] * G2[2 * a + b] * J[3 * b + j];
                Gc[3 * i + j] = s;
            }
        double GJ[6];
        for (int a = 0; a < 2; ++a)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int b = 0; b < 2; ++b)
                    for (int m = 0; m < 3; ++m) s += G2[2 * a + b] * J[3 * b + m] * o.Sc[3 * m + j];
                GJ[3 * a + j] = 2.0 * s;
            }

        /* dL/dp from J (entries J00, J02, J11, J12 depend on p) */
        double gp[3] = {0, 0, 0};
        gp[2] += GJ[0] * (-fx / (z * z));
        gp[2] += GJ[4] * (-fy / (z * z));
        if (o.clamp_x) {
            gp[2] += GJ[2] * (fx * o.limx / (z * z));
        } else {
            gp[0] += GJ[2] * (-fx / (z * z));
            gp[2] += GJ[2] * (2.0 * fx * x / (z * z * z));
        }
        if (o.clamp_y) {
            gp[2] += GJ[5] * (fy * o.limy / (z * z));
        } else {
            gp[1] += GJ[5] * (-fy / (z * z));
            gp[2] += GJ[5] * (2.0 * fy * y / (z * z * z));
        }
        /* from the 2D mean u = fx x/z + cx, v = fy y/z + cy, and depth d = z */
        gp[0] += g2[0] * fx / z;
        gp[1] += g2[1] * fy / z;
        gp[2] += -g2[0] * fx * x / (z * z) - g2[1] * fy * y / (z * z);
        gp[2] += g2[6];

        /* world frame: p = R mu + t, Sc = R Sigma R^T */
        double gmu[3];
        for (int j = 0; j < 3; ++j) gmu[j] = R[j] * gp[0] + R[3 + j] * gp[1] + R[6 + j] * gp[2];
        double RT[9], tmp[9], GS[9];
        mat3_T(R, RT);
        mat3_mul(RT, Gc, tmp);
        mat3_mul(tmp, R, GS);

        /* Sigma = M M^T, M = Rq diag(scale): dL/dM = 2 GS M */
        double GM[9];
        mat3_mul(GS, o.M, GM);
        for (int i = 0; i < 9; ++i) GM[i] *= 2.0;
        double gls[3], GR[9];
        for (int j = 0; j < 3; ++j) {
            gls[j] = 0;
            for (int i = 0; i < 3; ++i) gls[j] += GM[3 * i + j] * o.M[3 * i + j];
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) GR[3 * i + j] = GM[3 * i + j] * o.scale[j];
        /* rotation of the unit quaternion (w, x, y, z) */
        double w = o.qn[0], qx = o.qn[1], qy = o.qn[2], qz = o.qn[3];
        double gq[4];
        gq[0] = 2 * (-qz * GR[1] + qy * GR[2] + qz * GR[3] - qx * GR[5] - qy * GR[6] + qx * GR[7]);
        gq[1] = 2 * (qy * GR[1] + qz * GR[2] + qy * GR[3] - 2 * qx * GR[4] - w * GR[5] + qz * GR[6] +
                     w * GR[7] - 2 * qx * GR[8]);
        gq[2] = 2 * (-2 * qy * GR[0] + qx * GR[1] + w * GR[2] + qx * GR[3] + qz * GR[5] - w * GR[6] +
                     qz * GR[7] - 2 * qy * GR[8]);
        gq[3] = 2 * (-2 * qz * GR[0] - w * GR[1] + qx * GR[2] + w * GR[3] - 2 * qz * GR[4] +
                     qy * GR[5] + qx * GR[6] + qy * GR[7]);
        /* through the normalisation q / |q| */
        double dotq = 0;
        for (int i = 0; i < 4; ++i) dotq += o.qn[i] * gq[i];
        if (d_means) for (int i = 0; i < 3; ++i) d_means[3 * k + i] = gmu[i];
        if (d_log_scales) for (int i = 0; i < 3; ++i) d_log_scales[3 * k + i] = gls[i];
        if (d_quats)
            for (int i = 0; i < 4; ++i) d_quats[4 * k + i] = (gq[i] - o.qn[i] * dotq) / o.qlen;
        if (d_opacity_logit) d_opacity_logit[k] = g2[5] * o.opacity * (1.0 - o.opacity);
        if (d_rgb) for (int i = 0; i < 3; ++i) d_rgb[3 * k + i] = g2[8 + i];
        if (d_pcam) for (int i = 0; i < 3; ++i) d_pcam[3 * k + i] = gp[i];
        if (d_Sc) for (int i = 0; i < 9; ++i) d_Sc[9 * k + i] = Gc[i];
        if (score_terms) {
            score_terms[2 * k] = sqrt(gmu[0] * gmu[0] + gmu[1] * gmu[1] + gmu[2] * gmu[2]);
            double fr = 0;
            for (int i = 0; i < 9; ++i) fr += GS[i] * GS[i];
            score_terms[2 * k + 1] = sqrt(fr);
        }
        if (pose_grad) {
            const double* p = o.p;
            pose_grad[0] += gp[0];
            pose_grad[1] += gp[1];
            pose_grad[2] += gp[2];
            double cr[3] = {p[1] * gp[2] - p[2] * gp[1], p[2] * gp[0] - p[0] * gp[2],
                            p[0] * gp[1] - p[1] * gp[0]};
            for (int e = 0; e < 3; ++e) {
                double E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                /* [e]x for unit axis e */
                if (e == 0) { E[5] = -1; E[7] = 1; }
                if (e == 1) { E[2] = 1; E[6] = -1; }
                if (e == 2) { E[1] = -1; E[3] = 1; }
                double ES[9], SE[9];
                mat3_mul(E, o.Sc, ES);
                mat3_mul(o.Sc, E, SE);
                double s = 0;
                for (int i = 0; i < 9; ++i) s += Gc[i] * (ES[i] - SE[i]);
                pose_grad[3 + e] += cr[e] + s;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Adaptive Gaussian pruning (Sec. 4.1, Eq. 7)                               */
/* ------------------------------------------------------------------------ */

typedef struct { uint32_t sbits; int64_t k; } or_sk;
static int cmp_sk(const void* pa, const void* pb) {
    const or_sk* a = (const or_sk*)pa;
    const or_sk* b = (const or_sk*)pb;
    if (a->sbits != b->sbits) return a->sbits < b->sbits ? -1 : 1;
    return a->k < b->k ? -1 : (a->k > b->k);
}

/* Score_k = ||dL/dmu_k|| + lambda ||dL/dSigma_k|| (Eq. 7), formed in float32
 * exactly as the GPU forms it (product rounded, then sum rounded; no fused
 * multiply-add), because the score decides which Gaussians are masked.
 * Among the Gaussians not yet masked (mask[k] == 0), the m = min(floor(frac
 * * n_active), max_select) ones smallest in (score, id) order are masked
 * (mask[k] = 1).  Non-negative float scores order like their bit patterns.
 * Returns m. */
int64_t or_prune_select(int64_t n, const float* t_mu, const float* t_sigma, float lambda,
                        double frac, int64_t max_select, uint8_t* mask) {
    or_sk* a = (or_sk*)malloc(sizeof(or_sk) * (size_t)(n + 1));
    int64_t na = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (mask[k]) continue;
        float prod = lambda * t_sigma[k];
        float s = t_mu[k] + prod;
        uint32_t b;
        memcpy(&b, &s, 4);
        a[na].sbits = b;
        a[na].k = k;
        ++na;
    }
    int64_t m = (int64_t)floor(frac * (double)na);
    if (m > max_select) m = max_select;
    if (m < 0) m = 0;
    qsort(a, (size_t)na, sizeof(or_sk), cmp_sk);
    for (int64_t q = 0; q < m; ++q) mask[a[q].k] = 1;
    free(a);
    return m;
}

/* Next pruning interval (Sec. 4.1).  After an interval of K iterations the
 * change ratio r of tile-Gaussian intersections is measured; if r exceeds the
 * threshold (5 %) the interval halves, else it doubles.  The paper states the
 * rule with K0 for the first interval; the current K plays that role for the
 * next one, floored at 1 and capped at k_max.  literal != 0 keeps the
 * paper's constants instead: K0/2 (integer division, at least 1) or 2 K0. */
int32_t or_next_interval(int32_t K, int32_t K0, double r, double thr, int32_t k_max, int literal) {
    if (literal) {
        if (r > thr) return K0 / 2 > 0 ? K0 / 2 : 1;
        return 2 * K0;
    }
    int32_t nk = r > thr ? K / 2 : 2 * K;
    if (nk < 1) nk = 1;
    if (nk > k_max) nk = k_max;
    return nk;
}

/* Change ratio of tile-Gaussian intersections: |A xor B| / max(1, |A|) over
 * the sets of (tile, Gaussian id) pairs, each given as a list of 64-bit codes
 * tile << 32 | id (any order, no duplicates). */
static int cmp_u64(const void* pa, const void* pb) {
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    return a < b ? -1 : (a > b);
}
double or_change_ratio(int64_t na, const uint64_t* A, int64_t nb, const uint64_t* B) {
    uint64_t* a = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(na + 1));
    uint64_t* b = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nb + 1));
    memcpy(a, A, sizeof(uint64_t) * (size_t)na);
    memcpy(b, B, sizeof(uint64_t) * (size_t)nb);
    qsort(a, (size_t)na, sizeof(uint64_t), cmp_u64);
    qsort(b, (size_t)nb, sizeof(uint64_t), cmp_u64);
    int64_t i = 0, j = 0, common = 0;
    while (i < na && j < nb) {
        if (a[i] == b[j]) { ++common; ++i; ++j; }
        else if (a[i] < b[j]) ++i;
        else ++j;
    }
    free(a);
    free(b);
    double sym = (double)(na - common) + (double)(nb - common);
    return sym / (double)(na > 1 ? na : 1);
}

/* ------------------------------------------------------------------------ */
/* Dynamic downsampling (Sec. 4.2)                                           */
/* ------------------------------------------------------------------------ */

/* Resolution of frame n: R0 for a keyframe, else min(R0/16 * m^(n-k-1),
 * R0/4) with k the last keyframe.  R is read as a pixel count and realised
 * as point sampling with strides (sx, sy) whose product is R0/R: 16 -> (4,4),
 * 8 -> (4,2), 4 -> (2,2).  m must be a power of two (the paper uses 2) so
 * that R0/R is one of those.  Returns 0 on success, -1 on a bad argument. */
int or_downsample_schedule(int64_t n, int64_t k, int is_keyframe, int64_t m, int32_t* sx, int32_t* sy) {
    if (is_keyframe) { *sx = 1; *sy = 1; return 0; }
    if (m < 2 || (m & (m - 1)) != 0 || n <= k) return -1;
    /* R0/R = max(16 / m^(n-k-1), 4) */
    int64_t e = n - k - 1;
    int64_t ratio = 16;
    for (int64_t q = 0; q < e && ratio > 4; ++q) ratio /= m;
    if (ratio < 4) ratio = 4;
    if (ratio == 16) { *sx = 4; *sy = 4; }
    else if (ratio == 8) { *sx = 4; *sy = 2; }
    else { *sx = 2; *sy = 2; }
    return 0;
}

/* Target at the sampled pixels: out[c, j, i] = full[c, sy*j, sx*i]. */
void or_gather(const double* full, int64_t C, int64_t W, int64_t H, int32_t sx, int32_t sy,
               double* out) {
    int64_t Ws = ceil_div(W, sx), Hs = ceil_div(H, sy);
    for (int64_t c = 0; c < C; ++c)
        for (int64_t j = 0; j < Hs; ++j)
            for (int64_t i = 0; i < Ws; ++i)
                out[(c * Hs + j) * Ws + i] = full[(c * H + j * sy) * W + i * sx];
}
