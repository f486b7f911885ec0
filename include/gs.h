/*
 * gs.h -- C ABI of a GB300 (sm_103a) differentiable tile-based 3D Gaussian
 * rasterizer: the per-iteration hot path of 3DGS-SLAM tracking and mapping as
 * described by RTGS (arXiv 2510.06644, Sec. 2.1-2.2 and Sec. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Every array argument is a DEVICE pointer unless a comment says
 *   "host".  The caller allocates and frees all device memory, including
 *   workspace; the library never allocates, frees or synchronises, except
 *   gs_status_poll(..., blocking=1), which synchronises the given stream.
 * Streams.  Work is enqueued asynchronously on the caller's stream (a
 *   cudaStream_t passed as gs_stream; NULL = the legacy default stream).
 * Workspace.  Entry points that need scratch take (void* workspace,
 *   size_t* workspace_bytes).  With workspace == NULL they only store the
 *   required size in *workspace_bytes and return GS_OK.  Otherwise
 *   *workspace_bytes must be at least that size (GS_ERR_WORKSPACE if not) and
 *   the workspace must be 256-byte aligned.
 * Errors.  Argument checks are synchronous and return a gs_status; the
 *   thread-local message is in gs_last_error().  Conditions found on the
 *   device (a bounded wait that gave up, a key count above the capacity) set
 *   a per-device status word that gs_status_poll() reads.  No C++ exception
 *   crosses this boundary.
 * Images.  The camera renders the full-resolution W x H image sampled with
 *   strides (sx, sy) (Sec. 4.2 dynamic downsampling): the sampled image has
 *   Ws = ceil(W/sx) columns and Hs = ceil(H/sy) rows, sampled pixel (i, j) is
 *   full-resolution pixel (sx*i, sy*j) and is evaluated at its centre
 *   (sx*i + 0.5, sy*j + 0.5).  Images are planar float32: rgb [3][Hs][Ws],
 *   depth [Hs][Ws].  Tiles are tw x th sampled pixels with tw = 16 / p2(sx)
 *   and th = 16 / p2(sy), at least 4 (p2(s) = smallest power of two >= s),
 *   so every tile keeps the 16 x 16 full-resolution footprint of the paper's
 *   tile (Sec. 2.1, Step 1-2 footnote): 16 x 16 at full resolution.
 *   TX = ceil(Ws/tw) by TY = ceil(Hs/th), row-major tile ids.
 * Empty inputs.  n = 0 Gaussians, zero keys and empty tiles are valid.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs_stream; /* identical to cudaStream_t */

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,   /* bad pointer, size, stride or enum */
    GS_ERR_WORKSPACE = 2,     /* workspace smaller than required */
    GS_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    GS_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    GS_ERR_CAPACITY = 5,      /* more (tile, Gaussian) keys than the output holds */
    GS_ERR_DEVICE_CHECK = 6,  /* a device-side consistency check failed */
    GS_ERR_UNIMPLEMENTED = 7
} gs_status;

enum { GS_TRACK = 0, GS_MAP = 1 };           /* backward modes (Sec. 2.2) */
enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 }; /* 2D record storage types */
enum { GS_IDLE = 0, GS_EXECUTING = 1 };       /* gs_status_poll state */

/* Pinhole camera.  R, t map world to camera (x_c = R x_w + t), row-major R.
 * fx, fy focal lengths and cx, cy principal point, in full-resolution pixels;
 * the 2D mean of a camera point (x, y, z) is (fx x/z + cx, fy y/z + cy). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height; /* full-resolution image W, H */
    int32_t sx, sy;        /* sampling strides, >= 1 */
    const float* pose;     /* NULL, or a DEVICE float[12] (R row-major, then t)
                              that replaces R and t when a kernel starts, so a
                              pose updated on the device (gs_pose_update) is
                              used without a host round trip */
} gs_camera;

/* Method constants.  gs_default_config() fills the values used throughout:
 * near_z 0.2, dilation 0.3, alpha_min 1/255, alpha_max 0.99, t_eps 1e-4,
 * bg (0,0,0), lambda_score 0.8 (Sec. 6.1), prune_frac 0.1, prune_cap 0.5
 * (Sec. 6.2 ablation cap), change_thr 0.05 (Sec. 4.1), k0 5 (Sec. 6.1),
 * k_max 64, w_rgb 1, w_depth 0.5 (tracking loss), balance 1. */
typedef struct {
    float near_z;       /* cull when camera-frame z < near_z */
    float dilation;     /* low-pass term added to the 2D covariance diagonal */
    float alpha_min;    /* fragments with alpha below this are skipped */
    float alpha_max;    /* alpha is clamped to this value */
    float t_eps;        /* stop before a fragment when T (1 - alpha) < t_eps */
    float bg[3];        /* background colour */
    float lambda_score; /* weight of ||dL/dSigma|| in the score (Eq. 7) */
    float prune_frac;   /* fraction of active Gaussians masked per interval */
    float prune_cap;    /* cap on the pruned fraction of the reference count */
    float change_thr;   /* change-ratio threshold of the interval rule */
    int32_t k0;         /* initial pruning interval K0 */
    int32_t k_max;      /* largest interval */
    float w_rgb;        /* photometric weight of the loss (Eq. 6) */
    float w_depth;      /* geometric weight of the loss (Eq. 6) */
    int32_t balance;    /* 1: in downsampled frames (both strides >= 2)
                           gs_render_fwd reads last_idx on entry as the
                           previous iteration's per-pixel list positions and
                           pairs heavy with light pixels on the warps of a
                           tile (the workload scheduling of Sec. 5.2); any
                           content is valid and only changes scheduling,
                           never results.  0: no pairing in the forward.
                           gs_render_bwd always pairs by its last_idx. */
} gs_config;

/* 3D Gaussians (Sec. 2.1, Eq. 1), structure of arrays, float32:
 * means [n][3]; log_scales [n][3] (Sigma = Rq diag(exp(2 s)) Rq^T);
 * quats [n][4] as (w, x, y, z), need not be normalised; opacity_logit [n]
 * (opacity = sigmoid); rgb [n][3].  mask [n] or NULL: nonzero = masked out of
 * rendering by the mask-prune step (Sec. 4.1). */
typedef struct {
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logit;
    const float* rgb;
    const uint8_t* mask;
    int64_t n;
} gs_gaussians;

/* One projected 2D Gaussian (Sec. 2.1, Step 1-1), 48 bytes, 16-byte aligned.
 * Array of structures so that the compositing kernels gather one Gaussian
 * with three 16-byte loads. */
typedef struct {
    float x, y;           /* 2D mean, full-resolution pixels */
    float conic_a;        /* inverse 2D covariance [[a, b], [b, c]] */
    float conic_b;
    float conic_c;
    float opacity;        /* sigmoid(opacity_logit) */
    float depth;          /* camera-frame z */
    int32_t radius;       /* ceil(3 sqrt(lambda_max)); 0 = culled or masked */
    float r, g, b;        /* colour */
    uint32_t tiles_touched;
} gs_splat;

/* The same record with opacity, conic and colour stored as 16-bit floats
 * (bf16 or fp16, the GS_BF16 / GS_F16 precision form), 32 bytes.  Mean and
 * depth stay float32.  tiles_touched saturates at 65535. */
typedef struct {
    float x, y;
    float depth;
    int32_t radius;
    uint16_t conic_a, conic_b, conic_c, opacity;
    uint16_t r, g, b;
    uint16_t tiles_touched;
} gs_splat16;

/* Gradients of the 3D parameters, same layouts as gs_gaussians; any member
 * may be NULL to skip it. */
typedef struct {
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logit;
    float* rgb;
} gs_grads;

/* Per-Gaussian 2D gradient, 12 float32 (48 bytes) per Gaussian:
 * [0] dL/dx [1] dL/dy [2] dL/dconic_a [3] dL/dconic_b [4] dL/dconic_c
 * [5] dL/dopacity [6] dL/ddepth [7] unused [8..10] dL/drgb [11] unused. */
#define GS_GRAD2D_STRIDE 12

/* Fills *cfg with the defaults listed above. */
void gs_default_config(gs_config* cfg);

/* Library version string and the device architecture it was built for. */
const char* gs_version(void);

/* ---------------------------------------------------------------------- */
/* A-1 Projection (Sec. 2.1, Step 1-1; Eq. 1)                               */
/* ---------------------------------------------------------------------- */
/* Projects each Gaussian: camera point p = R mu + t; culled (radius 0) when
 * masked, when p.z < near_z or when the 2D covariance is singular; 2D
 * covariance J R Sigma R^T J^T + dilation I with the perspective Jacobian J
 * (x/z, y/z clamped to +-1.3 (W/2)/fx, +-1.3 (H/2)/fy); conic = its
 * inverse; radius = ceil(3 sqrt(lambda_max)); tiles_touched = number of tiles
 * of the sampled grid that the integer box [floor(x)-r, floor(x)+r] x
 * [floor(y)-r, floor(y)+r] reaches.
 * splats: [n] gs_splat (rec_dtype GS_F32) or gs_splat16 (GS_BF16, GS_F16),
 * caller-owned, fully overwritten. */
gs_status gs_project(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                     int rec_dtype, void* splats, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* A-2..A-4 Tile intersection, key duplication, 64-bit key sort, ranges     */
/* (Sec. 2.1, Step 1-2 and Step 2)                                          */
/* ---------------------------------------------------------------------- */
/* For every Gaussian with radius > 0 and every tile of its rect one key
 *     key = tile_id << 32 | float32 bits of depth,   value = Gaussian id,
 * sorted by (key, id) (the sort is a function of the keys: ties in depth
 * are ordered by id), so each tile's list is in (depth, id) order; finally
 * tile_ranges[2t], tile_ranges[2t+1] = [first, last+1) of tile t ([0,0) when
 * empty).  The rect is recomputed from the records: the tiles holding a
 * sampled in-image pixel of the Gaussian's integer box [floor(x) - r,
 * floor(x) + r] x [floor(y) - r, floor(y) + r], shrunk to the pixels whose
 * centre can reach alpha >= cfg->alpha_min: |p + 0.5 - x| <= ex with
 * ex = sqrt(2 (B + 1e-3) (Q^-1)_xx) 1.002 + 2e-3 (likewise y), Q the conic
 * and B = 64 ((op / alpha_min)^(1/64) - 1) >= ln(op / alpha_min), all in
 * float32 with correctly rounded operations (six square roots); a Gaussian
 * with op < alpha_min gets no tile.  Every fragment the compositing can
 * blend is in its tile's list; lists hold about 20 % fewer keys than with
 * the integer box alone.
 * Implementation: a counting scatter on the tile id (per-CTA tile rows and a
 * column scan) and a merge sort of each tile's (depth, id) bucket.
 * keys_out [keys_capacity] u64, vals_out [keys_capacity] u32,
 * n_keys_out: one device int64 receiving the true key count, tile_ranges
 * [2*TX*TY] u32.  If the count exceeds keys_capacity, only keys_capacity keys
 * are sorted and the device status becomes GS_ERR_CAPACITY.
 * tile_order (may be NULL): [TX*TY] u32 permutation of the tile ids, longest
 * lists first: tiles grouped by quarter octaves of their length (x = length
 * - 1 in [2^m + q 2^(m-2), 2^m + (q + 1) 2^(m-2)), q = 0..3), then lengths 1
 * and 0, ascending tile id inside a group (a function of the lists alone);
 * passing it to the compositing calls makes long tiles start first.
 * Workspace: query with workspace == NULL (depends on n, keys_capacity and
 * the tile count). */
gs_status gs_bin_sort(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats, int64_t n,
                      int64_t keys_capacity, void* workspace, size_t* workspace_bytes,
                      uint64_t* keys_out, uint32_t* vals_out, int64_t* n_keys_out,
                      uint32_t* tile_ranges, uint32_t* tile_order, gs_stream stream);

/* Key count only (the first two stages of gs_bin_sort), so that a caller can
 * size keys_capacity.  Same workspace as gs_bin_sort. */
gs_status gs_bin_count(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats, int64_t n,
                       void* workspace, size_t* workspace_bytes, int64_t* n_keys_out,
                       gs_stream stream);

/* Projection and binning in one call (a fusion of the tracking iteration):
 * gs_project followed by gs_bin_sort, with the binning's first pass (per-CTA
 * tile counts) done by the projection kernel and the scatter reusing the
 * tile rects it computed.  Outputs identical to the two calls (records in
 * `splats`, keys, values, n_keys, ranges, order).  Workspace: NULL asks for
 * its size (gs_bin_sort's plus 8 bytes per Gaussian), 256-byte aligned.
 * Grids of more than 8192 tiles run the two calls. */
gs_status gs_project_bin_sort(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                              int rec_dtype, void* splats, int64_t keys_capacity, void* workspace,
                              size_t* workspace_bytes, uint64_t* keys_out, uint32_t* vals_out,
                              int64_t* n_keys_out, uint32_t* tile_ranges, uint32_t* tile_order,
                              gs_stream stream);

/* ---------------------------------------------------------------------- */
/* A-5 Forward compositing (Sec. 2.1, Step 3; Eq. 2 and Eq. 3)              */
/* ---------------------------------------------------------------------- */
/* For each sampled pixel, front to back over its tile's sorted list: a
 * Gaussian whose integer box does not contain the pixel is skipped;
 * power = -(a dx^2 + c dy^2)/2 - b dx dy with (dx, dy) = pixel centre - mean;
 * power > 0 skipped; alpha = min(alpha_max, opacity exp(power)); alpha <
 * alpha_min skipped; if T (1 - alpha) < t_eps the pixel stops before this
 * fragment; else C += T alpha c, D += T alpha depth, T *= (1 - alpha).
 * Finally C += T bg.
 * Outputs: rgb [3][Hs][Ws], depth [Hs][Ws], t_final [Hs][Ws], last_idx
 * [Hs][Ws] (list position + 1 of the last blended fragment, relative to the
 * tile's first entry; 0 if none), n_blended [Hs][Ws] (may be NULL: number of
 * fragments blended into the pixel).  vals, tile_ranges and tile_order (may be
 * NULL: tiles in id order) come from gs_bin_sort with the same camera.
 * blend_masks (may be NULL): device uint32 array of gs_blend_mask_words
 * words that receives, per pixel and run of 32 list entries, which entries
 * the forward blended into the pixel; gs_render_bwd given the same array
 * visits only those (the same result, fewer visits) and takes the forward's
 * decisions from it instead of re-deriving them. */
gs_status gs_render_fwd(const gs_config* cfg, const gs_camera* cam, int rec_dtype,
                        const void* splats, int64_t n, const uint32_t* vals,
                        const uint32_t* tile_ranges, const uint32_t* tile_order, float* rgb,
                        float* depth, float* t_final, uint32_t* last_idx, uint32_t* n_blended,
                        uint32_t* blend_masks, gs_stream stream);

/* Words of a blend-mask array for `cam`'s tile grid and lists of up to
 * key_capacity entries (host arithmetic; 0 for an invalid camera). */
size_t gs_blend_mask_words(const gs_camera* cam, int64_t key_capacity);

/* ---------------------------------------------------------------------- */
/* A-6 Loss (Sec. 4.1, Eq. 6)                                               */
/* ---------------------------------------------------------------------- */
/* L = w_rgb mean_{3P}|C - C*| + w_depth mean_{P}|D - D*| (P = Ws*Hs; the
 * depth term only where D* != 0), and dL/drgb, dL/ddepth with sign(0) = 0.
 * target_rgb [3][Hs][Ws], target_depth [Hs][Ws] at the sampled pixels.
 * loss_out: one device double (overwritten).  d_rgb, d_depth: outputs. */
gs_status gs_loss_l1(const gs_config* cfg, const gs_camera* cam, const float* rgb,
                     const float* depth, const float* target_rgb, const float* target_depth,
                     float* d_rgb, float* d_depth, double* loss_out, gs_stream stream);

/* Forward compositing and the loss in one launch (a fusion of the tracking
 * iteration; the paper's Sec. 5 pipeline feeds the loss straight from the
 * rendering engines): gs_render_fwd's outputs, plus gs_loss_l1's d_rgb and
 * d_depth computed by the thread that finishes each pixel (identical
 * values), and loss_out (device double, overwritten: the call zeroes it
 * first) summed per warp in float32 and across warps in float64 (equal to
 * gs_loss_l1's to float32 rounding of the partial sums). */
gs_status gs_render_fwd_loss(const gs_config* cfg, const gs_camera* cam, int rec_dtype,
                             const void* splats, int64_t n, const uint32_t* vals,
                             const uint32_t* tile_ranges, const uint32_t* tile_order, float* rgb,
                             float* depth, float* t_final, uint32_t* last_idx,
                             uint32_t* n_blended, uint32_t* blend_masks, const float* target_rgb,
                             const float* target_depth, float* d_rgb, float* d_depth,
                             double* loss_out, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* A-7 Backward compositing (Sec. 2.2, Step 4; Eq. 4 and Eq. 5)             */
/* ---------------------------------------------------------------------- */
/* Reverse traversal of each pixel's blended fragments: T_k is recovered from
 * t_final by dividing by (1 - alpha_k) (Eq. 5); dL/dalpha_k =
 * T_k (c_k - A_k) . dL/dC + T_k (d_k - A^D_k) dL/dD with the normalised
 * suffix A_k = sum_{n>k} (T_n/T_{k+1}) alpha_n c_n + (T_final/T_{k+1}) bg
 * (Eq. 3 differentiated; the printed Eq. 4 omits T_k and the normalisation);
 * then through alpha = opacity exp(power) to opacity, conic and 2D mean
 * unless alpha was clamped.  Per-fragment gradients are summed per Gaussian
 * inside each warp; with blend_masks (pixel-parallel frames) each warp's
 * sums go to grad2d with one global atomic per (Gaussian, warp, field),
 * otherwise they are summed per tile in shared memory first (one atomic per
 * (Gaussian, tile, field)).
 * grad2d [n][12] float (GS_GRAD2D_STRIDE layout): zeroed by this call.
 * mode GS_TRACK skips dL/dopacity and dL/drgb (not needed for the pose).
 * If grads, pose_grad6 or score_terms is non-NULL, gs_project_bwd runs as
 * well on the same stream (same workspace).  blend_masks (may be NULL) must
 * come from the forward call that produced t_final and last_idx. */
gs_status gs_render_bwd(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                        int rec_dtype, const void* splats, const uint32_t* vals,
                        const uint32_t* tile_ranges, const uint32_t* tile_order,
                        const float* t_final, const uint32_t* last_idx,
                        const uint32_t* blend_masks, const float* d_rgb, const float* d_depth,
                        int mode, float* grad2d, gs_grads* grads, double* pose_grad6,
                        float* score_terms, void* workspace, size_t* workspace_bytes,
                        gs_stream stream);

/* ---------------------------------------------------------------------- */
/* A-8 Backward projection and camera pose (Sec. 2.2, Step 5)               */
/* ---------------------------------------------------------------------- */
/* Chains grad2d back through the projection of each Gaussian.
 * grads (GS_MAP): 3D gradients w.r.t. means, log_scales, unnormalised quats,
 *   opacity_logit and rgb (members may be NULL).
 * pose_grad6: one device double[6], dL/dxi for the left perturbation
 *   T_cw <- exp(xi^) T_cw, xi = (rho, phi) at 0:
 *   dL/drho = sum_k dL/dp_k,
 *   dL/dphi = sum_k p_k x dL/dp_k + (<G_k, [e_i]x S_k - S_k [e_i]x>)_i,
 *   with p_k the camera point, S_k its camera-frame covariance and G_k =
 *   dL/dS_k.  Per-Gaussian terms in float32, warp sums in float32, block
 *   and cross-block sums as float32 pairs (hi + lo, error-free two-sums:
 *   about 48 significant bits) in a fixed order, returned as float64.
 * score_terms [n][2] float: (||dL/dmu||_2, ||dL/dSigma||_F) for Eq. 7.
 * Any of the three outputs may be NULL. */
gs_status gs_project_bwd(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                         const float* grad2d, gs_grads* grads, double* pose_grad6,
                         float* score_terms, void* workspace, size_t* workspace_bytes,
                         gs_stream stream);

/* Variant of gs_project_bwd for callers that cannot allocate device memory
 * (no counterpart in the paper; it exists for integrations such as a
 * real-time tracking thread that runs under a fixed memory budget, or a host
 * framework that owns every allocation and offers the library no allocator).
 * Same arguments and results as gs_project_bwd, minus the workspace: the
 * scratch (per-block pose partials and a ticket) lives in a static device
 * array of GS_NOALLOC_SCRATCH_BYTES (768 KiB: 786,688 bytes) that every device which loads
 * the library holds until the process exits.  n is limited to
 * GS_NOALLOC_MAX_GAUSSIANS; a larger n returns GS_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset the
 * entry point must not be called again, and it serves the device's primary
 * context only.  All
 * calls share the one array: calls that overlap on the GPU (different
 * streams, or different host threads, without ordering) race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
#define GS_NOALLOC_MAX_GAUSSIANS 4194304
#define GS_NOALLOC_SCRATCH_BYTES (((GS_NOALLOC_MAX_GAUSSIANS / 256) * 48 + 511) / 256 * 256)
gs_status gs_project_bwd_noalloc(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                 const float* grad2d, gs_grads* grads, double* pose_grad6,
                                 float* score_terms, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* A-9 Gradient-reuse pruning (Sec. 4.1, Eq. 7)                              */
/* ---------------------------------------------------------------------- */
/* Mask-prune state machine of one pruning interval of K iterations.
 * iter_in_interval == 0 (selection): score_k = t_mu + lambda_score * t_sigma
 *   in float32 (product rounded, then sum rounded); among Gaussians with
 *   mask_inout[k] == 0 the m = min(floor(prune_frac * n_active), max_select)
 *   smallest in (score, id) order get mask_inout[k] = 1.
 * iter_in_interval == *k_inout (the (K+1)-th iteration, removal):
 *   compact_map_out[k] = new index of each unmasked Gaussian in id order, or
 *   0xFFFFFFFF for a masked one; *n_kept_out (device int64) = kept count;
 *   *k_inout (host) becomes the next interval: max(1, K/2) if change_ratio >
 *   change_thr, else min(2K, k_max).
 * Any other iter_in_interval: nothing to do.
 * score_terms [n][2] float (from gs_project_bwd).  max_select: host value
 * (the caller's remaining cap, e.g. prune_cap * n_ref - already pruned). */
gs_status gs_prune(const gs_config* cfg, const float* score_terms, int64_t n,
                   uint8_t* mask_inout, int iter_in_interval, int* k_inout,
                   float change_ratio, int64_t max_select, uint32_t* compact_map_out,
                   int64_t* n_kept_out, void* workspace, size_t* workspace_bytes,
                   gs_stream stream);

/* Length of the next pruning interval (Sec. 4.1): after an interval of K
 * iterations whose tile-Gaussian intersections changed by change_ratio,
 * max(1, floor(K / 2)) if change_ratio > cfg->change_thr, else
 * min(2 K, cfg->k_max) (the current K playing the paper's K0).  Host, pure;
 * the rule gs_prune applies at the removal iteration.  Returns 1 for a NULL
 * cfg or K < 1. */
int32_t gs_next_interval(const gs_config* cfg, int32_t K, float change_ratio);

/* Change ratio of tile-Gaussian intersections between two binnings of the
 * same n Gaussians on the same tile grid (Sec. 4.1): |A xor B| / max(1, |A|)
 * over the sets of (tile, Gaussian) pairs.  Each Gaussian's tiles form the
 * rect of its record (the rect of gs_bin_sort, with cfg->alpha_min), so
 * |A xor B| = sum_k |rect_a(k)| +
 * |rect_b(k)| - 2 |rect_a(k) & rect_b(k)|.  For the mask-prune rule both
 * binnings should include the masked Gaussians (project with mask = NULL).
 * ratio_out: one device float. */
gs_status gs_change_ratio(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats_a,
                          const void* splats_b, int64_t n, void* workspace,
                          size_t* workspace_bytes, float* ratio_out, gs_stream stream);

/* Gathers the rows of a float array [n][width] through a compaction map
 * (0xFFFFFFFF = dropped): dst[map[k]] = src[k].  dst has *n_kept rows. */
gs_status gs_compact(const float* src, int64_t n, int32_t width, const uint32_t* compact_map,
                     float* dst, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* A-10 Keyframe-driven dynamic downsampling (Sec. 4.2)                      */
/* ---------------------------------------------------------------------- */
/* Schedule (host, pure): keyframe -> (1,1); non-keyframe n after keyframe k
 * -> resolution min(R0/16 m^(n-k-1), R0/4) as a pixel count, realised by the
 * strides 16 -> (4,4), 8 -> (4,2), 4 -> (2,2).  m must be a power of two.
 * Writes *sx, *sy (host).  If target_full is non-NULL also gathers
 * target_out[c][j][i] = target_full[c][sy j][sx i] for `channels` planes of
 * W x H (device). */
gs_status gs_downsample(int64_t frame_idx, int64_t last_kf_idx, int is_keyframe, int m,
                        int32_t* sx, int32_t* sy, const float* target_full, int32_t channels,
                        int32_t W, int32_t H, float* target_out, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* Camera pose step (tracking, Sec. 2.2 Step 5: dL/dP drives the pose)       */
/* ---------------------------------------------------------------------- */
/* One Adam step on the 6-vector xi = (rho, phi) followed by the left update
 * T_cw <- exp(xi^) T_cw (SE(3) exponential map), entirely on the device:
 *   g = pose_grad6 (device double[6]); adam (device float[13]) = m[6], v[6],
 *   step count; m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   xi_i = -lr_i mhat_i / (sqrt(vhat_i) + eps) with lr_i = lr_trans for rho
 *   and lr_rot for phi.  pose (device float[12], R row-major then t) is
 *   updated in place.  adam must start zeroed.  The paper's Pose Computing
 *   Unit (Sec. 5.1) does not fix the optimizer; Adam is this library's. */
gs_status gs_pose_update(float* pose, const double* pose_grad6, float* adam, float lr_trans,
                         float lr_rot, float beta1, float beta2, float eps, gs_stream stream);

/* The pose step of gs_pose_update, as an argument of gs_project_bwd_step. */
typedef struct {
    float* pose;    /* device float[12], updated in place */
    float* adam;    /* device float[13]: m[6], v[6], step count (starts zeroed) */
    float lr_trans; /* learning rate of rho */
    float lr_rot;   /* learning rate of phi */
    float beta1, beta2, eps;
} gs_pose_step;

/* gs_project_bwd with the pose step fused into its last block: the block that
 * completes the pose-gradient reduction (pose_grad6,
 * required here) applies gs_pose_update's Adam step and SE(3) update with
 * `step` (same arithmetic, one launch fewer per tracking iteration).  Every
 * block reads the pose before the last block updates it, so a camera whose
 * `pose` is step->pose sees the old pose throughout the call.  step NULL:
 * plain gs_project_bwd.  Workspace as gs_project_bwd. */
gs_status gs_project_bwd_step(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                              const float* grad2d, gs_grads* grads, double* pose_grad6,
                              float* score_terms, const gs_pose_step* step, void* workspace,
                              size_t* workspace_bytes, gs_stream stream);

/* ---------------------------------------------------------------------- */
/* Multi-session waves (serving form)                                       */
/* ---------------------------------------------------------------------- */
/* One session's fused tracking iteration inside a wave: everything
 * gs_project_bin_sort + gs_render_fwd_loss + gs_render_bwd(GS_TRACK) +
 * gs_project_bwd_step take for that session, with the same meaning and
 * layouts.  All pointers are device memory owned by the caller and must stay
 * valid until the wave's work on `stream` has completed.  The paper runs
 * many frames through one rasterizer (its frame-level programming interface,
 * Sec. 5.5); a wave is that interface for many concurrent sessions. */
typedef struct {
    gs_camera cam;            /* the session's camera; cam.pose is read on the device */
    gs_gaussians g;           /* the session's map; g.n >= 1 */
    float* splats;            /* float32 records [g.n][12] (GS_F32 layout) */
    int64_t keys_capacity;    /* in [1, 2^30) */
    void* bin_workspace;      /* gs_project_bin_sort's workspace (256-byte aligned) */
    size_t bin_workspace_bytes;
    uint64_t* keys;           /* [keys_capacity] */
    uint32_t* vals;           /* [keys_capacity] */
    int64_t* n_keys;          /* device int64 */
    uint32_t* tile_ranges;    /* [T][2] */
    uint32_t* tile_order;     /* [T] */
    float* rgb;               /* [3][Hs][Ws] */
    float* depth;             /* [Hs][Ws] */
    float* t_final;           /* [Hs][Ws] */
    uint32_t* last_idx;       /* [Hs][Ws] */
    uint32_t* n_blended;      /* [Hs][Ws] or NULL */
    uint32_t* blend_masks;    /* gs_blend_mask_words(cam, keys_capacity) words, or NULL */
    const float* target_rgb;  /* [3][Hs][Ws] */
    const float* target_depth;/* [Hs][Ws] (0 = no depth measurement) */
    float* d_rgb;             /* [3][Hs][Ws] */
    float* d_depth;           /* [Hs][Ws] */
    double* loss;             /* device double */
    float* grad2d;            /* [g.n][12], 16-byte aligned */
    double* pose_grad6;       /* device double[6] */
    float* score_terms;       /* [g.n][2] or NULL */
    void* bwd_workspace;      /* gs_project_bwd's workspace */
    size_t bwd_workspace_bytes;
    gs_pose_step step;        /* the pose step applied after the reduction */
} gs_track_job;

/* Largest number of sessions in one wave. */
#define GS_WAVE_MAX 32

/* One tracking iteration of every job (Sec. 2.1 Steps 1-3, Sec. 2.2 Steps
 * 4-5, Sec. 4.1 Eq. 6), each with the results of its own fused iteration,
 * in launches whose grids span all jobs: projection with the binning's tile
 * counts, the column scan with the tile scan and order, the key scatter, the
 * bucket sort, the forward compositing with the loss, the backward
 * compositing and the backward projection with the pose step -- one launch
 * each (the compositing ones once per kernel form present: full-resolution
 * tiles, strided tiles of up to 32 or 64 sampled pixels).  Each CTA finds its
 * job and its block inside the job from the wave's descriptor table, which
 * travels in the launch's parameter space (no device allocation, no copy).
 * jobs: host array of n_jobs (1..GS_WAVE_MAX) descriptors; the jobs' buffers
 * must not overlap.  Limits: float32 records, at most 8192 tiles per job.
 * Errors: GS_ERR_INVALID_ARG / GS_ERR_WORKSPACE (naming the job) before
 * anything is enqueued; key-capacity overflow sets the device status word as
 * in gs_bin_sort. */
gs_status gs_track_wave(const gs_config* cfg, const gs_track_job* jobs, int32_t n_jobs, gs_stream stream);

/* Mapping step: Adam over up to GS_ADAM_MAX_TENSORS float32 arrays in one
 * launch (the map update fed by the backward, Sec. 2.2 Step 5 / Sec. 5.4;
 * the optimizer itself is not fixed by the paper).  params[t], grads[t],
 * m[t], v[t] are device arrays of counts[t] elements (host arrays of
 * pointers and counts); m and v start zeroed.  state: device float[2] that
 * starts zeroed; state[0] is the step count, advanced by the launch itself so
 * a CUDA graph that replays the step stays correct. */
#define GS_ADAM_MAX_TENSORS 8
gs_status gs_adam(int n_tensors, float* const* params, const float* const* grads, float* const* m,
                  float* const* v, const int64_t* counts, float lr, float beta1, float beta2,
                  float eps, float* state, gs_stream stream);

/* The map's Adam step of a mapping iteration, for gs_project_bwd_adam:
 * moments of the five parameter arrays in gs_gaussians order (means,
 * log_scales, quats, opacity_logit, rgb; each the size of its parameter
 * array, starting zeroed) and the step state of gs_adam. */
typedef struct {
    float* m[5];
    float* v[5];
    float lr, beta1, beta2, eps;
    float* state;   /* device float[2]: step count, then a ticket word (starts zeroed) */
} gs_map_adam;

/* gs_project_bwd (Sec. 2.2 Step 5, mapping) with gs_adam's step fused into
 * it: each Gaussian's gradients are formed and applied to its parameters in
 * the same thread, with gs_adam's arithmetic (the same bits), and the step
 * count advances once.  g's five parameter arrays are updated in place (the
 * const of gs_gaussians aside); grads (optional, any member NULL) still
 * receive the gradients, score_terms (optional) the Eq. 7 terms.  No
 * workspace; no pose gradient (tracking uses gs_project_bwd_step).  The
 * paper's Preprocessing Engines feed the map update from the same pass
 * (Sec. 5.4). */
gs_status gs_project_bwd_adam(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                              const float* grad2d, const gs_map_adam* adam, gs_grads* grads, float* score_terms,
                              gs_stream stream);

/* ---------------------------------------------------------------------- */
/* Status (the frame-level status query of Sec. 5.5, as a device word)      */
/* ---------------------------------------------------------------------- */
/* Returns the current device status word of the calling thread's current
 * device (GS_OK if no device-side condition was raised).  blocking != 0
 * synchronises `stream` first; otherwise *state (host, may be NULL) is set to
 * GS_EXECUTING while work on `stream` is pending and the word read may be
 * stale.  gs_status_reset clears the word (enqueued on `stream`). */
gs_status gs_status_poll(gs_stream stream, int blocking, int* state);
gs_status gs_status_reset(gs_stream stream);

/* ---------------------------------------------------------------------- */
/* Measurement probe (not a step of the method)                             */
/* ---------------------------------------------------------------------- */
/* Global float32 reduction throughput, the operation that merges the
 * per-(Gaussian, tile) gradients into per-Gaussian arrays in the backward
 * (Sec. 2.2 Step 4): thread t of n_threads adds 1.0f to dst[t % n_dst]
 * per_thread times with red.global.add.f32 (n_dst >= n_threads: distinct
 * addresses; small n_dst: contended).  dst: device float[n_dst], owned by the
 * caller, accumulated into (not cleared).  Enqueued on `stream`; the caller
 * times it.  GS_ERR_INVALID_ARG for a NULL dst or a non-positive count. */
gs_status gs_probe_red_f32(float* dst, int64_t n_dst, int64_t n_threads, int32_t per_thread, gs_stream stream);

/* FP32 fused multiply-add throughput, the peak the compositing kernels'
 * per-fragment arithmetic (Sec. 2.1 Eq. 2-3, Sec. 2.2 Eq. 4-5) is measured
 * against: each of n_threads threads runs 8 independent chains of `iters`
 * FMAs (16 FLOP per iteration) and writes out[t] = 28 + 8 iters (exact for
 * iters < 2^21).  out: device float[n_threads], owned by the caller.
 * Enqueued on `stream`; the caller times it.  GS_ERR_INVALID_ARG for a NULL
 * out or a non-positive count. */
gs_status gs_probe_fma_f32(float* out, int64_t n_threads, int32_t iters, gs_stream stream);

/* Thread-local message of the last failing call on this thread. */
const char* gs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
