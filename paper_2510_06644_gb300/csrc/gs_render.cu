// A-5 forward compositing (Sec. 2.1, Step 3: Eq. 2, Eq. 3), A-6 loss
// (Sec. 4.1, Eq. 6) and A-7 backward compositing (Sec. 2.2, Step 4: Eq. 4,
// Eq. 5) on sm_103a.
//
// One CTA per tile, one pixel per thread (256 threads for the 16x16 tiles
// of a full-resolution image, fewer for the smaller sampled tiles of a
// downsampled one, at least one warp); CTAs are
// issued in the heavy-first tile order produced by the binning, so the block
// scheduler starts the longest lists first (the GPU counterpart of the
// paper's subtile streaming, Sec. 5.2).  The 8 warps cover 8x4 pixel blocks.
// The tile's sorted list is staged through shared memory in batches of 256
// records (one 48-byte gather per thread).  Each warp then builds a 256-bit
// mask of the staged Gaussians whose integer box meets its 8x4 block (8
// box tests and 8 ballots per lane) and visits only those.
//
// The backward walks each pixel's blended fragments in reverse from the
// forward's last position, recovering T_k by division (Eq. 5), and merges the
// per-pixel gradients of each Gaussian across the warp with a reduce-scatter
// butterfly (each level halves the fields a lane carries: 9 shuffles for 6
// fields, 16 for 10, instead of 5 per field), after which 8 or 16 lanes add
// distinct fields into the tile's shared-memory accumulators at once; one
// global atomic per (Gaussian, tile, field) follows.  This replaces the
// paper's Gradient Merging Unit (Sec. 5.3).
#include "gs_internal.cuh"

namespace gs {

#define R_THREADS 256            // largest CTA (16x16 tile)
#define R_BATCH 256              // entries staged per batch, whatever the CTA size
#define R_MASKW (R_BATCH / 32)

struct StagedSplat {
    float4 a;   // x, y, conic_a, conic_b
    float4 b;   // conic_c, opacity, depth, unused
    float4 c;   // r, g, b, unused
    int4 box;   // full-resolution integer box x0, x1, y0, y1
};

struct PixelMap {
    int i, j;        // sampled pixel
    bool inside;
    int px, py;      // full-resolution pixel
    int wx0, wx1, wy0, wy1;  // full-resolution extent of this warp's 8x4 block
};

// Threads serving one tile: tw * th, at least one warp.  Warps cover BW x BH
// pixel blocks (8x4, or 4x8 for 4-wide tiles).
__host__ __device__ inline int tile_threads(const Grid& g) {
    const int t = g.tw * g.th;
    return t < 32 ? 32 : t;
}

// Every CTA has R_THREADS threads and serves R_THREADS / TT tiles (TT =
// tile_threads): a full-resolution 16x16 tile takes the whole CTA, the
// smaller sampled tiles of a downsampled frame take groups of 2 or 1 warps,
// each group with its own slice of the staging buffer and its own named
// barrier, so a CTA always holds 8 warps.
struct Group {
    int TT;     // threads of the group
    int gi;     // group index in the CTA
    int lt;     // thread index in the group
    int B;      // entries staged per batch
    int tile;   // tile served, -1 if none
};

__device__ __forceinline__ Group make_group(const Grid& g, const uint32_t* order) {
    Group G;
    G.TT = tile_threads(g);
    const int gpc = R_THREADS / G.TT;
    G.gi = threadIdx.x / G.TT;
    G.lt = threadIdx.x % G.TT;
    G.B = R_BATCH / gpc;
    const int t = blockIdx.x * gpc + G.gi;
    G.tile = t < g.TX * g.TY ? (order ? (int)__ldg(order + t) : t) : -1;
    return G;
}

__device__ __forceinline__ void group_sync(const Group& G) {
    if (G.TT == R_THREADS) __syncthreads();
    else if (G.TT == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + G.gi), "r"(G.TT) : "memory");
}

// Number of threads of the group with `pred` set (also a group barrier).
__device__ __forceinline__ int group_count(const Group& G, bool pred) {
    if (G.TT == R_THREADS) return __syncthreads_count(pred);
    if (G.TT == 32) return __popc(__ballot_sync(0xffffffffu, pred));
    int r;
    asm volatile("{ .reg .pred p; setp.ne.u32 p, %3, 0; bar.red.popc.u32 %0, %1, %2, p; }"
                 : "=r"(r) : "r"(1 + G.gi), "r"(G.TT), "r"((unsigned)pred) : "memory");
    return r;
}

__device__ __forceinline__ PixelMap map_pixel(const Grid& g, int tile, int lt) {
    PixelMap m;
    const int tx = tile % g.TX, ty = tile / g.TX;
    const int lane = lt & 31, w = lt >> 5;
    const int BW = g.tw < 8 ? g.tw : 8, BH = 32 / BW, WX = g.tw / BW;
    const int bx = (w % WX) * BW, by = (w / WX) * BH;
    const int lx = lane % BW, ly = lane / BW;
    m.i = tx * g.tw + bx + lx;
    m.j = ty * g.th + by + ly;
    m.inside = by + ly < g.th && m.i < g.Ws && m.j < g.Hs;
    m.px = m.i * g.sx;
    m.py = m.j * g.sy;
    m.wx0 = (tx * g.tw + bx) * g.sx;
    m.wx1 = (tx * g.tw + bx + BW - 1) * g.sx;
    m.wy0 = (ty * g.th + by) * g.sy;
    m.wy1 = (ty * g.th + by + BH - 1) * g.sy;
    return m;
}

// Pixel box of a staged Gaussian: its integer 3-sigma box (the definition of
// which pixels see it), shrunk to the pixels whose centre lies in the
// axis-aligned bounding box of the ellipse where alpha can reach alpha_min,
//     d^T Q d <= 2 ln(opacity / alpha_min),  half extents
//     sqrt(2 ln(opacity / alpha_min) (Q^-1)_xx), ... (Q = conic),
// widened against rounding (1e-4 added to the log threshold, a relative
// 1e-3 and 1e-3 px on the extent).  Every pixel it drops would fail the alpha
// test, so the image and gradients are unchanged; the compositing loops just
// visit fewer entries.  A Gaussian whose opacity is clearly below alpha_min
// gets an empty box.  Forward and backward use the same box.
__device__ __forceinline__ int4 pixel_box(const Splat& v, float alpha_min) {
    const int xi = pix_floor(v.x), yi = pix_floor(v.y), r = v.radius;
    int4 box = make_int4(xi - r, xi + r, yi - r, yi + r);
    const float det = v.ca * v.cc - v.cb * v.cb;
    if (!(det > 0.f) || !(v.op > 0.f) || !(alpha_min > 0.f)) return box;
    const float thr = logf(v.op / alpha_min);
    if (thr < -1e-4f) return make_int4(1, 0, 1, 0);  // empty: opacity < alpha_min
    const float t2 = 2.f * (fmaxf(thr, 0.f) + 1e-4f);
    const float ex = sqrtf(t2 * v.cc / det) * 1.001f + 1e-3f;
    const float ey = sqrtf(t2 * v.ca / det) * 1.001f + 1e-3f;
    if (!(ex < 1e8f) || !(ey < 1e8f)) return box;
    // pixel p qualifies when |p + 0.5 - x| <= ex
    box.x = max(box.x, (int)ceilf(v.x - ex - 0.5f));
    box.y = min(box.y, (int)floorf(v.x + ex - 0.5f));
    box.z = max(box.z, (int)ceilf(v.y - ey - 0.5f));
    box.w = min(box.w, (int)floorf(v.y + ey - 0.5f));
    return box;
}

template <int DT>
__device__ __forceinline__ void stage(const void* splats, uint32_t gid, float alpha_min, StagedSplat& s) {
    const Splat v = load_splat<DT>(splats, gid);
    s.a = make_float4(v.x, v.y, v.ca, v.cb);
    s.b = make_float4(v.cc, v.op, v.depth, 0.f);
    s.c = make_float4(v.r, v.g, v.b, 0.f);
    s.box = pixel_box(v, alpha_min);
}

// Bit e of word q set when staged entry 32q + e (below `limit`) meets the
// warp's block; words at or beyond `words` are cleared.
__device__ __forceinline__ void warp_masks(const StagedSplat* sp, int limit, int words, const PixelMap& m,
                                           unsigned* mask) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < R_MASKW; ++q) {
        const int e = q * 32 + lane;
        bool hit = false;
        if (q < words && e < limit) {
            const int4 box = sp[e].box;
            hit = !(box.y < m.wx0 || box.x > m.wx1 || box.w < m.wy0 || box.z > m.wy1);
        }
        mask[q] = __ballot_sync(0xffffffffu, hit);
    }
}

template <int DT>
__global__ void __launch_bounds__(R_THREADS) k_render_fwd(gs_config cfg, Grid g, const void* __restrict__ splats,
                                                          const uint32_t* __restrict__ vals,
                                                          const uint32_t* __restrict__ ranges,
                                                          const uint32_t* __restrict__ order,
                                                          float* __restrict__ out_rgb, float* __restrict__ out_depth,
                                                          float* __restrict__ out_t, uint32_t* __restrict__ out_last,
                                                          uint32_t* __restrict__ out_nb) {
    __shared__ StagedSplat sp_all[R_BATCH];
    const Group G = make_group(g, order);
    if (G.tile < 0) return;
    StagedSplat* sp = sp_all + G.gi * G.B;
    const int tile = G.tile;
    const PixelMap m = map_pixel(g, tile, G.lt);
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const float pxc = (float)m.px + 0.5f, pyc = (float)m.py + 0.5f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    uint32_t last = 0, nb = 0;
    bool done = !m.inside;
    const int words = G.B / 32;
    for (uint32_t b = start; b < end; b += G.B) {
        if (group_count(G, done) == G.TT) break;
        const int n_in = (int)min((uint32_t)G.B, end - b);
        for (int e = G.lt; e < n_in; e += G.TT) stage<DT>(splats, __ldg(vals + b + e), cfg.alpha_min, sp[e]);
        group_sync(G);
        if (!__all_sync(0xffffffffu, done)) {
            unsigned mask[R_MASKW];
            warp_masks(sp, n_in, words, m, mask);
#pragma unroll 1
            for (int q = 0; q < words; ++q) {
                unsigned mq = mask[q];
                while (mq) {
                    const int e = q * 32 + __ffs(mq) - 1;
                    mq &= mq - 1u;
                    const int4 box = sp[e].box;
                    if (done || m.px < box.x || m.px > box.y || m.py < box.z || m.py > box.w) continue;
                    const float4 A = sp[e].a;
                    const float dx = pxc - A.x, dy = pyc - A.y;
                    const float4 B = sp[e].b;
                    const float power = -0.5f * (A.z * dx * dx + B.x * dy * dy) - A.w * dx * dy;
                    if (power > 0.f) continue;
                    const float alpha = fminf(cfg.alpha_max, B.y * __expf(power));
                    if (alpha < cfg.alpha_min) continue;
                    const float Tn = T * (1.f - alpha);
                    if (Tn < cfg.t_eps) { done = true; continue; }
                    const float w = alpha * T;
                    const float4 Cc = sp[e].c;
                    C0 += w * Cc.x; C1 += w * Cc.y; C2 += w * Cc.z;
                    D += w * B.z;
                    T = Tn;
                    ++nb;
                    last = b - start + (uint32_t)e + 1u;
                }
                if (__all_sync(0xffffffffu, done)) break;
            }
        }
        group_sync(G);
    }
    if (m.inside) {
        const size_t P = (size_t)g.Ws * g.Hs;
        const size_t pix = (size_t)m.j * g.Ws + m.i;
        out_rgb[pix] = C0 + T * cfg.bg[0];
        out_rgb[P + pix] = C1 + T * cfg.bg[1];
        out_rgb[2 * P + pix] = C2 + T * cfg.bg[2];
        out_depth[pix] = D;
        out_t[pix] = T;
        out_last[pix] = last;
        if (out_nb) out_nb[pix] = nb;
    }
}

// ---------------------------------------------------------------------------
// Loss (Eq. 6) with L1 residuals
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_loss_l1(gs_config cfg, int64_t P, const float* __restrict__ rgb,
                                                 const float* __restrict__ depth, const float* __restrict__ trgb,
                                                 const float* __restrict__ tdepth, float* __restrict__ d_rgb,
                                                 float* __restrict__ d_depth, double* __restrict__ loss) {
    __shared__ float s_w[8];
    const float inv3 = 1.f / (3.f * (float)P), inv1 = 1.f / (float)P;
    float acc = 0.f;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = rgb[c * P + q] - trgb[c * P + q];
            acc += cfg.w_rgb * fabsf(r) * inv3;
            d_rgb[c * P + q] = cfg.w_rgb * (r > 0.f ? inv3 : (r < 0.f ? -inv3 : 0.f));
        }
        const float td = tdepth[q];
        float gd = 0.f;
        if (td != 0.f) {
            const float r = depth[q] - td;
            acc += cfg.w_depth * fabsf(r) * inv1;
            gd = cfg.w_depth * (r > 0.f ? inv1 : (r < 0.f ? -inv1 : 0.f));
        }
        d_depth[q] = gd;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)s_w[w];
        atomicAdd(loss, s);
    }
}

// ---------------------------------------------------------------------------
// Backward compositing
// ---------------------------------------------------------------------------
// Slots merged per fragment: GS_TRACK 8 (du, dv, dA, dB, dC, dd, -, -),
// GS_MAP 16 (du, dv, dA, dB, dC, dop, dd, dr, dg, db, -...).
template <int MODE>
struct Slots {
    static constexpr int N = MODE == GS_MAP ? 16 : 8;
    static constexpr int LOG = MODE == GS_MAP ? 4 : 3;
};

// grad2d column of a slot (-1 = padding).
template <int MODE>
__device__ __forceinline__ int slot_col(int s) {
    if (MODE == GS_MAP) return s < 7 ? s : (s < 10 ? s + 1 : -1);  // du dv dA dB dC dop dd | dr dg db
    return s < 5 ? s : (s == 5 ? 6 : -1);                             // du dv dA dB dC | dd
}

// Reduce-scatter of N values across the warp.  On return lane l holds the
// warp total of slot (l >> (5 - LOG)) when (l & ((1 << (5 - LOG)) - 1)) == 0.
template <int N, int LOG>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[N]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int lvl = 0; lvl < LOG; ++lvl) {
        const int off = 16 >> lvl;
        const int half = N >> (lvl + 1);
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            if (i < half) {
                const float send = up ? v[i] : v[i + half];
                const float keep = up ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
    }
    float x = v[0];
#pragma unroll
    for (int off = 16 >> LOG; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

template <int DT, int MODE>
__global__ void __launch_bounds__(R_THREADS) k_render_bwd(gs_config cfg, Grid g, const void* __restrict__ splats,
                                                          const uint32_t* __restrict__ vals,
                                                          const uint32_t* __restrict__ ranges,
                                                          const uint32_t* __restrict__ order,
                                                          const float* __restrict__ t_final,
                                                          const uint32_t* __restrict__ last_idx,
                                                          const float* __restrict__ d_rgb,
                                                          const float* __restrict__ d_depth,
                                                          float* __restrict__ grad2d) {
    constexpr int NS = Slots<MODE>::N;
    constexpr int LOG = Slots<MODE>::LOG;
    constexpr int SHIFT = 5 - LOG;  // lanes per slot = 1 << SHIFT
    __shared__ StagedSplat sp_all[R_BATCH];
    __shared__ uint32_t sid_all[R_BATCH];
    __shared__ float acc_all[R_BATCH][NS];
    __shared__ uint32_t s_max_all[R_THREADS / 32];
    const Group G = make_group(g, order);
    if (G.tile < 0) return;
    StagedSplat* sp = sp_all + G.gi * G.B;
    uint32_t* sid = sid_all + G.gi * G.B;
    float(*acc)[NS] = acc_all + G.gi * G.B;
    uint32_t& s_max = s_max_all[G.gi];
    const int tile = G.tile;
    const PixelMap m = map_pixel(g, tile, G.lt);
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const float pxc = (float)m.px + 0.5f, pyc = (float)m.py + 0.5f;
    const int lane = threadIdx.x & 31;
    float T = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f;
    uint32_t last = 0;
    if (m.inside) {
        const size_t P = (size_t)g.Ws * g.Hs;
        const size_t pix = (size_t)m.j * g.Ws + m.i;
        T = t_final[pix];
        last = last_idx[pix];
        gC0 = d_rgb[pix];
        gC1 = d_rgb[P + pix];
        gC2 = d_rgb[2 * P + pix];
        gD = d_depth[pix];
    }
    // a last_idx beyond the tile's list (inconsistent inputs) is clamped
    last = min(last, end - start);
    // normalised suffix sums (background enters with weight T_final)
    float A0 = cfg.bg[0], A1 = cfg.bg[1], A2 = cfg.bg[2], AD = 0.f;
    uint32_t wlast = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    if (G.lt == 0) s_max = 0;
    group_sync(G);
    if (lane == 0) atomicMax(&s_max, wlast);
    group_sync(G);
    const uint32_t end_eff = start + s_max;
    const int words = G.B / 32;
    for (uint32_t hi = end_eff; hi > start;) {
        const uint32_t lo = hi - start > (uint32_t)G.B ? hi - G.B : start;
        const int n_in = (int)(hi - lo);
        for (int e = G.lt; e < n_in; e += G.TT) {
            const uint32_t gid = __ldg(vals + lo + e);
            sid[e] = gid;
            stage<DT>(splats, gid, cfg.alpha_min, sp[e]);
        }
        for (int q = G.lt; q < G.B * NS; q += G.TT) (&acc[0][0])[q] = 0.f;
        group_sync(G);
        const uint32_t base_pos = lo - start;
        // entries at or beyond the warp's furthest blended position are skipped
        const int wlimit = (int)min((uint32_t)n_in, wlast > base_pos ? wlast - base_pos : 0u);
        unsigned mask[R_MASKW];
        warp_masks(sp, wlimit, words, m, mask);
#pragma unroll 1
        for (int q = words - 1; q >= 0; --q) {
            unsigned mq = mask[q];
            while (mq) {
                const int bit = 31 - __clz(mq);
                const int e = q * 32 + bit;
                mq &= ~(1u << bit);
                const int4 box = sp[e].box;
                bool contrib = (base_pos + (uint32_t)e) < last && m.px >= box.x && m.px <= box.y &&
                               m.py >= box.z && m.py <= box.w;
                float f[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) f[s] = 0.f;
                if (contrib) {
                    const float4 A = sp[e].a;
                    const float4 B = sp[e].b;
                    const float dx = pxc - A.x, dy = pyc - A.y;
                    const float power = -0.5f * (A.z * dx * dx + B.x * dy * dy) - A.w * dx * dy;
                    const float gk = __expf(power);
                    const float raw = B.y * gk;
                    const float alpha = fminf(cfg.alpha_max, raw);
                    contrib = !(power > 0.f) && !(alpha < cfg.alpha_min);
                    if (contrib) {
                        T = T / (1.f - alpha);
                        const float w = alpha * T;
                        const float4 Cc = sp[e].c;
                        const float dLda = T * ((Cc.x - A0) * gC0 + (Cc.y - A1) * gC1 + (Cc.z - A2) * gC2 +
                                                (B.z - AD) * gD);
                        A0 = alpha * Cc.x + (1.f - alpha) * A0;
                        A1 = alpha * Cc.y + (1.f - alpha) * A1;
                        A2 = alpha * Cc.z + (1.f - alpha) * A2;
                        AD = alpha * B.z + (1.f - alpha) * AD;
                        if (MODE == GS_MAP) {
                            f[6] = w * gD;
                            f[7] = w * gC0;
                            f[8] = w * gC1;
                            f[9] = w * gC2;
                        } else {
                            f[5] = w * gD;
                        }
                        if (!(raw > cfg.alpha_max)) {
                            if (MODE == GS_MAP) f[5] = gk * dLda;
                            const float dp = alpha * dLda;
                            f[2] = -0.5f * dx * dx * dp;
                            f[3] = -dx * dy * dp;
                            f[4] = -0.5f * dy * dy * dp;
                            f[0] = (A.z * dx + A.w * dy) * dp;
                            f[1] = (A.w * dx + B.x * dy) * dp;
                        }
                    }
                }
                if (__ballot_sync(0xffffffffu, contrib) == 0u) continue;
                const float v = warp_reduce_scatter<NS, LOG>(f);
                if ((lane & ((1 << SHIFT) - 1)) == 0) {
                    const int s = lane >> SHIFT;
                    if (slot_col<MODE>(s) >= 0) atomicAdd(&acc[e][s], v);
                }
            }
        }
        group_sync(G);
        for (int q = G.lt; q < n_in * NS; q += G.TT) {
            const float v = (&acc[0][0])[q];
            const int col = slot_col<MODE>(q % NS);
            if (v != 0.f && col >= 0) atomicAdd(grad2d + (size_t)sid[q / NS] * GS_GRAD2D_STRIDE + col, v);
        }
        group_sync(G);
        hi = lo;
    }
}

}  // namespace gs

using namespace gs;

static gs_status render_checks(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats,
                               int64_t n) {
    if (!cfg) return set_error(GS_ERR_INVALID_ARG, "config is NULL");
    if (!cam) return set_error(GS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1 || cam->width > (1 << 20) ||
        cam->height > (1 << 20))
        return set_error(GS_ERR_INVALID_ARG, "bad camera size or stride");
    if (rec_dtype != GS_F32 && rec_dtype != GS_BF16 && rec_dtype != GS_F16)
        return set_error(GS_ERR_INVALID_ARG, "bad record dtype %d", rec_dtype);
    if (n < 0) return set_error(GS_ERR_INVALID_ARG, "bad Gaussian count");
    if (n > 0 && (!splats || ((uintptr_t)splats & 15)))
        return set_error(GS_ERR_INVALID_ARG, "splats NULL or not 16-byte aligned");
    return GS_OK;
}

extern "C" gs_status gs_render_fwd(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats,
                                   int64_t n, const uint32_t* vals, const uint32_t* tile_ranges,
                                   const uint32_t* tile_order, float* rgb, float* depth, float* t_final,
                                   uint32_t* last_idx, uint32_t* n_blended, gs_stream stream) {
    gs_status s;
    if ((s = render_checks(cfg, cam, rec_dtype, splats, n)) != GS_OK) return s;
    if (!tile_ranges || !rgb || !depth || !t_final || !last_idx)
        return set_error(GS_ERR_INVALID_ARG, "an image or range pointer is NULL");
    const Grid g = make_grid(*cam);
    const int gpc = R_THREADS / tile_threads(g);
    const unsigned nt = (unsigned)((g.TX * g.TY + gpc - 1) / gpc);
    cudaStream_t st = (cudaStream_t)stream;
#define GS_RF(DT) \
    k_render_fwd<DT><<<nt, R_THREADS, 0, st>>>(*cfg, g, splats, vals, tile_ranges, tile_order, rgb, depth, t_final, last_idx, \
                                               n_blended)
    if (rec_dtype == GS_F32) GS_RF(GS_F32);
    else if (rec_dtype == GS_BF16) GS_RF(GS_BF16);
    else GS_RF(GS_F16);
#undef GS_RF
    return check_launch("k_render_fwd");
}

extern "C" gs_status gs_loss_l1(const gs_config* cfg, const gs_camera* cam, const float* rgb, const float* depth,
                                const float* target_rgb, const float* target_depth, float* d_rgb, float* d_depth,
                                double* loss_out, gs_stream stream) {
    if (!cfg || !cam) return set_error(GS_ERR_INVALID_ARG, "config or camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1)
        return set_error(GS_ERR_INVALID_ARG, "bad camera size or stride");
    if (!rgb || !depth || !target_rgb || !target_depth || !d_rgb || !d_depth || !loss_out)
        return set_error(GS_ERR_INVALID_ARG, "a loss pointer is NULL");
    const Grid g = make_grid(*cam);
    const int64_t P = (int64_t)g.Ws * g.Hs;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss_out, 0, sizeof(double), st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset loss");
    const int64_t want = (P + 255) / 256;
    const int sms = num_sms();
    const unsigned nb = (unsigned)(want < 4 * sms ? want : 4 * sms);
    k_loss_l1<<<nb, 256, 0, st>>>(*cfg, P, rgb, depth, target_rgb, target_depth, d_rgb, d_depth, loss_out);
    return check_launch("k_loss_l1");
}

size_t gs_project_bwd_ws(int64_t n);


extern "C" gs_status gs_render_bwd(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* gsn,
                                   int rec_dtype, const void* splats, const uint32_t* vals,
                                   const uint32_t* tile_ranges, const uint32_t* tile_order, const float* t_final,
                                   const uint32_t* last_idx, const float* d_rgb, const float* d_depth, int mode,
                                   float* grad2d, gs_grads* grads, double* pose_grad6, float* score_terms,
                                   void* workspace, size_t* workspace_bytes, gs_stream stream) {
    if (!gsn) return set_error(GS_ERR_INVALID_ARG, "gaussians is NULL");
    gs_status s;
    const int64_t n = gsn->n;
    if ((s = render_checks(cfg, cam, rec_dtype, splats, n)) != GS_OK) return s;
    if (!workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    if (mode != GS_TRACK && mode != GS_MAP) return set_error(GS_ERR_INVALID_ARG, "bad mode %d", mode);
    const bool chain = (grads != nullptr) || pose_grad6 || score_terms;
    const size_t need = chain ? gs_project_bwd_ws(n) : 0;
    if (!workspace && need > 0) { *workspace_bytes = need; return GS_OK; }
    if (!workspace) { *workspace_bytes = 0; }
    else if (*workspace_bytes < need) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, need);
    if (!tile_ranges || !t_final || !last_idx || !d_rgb || !d_depth || (n > 0 && !grad2d))
        return set_error(GS_ERR_INVALID_ARG, "an input or grad2d pointer is NULL");
    if (n > 0 && ((uintptr_t)grad2d & 15)) return set_error(GS_ERR_INVALID_ARG, "grad2d not 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0 && cudaMemsetAsync(grad2d, 0, sizeof(float) * GS_GRAD2D_STRIDE * (size_t)n, st) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "memset grad2d");
    const Grid g = make_grid(*cam);
    const int gpc = R_THREADS / tile_threads(g);
    const unsigned nt = (unsigned)((g.TX * g.TY + gpc - 1) / gpc);
#define GS_RB(DT, MD)                                                                                              \
    k_render_bwd<DT, MD><<<nt, R_THREADS, 0, st>>>(*cfg, g, splats, vals, tile_ranges, tile_order, t_final, last_idx, \
                                                   d_rgb, d_depth, grad2d)
    if (n > 0) {
        if (mode == GS_MAP) {
            if (rec_dtype == GS_F32) GS_RB(GS_F32, GS_MAP);
            else if (rec_dtype == GS_BF16) GS_RB(GS_BF16, GS_MAP);
            else GS_RB(GS_F16, GS_MAP);
        } else {
            if (rec_dtype == GS_F32) GS_RB(GS_F32, GS_TRACK);
            else if (rec_dtype == GS_BF16) GS_RB(GS_BF16, GS_TRACK);
            else GS_RB(GS_F16, GS_TRACK);
        }
        if ((s = check_launch("k_render_bwd")) != GS_OK) return s;
    }
#undef GS_RB
    if (chain) {
        size_t wb = *workspace_bytes;
        return gs_project_bwd(cfg, cam, gsn, grad2d, grads, pose_grad6, score_terms, workspace, &wb, stream);
    }
    return GS_OK;
}
