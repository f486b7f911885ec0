// A-5 forward compositing (Sec. 2.1, Step 3: Eq. 2, Eq. 3), A-6 loss
// (Sec. 4.1, Eq. 6) and A-7 backward compositing (Sec. 2.2, Step 4: Eq. 4,
// Eq. 5) on sm_103a.
//
// Two forms of the compositing, chosen per frame:
//
// Pixel-parallel (full resolution, or a stride of 1 in one axis): one pixel
// per thread; a full 16x16 tile takes a CTA of 256 threads, the smaller
// tiles of a downsampled frame take groups of 64 or 128 threads of such a
// CTA, each group with its own named barrier and slice of the staging
// buffer.  Groups are issued in the heavy-first tile order produced by the
// binning, so the longest lists start first (the GPU counterpart of the
// paper's subtile streaming, Sec. 5.2).  Warps cover 8x4 pixel blocks.  The
// forward stages a tile's sorted list through shared memory in batches of
// 768 records (4 CTAs per SM; one dummy slot per 32 records); the thread
// that stages an entry also marks the warp blocks its alpha >= alpha_min
// ellipse meets (block bits), each warp builds from those bits a mask of the
// entries it may blend and visits only them, three at a time (their alphas
// are independent; the blends then run in order without branches; a slot
// past the word's last entry reads the word's dummy).  The alpha of a
// fragment is one FMA and one ex2: op e^(-q/2) = 2^(log2 op - q log2(e)/2),
// with q = d.(Q d) and log2 op staged per entry.  The forward also records,
// per pixel and run of 32 list entries, the entries it blended (the blend
// masks).
//
// Entry-parallel (both strides >= 2): see the section of that name below.
//
// The backward, given the blend masks, runs every 8x4 warp block as its own
// one-warp CTA: it visits the entries one of its pixels blended, takes each
// lane's decision from the lane's own mask bit, walks the fragments in
// reverse recovering T_k by division (Eq. 5), and merges the per-pixel
// gradients of each Gaussian across the warp with a reduce-scatter
// butterfly (each level halves the fields a lane carries) before one global
// atomic per (Gaussian, warp, field).  Without masks a CTA per tile stages
// the list, visits the entries whose pixel box meets each warp's block and
// sums the warps in shared memory first.  This replaces the paper's Gradient
// Merging Unit (Sec. 5.3).
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

#define R_THREADS 256            // largest CTA (16x16 tile)
#define R_BATCH 1024             // largest batch of entries a tile stages at a time
#define R_MASKW (R_BATCH / 32)   // mask words of a batch (at most 32: lane q holds word q)
#define R_FWD_SMEM (48 * 1024)          // forward staging budget per CTA (768 entries: 4 CTAs per SM)
#define R_BWD_SMEM (70 * 1024)          // backward staging budget per CTA (512 entries: 51 KB, 4 CTAs per SM)
#define R_STEP 3                 // list entries evaluated side by side in the forward walk

struct StagedSplat {
    float4 a;   // x, y, conic_a, conic_b
    float4 b;   // conic_c, opacity, depth, log2(opacity)
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

// `blk` numbers the CTA among those serving tiles this way; its groups take
// tile slots blk * gpc + gi of the tile order.
__device__ __forceinline__ Group make_group(const Grid& g, const uint32_t* order, int B, int blk) {
    Group G;
    G.TT = tile_threads(g);
    const int gpc = R_THREADS / G.TT;
    G.gi = threadIdx.x / G.TT;
    G.lt = threadIdx.x % G.TT;
    G.B = B;
    const int t = blk * gpc + G.gi;
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

// Sampled pixel q of the tile: full-resolution coordinates, and whether it
// lies in the image.
__device__ __forceinline__ bool ep_pixel(const Grid& g, int tile, int q, int& i, int& j) {
    const int tx = tile % g.TX, ty = tile / g.TX;
    i = tx * g.tw + q % g.tw;
    j = ty * g.th + q / g.tw;
    return q < g.tw * g.th && i < g.Ws && j < g.Hs;
}

// The 2D Gaussian at offset d = (dx, dy) from its mean (Eq. 2): with the
// conic Q = [[ca, cb], [cb, cc]], (a, b) = Q d and q = d^T Q d = dx a + dy b,
// the exponent is -q/2 and the backward's mean gradient is (a, b) times
// dL/dexponent.  The operations are spelled out (no contraction left to the
// compiler) so that every compositing kernel, forward and backward, computes
// the same value and so takes the same blending decisions; q < 0 (a positive
// exponent, from rounding) skips the fragment.
struct Quad {
    float a, b, q;
};

__device__ __forceinline__ Quad quad_form(float ca, float cb, float cc, float dx, float dy) {
    Quad r;
    r.a = __fmaf_rn(cb, dy, __fmul_rn(ca, dx));
    r.b = __fmaf_rn(cc, dy, __fmul_rn(cb, dx));
    r.q = __fmaf_rn(dx, r.a, __fmul_rn(dy, r.b));
    return r;
}

// 2^x with the SFU's ex2 instruction.
__device__ __forceinline__ float exp2_sfu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2 of a staged opacity (the same instruction for every kernel that
// stages an entry, so all of them see the same value).
__device__ __forceinline__ float log2_opacity(float op) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(op));
    return y;
}

// -log2(e) / 2: op e^(-q/2) = 2^(log2(op) - q log2(e) / 2).
#define R_NEG_HALF_LOG2E (-0.721347520444481703680f)

// Unclamped alpha op e^(-q/2) of a fragment, one FMA and one ex2.
__device__ __forceinline__ float raw_alpha(float q, float log2_op) {
    return exp2_sfu(__fmaf_rn(q, R_NEG_HALF_LOG2E, log2_op));
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
// t2 receives the widened threshold 2 (ln(opacity / alpha_min) + 1e-4), or
// -1 when the box is the 3-sigma box alone (no usable ellipse).
__device__ __forceinline__ int4 pixel_box(const Splat& v, float alpha_min, float& t2) {
    const int xi = pix_floor(v.x), yi = pix_floor(v.y), r = v.radius;
    int4 box = make_int4(xi - r, xi + r, yi - r, yi + r);
    t2 = -1.f;
    const float det = v.ca * v.cc - v.cb * v.cb;
    if (!(det > 0.f) || !(v.op > 0.f) || !(alpha_min > 0.f)) return box;
    const float thr = logf(v.op / alpha_min);
    if (thr < -1e-4f) return make_int4(1, 0, 1, 0);  // empty: opacity < alpha_min
    const float t = 2.f * (fmaxf(thr, 0.f) + 1e-4f);
    const float ex = sqrtf(t * v.cc / det) * 1.001f + 1e-3f;
    const float ey = sqrtf(t * v.ca / det) * 1.001f + 1e-3f;
    if (!(ex < 1e8f) || !(ey < 1e8f)) return box;
    t2 = t;
    // pixel p qualifies when |p + 0.5 - x| <= ex
    box.x = max(box.x, (int)ceilf(v.x - ex - 0.5f));
    box.y = min(box.y, (int)floorf(v.x + ex - 0.5f));
    box.z = max(box.z, (int)ceilf(v.y - ey - 0.5f));
    box.w = min(box.w, (int)floorf(v.y + ey - 0.5f));
    return box;
}

// The warp blocks of a group's tile in full-resolution pixels: warp w's
// block (strip w / wx, column w % wx) spans columns x0 + (w % wx) sxb ..
// + bw and rows y0 + (w / wx) syb .. + bh (the extents map_pixel gives).
struct TileBlocks {
    int x0, y0, bw, bh, sxb, syb, wx, ns;
};

// (KST == 1: a full-resolution 16x16 tile of 8 warps, compile-time extents)
template <int KST>
__device__ __forceinline__ TileBlocks tile_blocks(const Grid& g, int tile, int TT) {
    const int tx = tile % g.TX, ty = tile / g.TX;
    TileBlocks b;
    if (KST == 1) {
        b.x0 = tx * 16;
        b.y0 = ty * 16;
        b.bw = 7;
        b.bh = 3;
        b.sxb = 8;
        b.syb = 4;
        b.wx = 2;
        b.ns = 4;
        return b;
    }
    const int BW = g.tw < 8 ? g.tw : 8, BH = 32 / BW, WX = g.tw / BW;
    b.x0 = tx * g.tw * g.sx;
    b.y0 = ty * g.th * g.sy;
    b.bw = (BW - 1) * g.sx;
    b.bh = (BH - 1) * g.sy;
    b.sxb = BW * g.sx;
    b.syb = BH * g.sy;
    b.wx = WX;
    b.ns = (TT >> 5) / WX;
    return b;
}

// Warp blocks of the tile in which a Gaussian can be blended: bit w when
// some pixel of warp w's block lies in the Gaussian's box (bx, staged form)
// and in the region d^T Q d <= t (t = t2 widened by 1 %; t2 < 0: the box
// alone decides).  Per strip of blocks (a band of rows) the ellipse's x
// extent over the band follows from its chord [(-cb dy -+ sqrt(t ca - det
// dy^2)) / ca] at the band's rows closest to the rightmost point (dy = -cb
// ex / cc) and the leftmost point (dy = cb ex / cc): the chord's right end
// is concave in dy and its left end convex.  The extent is widened by 1e-2
// ex + 0.05 px, well beyond the float32 rounding of the fragment test, so
// the bits never drop a fragment the compositing loop would blend.
__device__ __forceinline__ unsigned block_bits(const Splat& v, const int4& bx, float t2, const TileBlocks& tb) {
    const bool ell = t2 > 0.f;
    const float det = v.ca * v.cc - v.cb * v.cb;
    float tA = 0.f, ey = 0.f, yr = 0.f, ia = 0.f, sl = 0.f;
    if (ell) {
        const float t = t2 * 1.01f;
        const float ex = sqrtf(t * v.cc / det);
        tA = t * v.ca;
        ey = sqrtf(tA / det);
        yr = -v.cb * ex / v.cc;
        ia = 1.f / v.ca;
        sl = 1e-2f * ex + 0.05f;
    }
    unsigned bits = 0u;
#pragma unroll 1
    for (int s = 0; s < tb.ns; ++s) {
        const int ry = tb.y0 + s * tb.syb;
        const int r0 = max(ry, bx.z), r1 = min(ry + tb.bh, bx.z + bx.w);
        if (r0 > r1) continue;
        int c0 = bx.x, c1 = bx.x + bx.y;
        if (ell) {
            const float ylo = fminf(fmaxf((float)r0 + 0.5f - v.y, -ey), ey);
            const float yhi = fminf(fmaxf((float)r1 + 0.5f - v.y, -ey), ey);
            const float dr = fminf(fmaxf(yr, ylo), yhi), dl = fminf(fmaxf(-yr, ylo), yhi);
            const float xr = (sqrtf(fmaxf(tA - det * dr * dr, 0.f)) - v.cb * dr) * ia;
            const float xl = (-sqrtf(fmaxf(tA - det * dl * dl, 0.f)) - v.cb * dl) * ia;
            c0 = max(c0, (int)ceilf(v.x + xl - sl - 0.5f));
            c1 = min(c1, (int)floorf(v.x + xr + sl - 0.5f));
        }
        for (int c = 0; c < tb.wx; ++c) {
            const int x = tb.x0 + c * tb.sxb;
            if (c0 <= x + tb.bw && c1 >= x) bits |= 1u << (s * tb.wx + c);
        }
    }
    return bits;
}

// Stages a Gaussian; with tb (the forward) c.w holds its block bits.
__device__ __forceinline__ void fill_staged(const Splat& v, float alpha_min, StagedSplat& s,
                                            const TileBlocks* tb = nullptr) {
    s.a = make_float4(v.x, v.y, v.ca, v.cb);
    s.b = make_float4(v.cc, v.op, v.depth, log2_opacity(v.op));
    // the box as (x0, x1 - x0, y0, y1 - y0), clamped far outside any image;
    // an empty box never matches
    float t2;
    const int4 bx = pixel_box(v, alpha_min, t2);
    const int lo = -(1 << 28), hi = 1 << 28;
    const int x0 = max(bx.x, lo), x1 = min(bx.y, hi), y0 = max(bx.z, lo), y1 = min(bx.w, hi);
    s.box = x1 < x0 || y1 < y0 ? make_int4(hi, 0, hi, 0) : make_int4(x0, x1 - x0, y0, y1 - y0);
    s.c = make_float4(v.r, v.g, v.b, tb ? __uint_as_float(block_bits(v, s.box, t2, *tb)) : 0.f);
}

// Stages list entries [0, n_in) of `ids` into sp[] (and their ids into sid[]
// when given) with the group's TT threads.  Each thread gathers KST records
// before it converts any, so KST dependent id -> record loads are in flight
// per thread (KST = 4 for the small groups of downsampled frames, which
// stage several entries per thread; 1 for full-resolution tiles).
// Forward layout of a staged batch: slot 33 q of each run of 32 entries is
// a dummy that never blends (an empty box), entry e sits at slot il_slot(e):
// a step slot with no entry left in its word reads the word's dummy instead
// of testing for one.
__device__ __forceinline__ int il_slot(int e) { return (e >> 5) * 33 + (e & 31) + 1; }

template <int DT, int KST, bool IL = false>
__device__ __forceinline__ void stage_batch(const void* __restrict__ splats, const uint32_t* __restrict__ ids,
                                            int n_in, int lt, int TT, float alpha_min, StagedSplat* sp,
                                            uint32_t* sid, const TileBlocks* tb = nullptr) {
    for (int e0 = lt; e0 < n_in; e0 += KST * TT) {
        uint32_t id[KST];
#pragma unroll
        for (int k = 0; k < KST; ++k) id[k] = e0 + k * TT < n_in ? __ldg(ids + e0 + k * TT) : 0u;
        Splat v[KST];
#pragma unroll
        for (int k = 0; k < KST; ++k)
            if (e0 + k * TT < n_in) v[k] = load_splat<DT>(splats, id[k]);
#pragma unroll
        for (int k = 0; k < KST; ++k)
            if (e0 + k * TT < n_in) {
                fill_staged(v[k], alpha_min, sp[IL ? il_slot(e0 + k * TT) : e0 + k * TT], tb);
                if (sid) sid[e0 + k * TT] = id[k];
            }
    }
}

// Overlap masks of the staged entries with the warp's block: bit e of word q
// is set when entry 32q + e (below `limit`) meets the block.  Lane q returns
// word q (words at or beyond `words` are zero), so a word is one shuffle away
// and the masks stay in registers.  Only the words that hold entries are
// built (a loop to the batch's last word rather than over all R_MASKW:
// tracking step 236.6 -> 231.5 us).
__device__ __forceinline__ unsigned warp_masks(const StagedSplat* sp, int limit, int words, const PixelMap& m) {
    const int lane = threadIdx.x & 31;
    unsigned mine = 0u;
    const int nq = min(words, (limit + 31) >> 5);  // the words holding entries
#pragma unroll 4
    for (int q = 0; q < nq; ++q) {
        const int e = q * 32 + lane;
        bool hit = false;
        if (e < limit) {
            const int4 box = sp[e].box;
            hit = !(box.x + box.y < m.wx0 || box.x > m.wx1 || box.z + box.w < m.wy0 || box.z > m.wy1);
        }
        const unsigned w = __ballot_sync(0xffffffffu, hit);
        if (lane == q) mine = w;
    }
    return mine;
}

// The same masks from the block bits of a forward batch (warp wg of its
// group): entries whose alpha region misses the block are left out too.
__device__ __forceinline__ unsigned warp_masks_bits(const StagedSplat* sp, int limit, int words, int wg) {
    const int lane = threadIdx.x & 31;
    unsigned mine = 0u;
    const int nq = min(words, (limit + 31) >> 5);  // the words holding entries
#pragma unroll 4
    for (int q = 0; q < nq; ++q) {
        const int e = q * 32 + lane;
        const bool hit = e < limit && ((__float_as_uint(sp[il_slot(e)].c.w) >> wg) & 1u);
        const unsigned w = __ballot_sync(0xffffffffu, hit);
        if (lane == q) mine = w;
    }
    return mine;
}

// Alpha of a staged Gaussian at the pixel (Eq. 2), or -1 when the pixel is
// outside its box or the exponent is positive (the fragment is skipped).
__device__ __forceinline__ float frag_alpha(const StagedSplat& s, const PixelMap& m, float pxc, float pyc,
                                           float alpha_max) {
    const int4 box = s.box;
    const float4 A = s.a;
    const float cc = s.b.x, lop = s.b.w;
    const Quad Qd = quad_form(A.z, A.w, cc, pxc - A.x, pyc - A.y);
    const float alpha = fminf(alpha_max, raw_alpha(Qd.q, lop));
    const bool in = (unsigned)(m.px - box.x) <= (unsigned)box.y && (unsigned)(m.py - box.z) <= (unsigned)box.w &&
                    !(Qd.q < 0.f);
    return in ? alpha : -1.f;
}

// Forward outputs (gs_render_fwd) and, when trgb is given, the fused loss
// (gs_render_fwd_loss).
struct FwdOut {
    float* rgb;
    float* depth;
    float* t;
    uint32_t* last;
    uint32_t* nb;
    const float* trgb;  // NULL: no loss
    const float* tdepth;
    float* d_rgb;
    float* d_depth;
    double* loss;
    uint32_t* bmask;    // NULL: no blend masks
};

// Blend masks: for each pixel of a tile and each run of 32 list entries,
// the entries the forward blended into that pixel (bit e of run r: entry
// 32 r + e of the tile's list).  A pixel-parallel tile (TT <= 256 threads,
// pixel = thread lt of the group) with list [s, s + len) keeps run r of
// pixel lt at word 256 (floor(s / 32) + t) + r TT + lt: run-major, so a
// warp's 32 pixels read one 128-byte line; the TT ceil(len / 32) words of a
// tile end before the next tile's first word.
__host__ __device__ inline size_t blend_mask_base(int tile, uint32_t start) {
    return (size_t)256 * ((size_t)(start >> 5) + (size_t)tile);
}

// Entry-parallel tiles (at most 64 sampled pixels) keep one run per pixel
// instead of one per warp: pixel q of tile t at word 64 (floor(s / 32) + t)
// + q ceil(len / 32).
__host__ __device__ inline size_t blend_mask_base_ep(int tile, uint32_t start) {
    return (size_t)64 * ((size_t)(start >> 5) + (size_t)tile);
}

// Writes sampled pixel (i, j)'s results; with the fused loss also its image
// gradient (the formulas of k_loss_l1 on the same float values) and returns
// its share of the loss.
__device__ __forceinline__ float write_pixel(const gs_config& cfg, const Grid& g, const FwdOut& O, int i, int j,
                                             float C0, float C1, float C2, float D, float T, uint32_t last,
                                             uint32_t nb) {
    const size_t P = (size_t)g.Ws * g.Hs;
    const size_t pix = (size_t)j * g.Ws + i;
    const float c[3] = {C0 + T * cfg.bg[0], C1 + T * cfg.bg[1], C2 + T * cfg.bg[2]};
    O.rgb[pix] = c[0];
    O.rgb[P + pix] = c[1];
    O.rgb[2 * P + pix] = c[2];
    O.depth[pix] = D;
    O.t[pix] = T;
    O.last[pix] = last;
    if (O.nb) O.nb[pix] = nb;
    if (!O.trgb) return 0.f;
    const float inv3 = 1.f / (3.f * (float)P), inv1 = 1.f / (float)P;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float r = c[k] - O.trgb[k * P + pix];
        acc += cfg.w_rgb * fabsf(r) * inv3;
        O.d_rgb[k * P + pix] = cfg.w_rgb * (r > 0.f ? inv3 : (r < 0.f ? -inv3 : 0.f));
    }
    const float td = O.tdepth[pix];
    float gd = 0.f;
    if (td != 0.f) {
        const float r = D - td;
        acc += cfg.w_depth * fabsf(r) * inv1;
        gd = cfg.w_depth * (r > 0.f ? inv1 : (r < 0.f ? -inv1 : 0.f));
    }
    O.d_depth[pix] = gd;
    return acc;
}

// Warp sum of the pixels' loss shares, one float64 atomic per warp (all 32
// lanes call it).
__device__ __forceinline__ void add_loss(const FwdOut& O, float part) {
    if (!O.trgb) return;
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0 && part != 0.f) atomicAdd(O.loss, (double)part);
}

// Forward compositing of group G's tile, pixel-parallel (sp_all: the CTA's
// staging buffer, G.B entries plus one dummy per 32 per group).
template <int DT, int KST>
__device__ __forceinline__ void fwd_pp(const gs_config& cfg, const Grid& g, const void* __restrict__ splats,
                                       const uint32_t* __restrict__ vals, const uint32_t* __restrict__ ranges,
                                       const FwdOut& O, const Group& G, StagedSplat* sp_all) {
    StagedSplat* sp = sp_all + G.gi * (G.B / 32 * 33);
    const int tile = G.tile;
    const PixelMap m = map_pixel(g, tile, G.lt);
    const TileBlocks tb = tile_blocks<KST>(g, tile, G.TT);
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const float pxc = (float)m.px + 0.5f, pyc = (float)m.py + 0.5f;
    for (int q = G.lt; q < G.B / 32; q += G.TT) {  // the dummies
        sp[q * 33].a = make_float4(0.f, 0.f, 0.f, 0.f);
        sp[q * 33].b = make_float4(0.f, 0.f, 0.f, 0.f);
        sp[q * 33].c = make_float4(0.f, 0.f, 0.f, 0.f);
        sp[q * 33].box = make_int4(1 << 28, 0, 1 << 28, 0);
    }
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    uint32_t last = 0, nb = 0;
    bool done = !m.inside;
    const int words = G.B / 32;
    // this pixel's blend-mask words (run r at bm_pix[r TT])
    uint32_t* bm_pix = O.bmask ? O.bmask + blend_mask_base(tile, start) + G.lt : nullptr;
    for (uint32_t b = start; b < end; b += G.B) {
        // from the second batch on: a barrier (the previous batch's records
        // are no longer read) that also ends the tile once every pixel stopped
        if (b != start && group_count(G, done) == G.TT) break;
        const int n_in = (int)min((uint32_t)G.B, end - b);
        stage_batch<DT, KST, true>(splats, vals + b, n_in, G.lt, G.TT, cfg.alpha_min, sp, nullptr, &tb);
        group_sync(G);
        if (!__all_sync(0xffffffffu, done)) {
            const unsigned mword = warp_masks_bits(sp, n_in, words, G.lt >> 5);
            const uint32_t base = b - start;
            const int wq = (n_in + 31) >> 5;
#pragma unroll 1
            for (int q = 0; q < wq; ++q) {
                unsigned mq = __shfl_sync(0xffffffffu, mword, q);
                unsigned bq = 0u;  // entries of word q this pixel blended
                while (mq) {
                    // R_STEP entries per step: their alphas do not depend on
                    // T, so they are evaluated side by side; the blends then
                    // run in list order without branches (a skipped fragment
                    // adds zero weight).  Front to back, a fragment with
                    // alpha >= alpha_min is blended unless it would take T
                    // below t_eps, where the pixel stops (Eq. 3).
                    // slot of the next entry, or the word's dummy once none is left
                    int eu[R_STEP];
                    float au[R_STEP];
#pragma unroll
                    for (int u = 0; u < R_STEP; ++u) {
                        eu[u] = q * 33 + __ffs(mq);
                        mq &= mq - 1u;
                    }
#pragma unroll
                    for (int u = 0; u < R_STEP; ++u) au[u] = frag_alpha(sp[eu[u]], m, pxc, pyc, cfg.alpha_max);
#pragma unroll
                    for (int u = 0; u < R_STEP; ++u) {
                        const float alpha = au[u];
                        const bool valid = !done && alpha >= cfg.alpha_min;
                        const float Tn = T * (1.f - alpha);
                        const bool stop = valid && Tn < cfg.t_eps;
                        const bool ok = valid && !stop;
                        done = done || stop;
                        const int e = eu[u];
                        const float4 Cc = sp[e].c;
                        const float dep = sp[e].b.z;
                        const float w = ok ? alpha * T : 0.f;
                        C0 += w * Cc.x;
                        C1 += w * Cc.y;
                        C2 += w * Cc.z;
                        D += w * dep;
                        T = ok ? Tn : T;
                        bq |= ok ? 1u << ((e - q * 33 - 1) & 31) : 0u;
                    }
                    if (__all_sync(0xffffffffu, done)) break;
                }
                // the count and the last position follow from the word's blended bits
                nb += __popc(bq);
                if (bq != 0u) last = base + (uint32_t)(q * 32 + 32 - __clz(bq));
                // every run up to the one where the warp stops is written (a
                // run past every pixel's last position is never read)
                if (bm_pix) bm_pix[(size_t)((base >> 5) + q) * G.TT] = bq;
                if (__all_sync(0xffffffffu, done)) break;
            }
        }
    }
    float lpart = 0.f;
    if (m.inside) lpart = write_pixel(cfg, g, O, m.i, m.j, C0, C1, C2, D, T, last, nb);
    add_loss(O, lpart);
}

template <int DT, int KST>
__global__ void __launch_bounds__(R_THREADS, KST == 1 ? 4 : 2)
    k_render_fwd(gs_config cfg, Grid g, const void* __restrict__ splats, const uint32_t* __restrict__ vals,
                 const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ order, FwdOut O, int B) {
    extern __shared__ __align__(16) unsigned char r_smem[];
    const Group G = make_group(g, order, B, blockIdx.x);
    if (G.tile < 0) return;
    fwd_pp<DT, KST>(cfg, g, splats, vals, ranges, O, G, reinterpret_cast<StagedSplat*>(r_smem));
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
// Fields merged per fragment, in the order the backward forms them:
//   GS_TRACK  a h, b h, u dx, u dy, v dy, w gD                      (6)
//   GS_MAP    a h, b h, u dx, u dy, v dy, G T (dL/dalpha T^-1), w gD,
//             w gR, w gG, w gB                                      (10)
// with h = -dL/d(exponent) / 2 = -alpha dL/dalpha / 2, (u, v) = h (dx, dy),
// (a, b) = Q d and w = T alpha.  The gradients follow by exact power-of-two
// scalings applied once per entry when a batch is written out:
// dL/dmean = -2 (a h, b h) (since dL/dmean = Q d dL/d(exponent)),
// dL/dconic = (u dx, 2 u dy, v dy) (the exponent is -(A dx^2 + 2 B dx dy +
// C dy^2) / 2).
template <int MODE>
struct Fields {
    static constexpr int N = MODE == GS_MAP ? 10 : 6;
};

// grad2d column of a merged field, and its scale.
template <int MODE>
__device__ __forceinline__ int field_col(int f) {
    if (MODE == GS_MAP) return f < 7 ? f : f + 1;  // du dv dA dB dC dop dd | dr dg db
    return f < 5 ? f : 6;                          // du dv dA dB dC | dd
}
__device__ __forceinline__ float field_scale(int f) { return f < 2 ? -2.f : (f == 3 ? 2.f : 1.f); }

// Per-fragment quantities of the backward that do not depend on the
// running state: offsets, Gaussian falloff G, unclamped and clamped alpha,
// and whether the fragment was blended.
struct FragGeo {
    float dx, dy, a, b, q, raw, alpha, dep;  // offset, Q d, d^T Q d, alphas, depth
    bool contrib;
};

// The geometry of a staged entry at the pixel, with the forward's arithmetic
// (so the same alpha); `blended` says whether the forward blended it.
__device__ __forceinline__ FragGeo frag_geo_at(const StagedSplat& s, float pxc, float pyc, const gs_config& cfg,
                                               bool blended) {
    FragGeo f;
    const float4 A = s.a;
    const float4 Bv = s.b;
    f.dep = Bv.z;
    f.dx = pxc - A.x;
    f.dy = pyc - A.y;
    const Quad Qd = quad_form(A.z, A.w, Bv.x, f.dx, f.dy);
    f.a = Qd.a;
    f.b = Qd.b;
    f.q = Qd.q;
    f.raw = raw_alpha(Qd.q, Bv.w);
    f.alpha = fminf(cfg.alpha_max, f.raw);
    f.contrib = blended;
    return f;
}

// Without blend masks the decision is re-derived: inside the box, exponent
// <= 0, alpha >= alpha_min, before the pixel's last blended position.
__device__ __forceinline__ FragGeo frag_geo(const StagedSplat& s, const PixelMap& m, float pxc, float pyc,
                                            const gs_config& cfg, bool before_last) {
    FragGeo f = frag_geo_at(s, pxc, pyc, cfg, false);
    const int4 box = s.box;
    f.contrib = before_last && (unsigned)(m.px - box.x) <= (unsigned)box.y &&
                (unsigned)(m.py - box.z) <= (unsigned)box.w && !(f.q < 0.f) && !(f.alpha < cfg.alpha_min);
    return f;
}

// A pixel's running state in the backward walk: the transmittance in front
// of the current entry, s = A . g (the normalised suffix sum A of colour and
// depth behind it -- the background entering with weight T_final -- dotted
// with the image gradient g) and g itself.
struct BackState {
    float T, sg, gC0, gC1, gC2, gD;
};

// Loads a pixel's backward inputs (t_final, image gradients); pixels outside
// the image keep T = 1 and zero gradients.  Returns its last_idx (0 outside).
__device__ __forceinline__ uint32_t back_start(const gs_config& cfg, const Grid& g, const PixelMap& m,
                                               const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                                               const float* __restrict__ d_rgb, const float* __restrict__ d_depth,
                                               BackState& S) {
    S.T = 1.f;
    S.gC0 = S.gC1 = S.gC2 = S.gD = 0.f;
    uint32_t last = 0;
    if (m.inside) {
        const size_t P = (size_t)g.Ws * g.Hs;
        const size_t pix = (size_t)m.j * g.Ws + m.i;
        S.T = t_final[pix];
        last = last_idx[pix];
        S.gC0 = d_rgb[pix];
        S.gC1 = d_rgb[P + pix];
        S.gC2 = d_rgb[2 * P + pix];
        S.gD = d_depth[pix];
    }
    S.sg = cfg.bg[0] * S.gC0 + cfg.bg[1] * S.gC1 + cfg.bg[2] * S.gC2;
    return last;
}

// One fragment, back to front: T_k recovered by division (Eq. 5).  With
// w = T_k alpha_k and c_k . g (colour and depth dotted with the image
// gradient),
//   dL/dalpha_k = T_k (c_k . g - s_k),  s_k = A_k . g,
//   s_{k-1} = s_k + alpha_k (c_k . g - s_k),
// and alpha dL/dalpha = w (c . g - s) is the exponent's gradient.  Writes the
// fragment's merged fields f[0, Fields<MODE>::N).  Branch-free: every lane
// evaluates the recursion (all values are finite: 1 - alpha >= 1 -
// alpha_max); a lane whose pixel did not blend the entry keeps its state and
// contributes zeros.
template <int MODE>
__device__ __forceinline__ void back_frag(BackState& S, const FragGeo& fg, const float4& Cc, const gs_config& cfg,
                                          float* f) {
    const float alpha = fg.alpha;
    // fast division (at most 2 ulp for these operands: 1 - alpha in
    // [0.01, 1], T in [t_eps, 1]); over the few hundred entries a pixel
    // recovers the relative drift stays near 1e-5
    S.T = fg.contrib ? __fdividef(S.T, 1.f - alpha) : S.T;
    const float w = fg.contrib ? alpha * S.T : 0.f;
    const float cg = __fmaf_rn(fg.dep, S.gD, __fmaf_rn(Cc.z, S.gC2, __fmaf_rn(Cc.y, S.gC1, Cc.x * S.gC0)));
    const float dif = cg - S.sg;
    S.sg = fg.contrib ? __fmaf_rn(alpha, dif, S.sg) : S.sg;
    // the clamp passes no gradient to opacity or shape
    const bool clamped = fg.raw > cfg.alpha_max;
    const float h = clamped ? 0.f : (-0.5f * w) * dif;  // -dL/d(exponent) / 2
    const float u = h * fg.dx, v = h * fg.dy;
    f[0] = fg.a * h;
    f[1] = fg.b * h;
    f[2] = u * fg.dx;
    f[3] = u * fg.dy;
    f[4] = v * fg.dy;
    if (MODE == GS_MAP) {
        // dalpha/dopacity = e^(-q/2)
        f[5] = (fg.contrib && !clamped) ? exp2_sfu(__fmul_rn(fg.q, R_NEG_HALF_LOG2E)) * (S.T * dif) : 0.f;
        f[6] = w * S.gD;
        f[7] = w * S.gC0;
        f[8] = w * S.gC1;
        f[9] = w * S.gC2;
    } else {
        f[5] = w * S.gD;
    }
}

// Backward compositing of group G's tile, pixel-parallel, without blend
// masks (smem: the CTA's staging, id and accumulator buffers for gpc groups
// of G.B entries; s_max_all: one word per warp).  Each warp visits the
// staged entries whose pixel box meets its block, up to the furthest last
// position of its pixels.
template <int DT, int MODE, int KST>
__device__ __forceinline__ void bwd_pp(const gs_config& cfg, const Grid& g, const void* __restrict__ splats,
                                       const uint32_t* __restrict__ vals, const uint32_t* __restrict__ ranges,
                                       const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                                       const float* __restrict__ d_rgb, const float* __restrict__ d_depth,
                                       float* __restrict__ grad2d, const Group& G, unsigned char* smem,
                                       uint32_t* s_max_all) {
    constexpr int NF = Fields<MODE>::N;
    constexpr int BSTEP = 2;  // entries per backward step, merged together
    static_assert(BSTEP * NF <= 32, "one lane per merged value");
    const int gpc = R_THREADS / G.TT;
    StagedSplat* sp_all = reinterpret_cast<StagedSplat*>(smem);
    uint32_t* sid_all = reinterpret_cast<uint32_t*>(sp_all + gpc * G.B);
    float(*acc_all)[NF] = reinterpret_cast<float(*)[NF]>(sid_all + gpc * G.B);
    StagedSplat* sp = sp_all + G.gi * G.B;
    uint32_t* sid = sid_all + G.gi * G.B;
    float(*acc)[NF] = acc_all + G.gi * G.B;
    uint32_t* s_wl = s_max_all + G.gi * (G.TT >> 5);  // the group's per-warp maxima
    const int tile = G.tile;
    const PixelMap m = map_pixel(g, tile, G.lt);
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const float pxc = (float)m.px + 0.5f, pyc = (float)m.py + 0.5f;
    const int lane = threadIdx.x & 31;
    // the merged field this lane adds (entry owner / NF of a step, field
    // owner % NF), or -1
    const int owner = merge_owner<BSTEP * NF>();
    BackState S;
    uint32_t last = back_start(cfg, g, m, t_final, last_idx, d_rgb, d_depth, S);
    // a last_idx beyond the tile's list (inconsistent inputs) is clamped
    last = min(last, end - start);
    uint32_t wlast = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    if (lane == 0) s_wl[G.lt >> 5] = wlast;
    group_sync(G);
    uint32_t s_max = 0;
    for (int w = 0; w < (G.TT >> 5); ++w) s_max = max(s_max, s_wl[w]);
    const int words = G.B / 32;
    // batches [start + k B, start + (k + 1) B) from the last one holding a
    // blended entry back to the first (whole mask words for every batch)
    for (int k = (int)((s_max + G.B - 1) / G.B) - 1; k >= 0; --k) {
        const uint32_t base_pos = (uint32_t)k * G.B;
        const uint32_t lo = start + base_pos, hi = start + min(s_max, base_pos + G.B);
        const int n_in = (int)(hi - lo);
        stage_batch<DT, KST>(splats, vals + lo, n_in, G.lt, G.TT, cfg.alpha_min, sp, sid);
        for (int q = G.lt; q < G.B * NF; q += G.TT) (&acc[0][0])[q] = 0.f;
        group_sync(G);
        // entries at or beyond the warp's furthest blended position are skipped
        const int wlimit = (int)min((uint32_t)n_in, wlast > base_pos ? wlast - base_pos : 0u);
        const unsigned mword = warp_masks(sp, wlimit, words, m);
#pragma unroll 1
        for (int q = words - 1; q >= 0; --q) {
            unsigned mq = __shfl_sync(0xffffffffu, mword, q);
            while (mq) {
                // BSTEP entries per step, last first: their geometry does
                // not depend on the running state
                int eu[BSTEP];
#pragma unroll
                for (int u = 0; u < BSTEP; ++u) {
                    const int bit = mq ? 31 - __clz(mq) : -1;
                    eu[u] = bit >= 0 ? q * 32 + bit : -1;
                    if (bit >= 0) mq &= ~(1u << bit);
                }
                FragGeo gu[BSTEP];
#pragma unroll
                for (int u = 0; u < BSTEP; ++u) {
                    const int e = eu[u] >= 0 ? eu[u] : 0;
                    gu[u] = frag_geo(sp[e], m, pxc, pyc, cfg, eu[u] >= 0 && base_pos + (uint32_t)e < last);
                }
                float f[BSTEP * NF];
#pragma unroll
                for (int u = 0; u < BSTEP; ++u) back_frag<MODE>(S, gu[u], sp[eu[u] >= 0 ? eu[u] : 0].c, cfg, f + u * NF);
                // the step's fields merged at once
                bool any = false;
#pragma unroll
                for (int u = 0; u < BSTEP; ++u) any = any || gu[u].contrib;
                if (__any_sync(0xffffffffu, any)) {
                    const float v = warp_merge<BSTEP * NF>(f);
                    if (owner >= 0) {
                        const int u = owner / NF;
                        int e = eu[0];
#pragma unroll
                        for (int x = 1; x < BSTEP; ++x) e = u == x ? eu[x] : e;
                        if (e >= 0) atomicAdd(&acc[e][owner - u * NF], v);
                    }
                }
            }
        }
        group_sync(G);
        for (int q = G.lt; q < n_in * NF; q += G.TT) {
            const float v = (&acc[0][0])[q];
            const int f = q % NF;
            if (v != 0.f) atomicAdd(grad2d + (size_t)sid[q / NF] * GS_GRAD2D_STRIDE + field_col<MODE>(f),
                                    v * field_scale(f));
        }
        if (k > 0) group_sync(G);  // the next batch reuses the buffers
    }
}

// 4 CTAs per SM for the pose-only backward (64 registers); 3 when mapping,
// whose 16-slot merge would spill at 64 (measured 363 vs 342 us at 1200x680).
template <int DT, int MODE, int KST>
__global__ void __launch_bounds__(R_THREADS, KST == 1 ? (MODE == GS_TRACK ? 4 : 3) : 2)
    k_render_bwd(gs_config cfg, Grid g, const void* __restrict__ splats, const uint32_t* __restrict__ vals,
                 const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ order,
                 const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                 const float* __restrict__ d_rgb, const float* __restrict__ d_depth, float* __restrict__ grad2d,
                 int B) {
    extern __shared__ __align__(16) unsigned char r_smem[];
    __shared__ uint32_t s_max_all[R_THREADS / 32];
    const Group G = make_group(g, order, B, blockIdx.x);
    if (G.tile < 0) return;
    bwd_pp<DT, MODE, KST>(cfg, g, splats, vals, ranges, t_final, last_idx, d_rgb, d_depth, grad2d, G, r_smem,
                          s_max_all);
}

// Two float32 values in one 64-bit register for the packed f32x2
// instructions (add, sub, mul, fma with round-to-nearest: one instruction for
// both halves, each half rounded exactly as the scalar operation).
typedef unsigned long long x2f;

__device__ __forceinline__ x2f x2_pack(float lo, float hi) {
    x2f r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void x2_unpack(x2f v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ x2f x2_sub(x2f a, x2f b) {
    x2f r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ x2f x2_mul(x2f a, x2f b) {
    x2f r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ x2f x2_fma(x2f a, x2f b, x2f c) {  // a b + c
    x2f r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// One warp's staged run for the masked backward: the blended entries'
// fields, one array per field (slot k: the run's k-th blended entry from the
// top), so that slots k and k + 1 load as one packed pair.
struct __align__(16) RunStage {
    float x[32], y[32], ca[32], cb[32], cc[32], lop[32], dep[32], cr[32], cg[32], cl[32];
    uint32_t id[32];
};

__device__ __forceinline__ x2f x2_ld(const float* p) { return *reinterpret_cast<const x2f*>(p); }

// Two consecutive fragments of a warp's run, back to front (slot k + 1 is
// the earlier entry of the list, so slot k goes first): the geometry and the
// gradient products of both in packed pairs, with the forward's arithmetic
// in every half (the same alpha); the transmittance and suffix recursions
// (Eq. 5) run fragment by fragment as in back_frag.  c0, c1: whether the
// forward blended them.  Writes each fragment's merged fields to f0, f1.
template <int MODE>
__device__ __forceinline__ void back_pair(BackState& S, const RunStage& R, int k, bool c0, bool c1, x2f PXC, x2f PYC,
                                          const gs_config& cfg, float* f0, float* f1) {
    const x2f DX = x2_sub(PXC, x2_ld(R.x + k)), DY = x2_sub(PYC, x2_ld(R.y + k));
    const x2f CA = x2_ld(R.ca + k), CB = x2_ld(R.cb + k), CC = x2_ld(R.cc + k);
    const x2f A = x2_fma(CB, DY, x2_mul(CA, DX));  // Q d, as quad_form
    const x2f B = x2_fma(CC, DY, x2_mul(CB, DX));
    const x2f Q = x2_fma(DX, A, x2_mul(DY, B));
    float e0, e1;
    x2_unpack(x2_fma(Q, x2_pack(R_NEG_HALF_LOG2E, R_NEG_HALF_LOG2E), x2_ld(R.lop + k)), e0, e1);
    const float raw0 = exp2_sfu(e0), raw1 = exp2_sfu(e1);
    const float al0 = fminf(cfg.alpha_max, raw0), al1 = fminf(cfg.alpha_max, raw1);
    float d0, d1, r0, r1, g0, g1, b0, b1;
    x2_unpack(x2_ld(R.dep + k), d0, d1);
    x2_unpack(x2_ld(R.cr + k), r0, r1);
    x2_unpack(x2_ld(R.cg + k), g0, g1);
    x2_unpack(x2_ld(R.cl + k), b0, b1);
    const float cg0 = __fmaf_rn(d0, S.gD, __fmaf_rn(b0, S.gC2, __fmaf_rn(g0, S.gC1, r0 * S.gC0)));
    const float cg1 = __fmaf_rn(d1, S.gD, __fmaf_rn(b1, S.gC2, __fmaf_rn(g1, S.gC1, r1 * S.gC0)));
    S.T = c0 ? __fdividef(S.T, 1.f - al0) : S.T;
    const float T0 = S.T;
    const float w0 = c0 ? al0 * S.T : 0.f;
    const float dif0 = cg0 - S.sg;
    S.sg = c0 ? __fmaf_rn(al0, dif0, S.sg) : S.sg;
    S.T = c1 ? __fdividef(S.T, 1.f - al1) : S.T;
    const float T1 = S.T;
    const float w1 = c1 ? al1 * S.T : 0.f;
    const float dif1 = cg1 - S.sg;
    S.sg = c1 ? __fmaf_rn(al1, dif1, S.sg) : S.sg;
    // the clamp passes no gradient to opacity or shape
    const bool cl0 = raw0 > cfg.alpha_max, cl1 = raw1 > cfg.alpha_max;
    const x2f H = x2_mul(x2_pack(cl0 ? 0.f : -0.5f * w0, cl1 ? 0.f : -0.5f * w1), x2_pack(dif0, dif1));
    const x2f U = x2_mul(H, DX), V = x2_mul(H, DY);
    x2_unpack(x2_mul(A, H), f0[0], f1[0]);
    x2_unpack(x2_mul(B, H), f0[1], f1[1]);
    x2_unpack(x2_mul(U, DX), f0[2], f1[2]);
    x2_unpack(x2_mul(U, DY), f0[3], f1[3]);
    x2_unpack(x2_mul(V, DY), f0[4], f1[4]);
    if (MODE == GS_MAP) {
        float q0, q1;
        x2_unpack(Q, q0, q1);
        f0[5] = (c0 && !cl0) ? exp2_sfu(__fmul_rn(q0, R_NEG_HALF_LOG2E)) * (T0 * dif0) : 0.f;
        f1[5] = (c1 && !cl1) ? exp2_sfu(__fmul_rn(q1, R_NEG_HALF_LOG2E)) * (T1 * dif1) : 0.f;
        f0[6] = w0 * S.gD;
        f0[7] = w0 * S.gC0;
        f0[8] = w0 * S.gC1;
        f0[9] = w0 * S.gC2;
        f1[6] = w1 * S.gD;
        f1[7] = w1 * S.gC0;
        f1[8] = w1 * S.gC1;
        f1[9] = w1 * S.gC2;
    } else {
        f0[5] = w0 * S.gD;
        f1[5] = w1 * S.gD;
    }
}

// Backward compositing of one warp's block of a tile from the forward's
// per-pixel blend masks (warp w of the tile's).  Pixel-parallel tiles (EP
// false): the warp's 8x4 block, the masks in the run-major layout.
// Entry-parallel tiles of strided frames (EP true): the tile's sampled
// pixels 32 w .. 32 w + 31 in row-major order, the masks in the
// entry-parallel forward's pixel-major layout, whose words past a pixel's
// stopping batch were never written: each lane keeps only the bits before
// its own last blended position.  The warp walks its runs of 32 list
// entries from the last one holding an entry one of its pixels blended back
// to the first.  Per run it stages only those
// entries, one lane each (the record alone: no box, which the masks make
// unnecessary), the last first, then evaluates them back to front, 2 NP at
// a time in packed pairs; a lane's fragment counts when its own mask bit
// says the forward blended it, so both passes take identical decisions by
// construction, and the alpha it recomputes is the forward's (same staged
// values, same arithmetic).  The merged fields go straight to grad2d, one
// atomic per (entry, field, warp): the warps of a tile share nothing and run
// as one-warp CTAs that the hardware schedules as they free up, heavy tiles
// first.
template <int DT, int MODE, int NP, bool EP>
__device__ __forceinline__ void bwd_pw(const gs_config& cfg, const Grid& g, const void* __restrict__ splats,
                                       const uint32_t* __restrict__ vals, const uint32_t* __restrict__ ranges,
                                       const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                                       const float* __restrict__ d_rgb, const float* __restrict__ d_depth,
                                       float* __restrict__ grad2d, const uint32_t* __restrict__ bmask, int tile,
                                       int w, RunStage& R) {
    constexpr int NF = Fields<MODE>::N;
    constexpr int BSTEP = 2 * NP;  // entries per step, merged together
    static_assert(BSTEP * NF <= 32, "one lane per merged value");
    const int lane = threadIdx.x & 31;
    // slots past a run's entries are read by the last step's unused halves:
    // they must hold finite values (zeros, or an earlier run's records)
#pragma unroll
    for (int q = 0; q < (int)(sizeof(RunStage) / 4 / 32); ++q) (&R.x[0])[q * 32 + lane] = 0.f;
    __syncwarp();
    const int lt = w * 32 + lane;
    PixelMap m;
    if (EP) {
        int i, j;
        m.inside = ep_pixel(g, tile, lt, i, j);
        m.i = i;
        m.j = j;
        m.px = i * g.sx;
        m.py = j * g.sy;
    } else {
        m = map_pixel(g, tile, lt);
    }
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    BackState S;
    const uint32_t own = min(back_start(cfg, g, m, t_final, last_idx, d_rgb, d_depth, S), end - start);
    uint32_t last = own;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
    if (last == 0u) return;  // (warp-uniform) no pixel of the block blended anything
    const float pxc = (float)m.px + 0.5f, pyc = (float)m.py + 0.5f;
    const x2f PXC = x2_pack(pxc, pxc), PYC = x2_pack(pyc, pyc);
    const int owner = merge_owner<BSTEP * NF>();
    // this pixel's word of run r at bm[r rs]
    const uint32_t* bm = EP ? bmask + blend_mask_base_ep(tile, start) + (size_t)lt * ((end - start + 31) >> 5)
                            : bmask + blend_mask_base(tile, start) + lt;
    const size_t rs = EP ? 1 : (size_t)tile_threads(g);
    const int r_top = (int)((last + 31u) >> 5) - 1;
    // a run's list ids and mask word are loaded one run ahead (runs below
    // the top one are full: their 32 positions lie inside the list)
    uint32_t id_nx = r_top * 32 + lane < (int)(end - start)
                         ? __ldg(vals + start + (uint32_t)r_top * 32u + (uint32_t)lane)
                         : 0u;
    uint32_t bm_nx = __ldg(bm + (size_t)r_top * rs);
#pragma unroll 1
    for (int r = r_top; r >= 0; --r) {
        // only bits before the pixel's own last blended position count
        // (this also keeps masks from another forward from sending a load
        // outside the tile's list)
        const uint32_t lim = own > (uint32_t)r * 32u ? min(32u, own - (uint32_t)r * 32u) : 0u;
        const uint32_t mine = bm_nx & (lim == 32u ? ~0u : (1u << lim) - 1u);
        const uint32_t id = id_nx;
        if (r > 0) {
            id_nx = __ldg(vals + start + (uint32_t)(r - 1) * 32u + (uint32_t)lane);
            bm_nx = __ldg(bm + (size_t)(r - 1) * rs);
        }
        const unsigned mw = __reduce_or_sync(0xffffffffu, mine);
        if (mw == 0u) continue;
        // stage the run's blended entries: entry 32 r + lane into slot (its
        // rank from the top among the run's set bits)
        if ((mw >> lane) & 1u) {
            const int slot = __popc(mw & ~((2u << lane) - 1u));
            const Splat v = load_splat<DT>(splats, id);
            R.x[slot] = v.x;
            R.y[slot] = v.y;
            R.ca[slot] = v.ca;
            R.cb[slot] = v.cb;
            R.cc[slot] = v.cc;
            R.lop[slot] = log2_opacity(v.op);
            R.dep[slot] = v.depth;
            R.cr[slot] = v.r;
            R.cg[slot] = v.g;
            R.cl[slot] = v.b;
            R.id[slot] = id;
        }
        __syncwarp();
        unsigned mq = mw;
        for (int k = 0; mq; k += BSTEP) {
            bool cu[BSTEP], has[BSTEP];  // slot k + u: blended here, holds an entry
#pragma unroll
            for (int u = 0; u < BSTEP; ++u) {
                const int bit = mq ? 31 - __clz(mq) : -1;
                has[u] = bit >= 0;
                cu[u] = has[u] && ((mine >> (bit & 31)) & 1u);
                if (has[u]) mq &= ~(1u << bit);
            }
            float f[BSTEP * NF];
#pragma unroll
            for (int p = 0; p < NP; ++p)
                back_pair<MODE>(S, R, k + 2 * p, cu[2 * p], cu[2 * p + 1], PXC, PYC, cfg, f + 2 * p * NF,
                                f + (2 * p + 1) * NF);
            const float v = warp_merge<BSTEP * NF>(f);
            if (owner >= 0) {
                const int u = owner / NF, fl = owner - u * NF;
                bool valid = has[0];
#pragma unroll
                for (int x = 1; x < BSTEP; ++x) valid = u == x ? has[x] : valid;
                if (valid && v != 0.f)
                    atomicAdd(grad2d + (size_t)R.id[k + u] * GS_GRAD2D_STRIDE + field_col<MODE>(fl),
                              v * field_scale(fl));
            }
        }
        __syncwarp();  // the next run reuses the slots
    }
}

// Pairs per step of the masked backward: two for the pose-only fields (24
// merged values; 98.0-98.7 us against 99.0 with one pair, and 99.0 for three
// unpacked entries), one when mapping (20).
template <int MODE>
struct PwPairs {
    static constexpr int N = MODE == GS_TRACK ? 2 : 1;
};

// One-warp CTAs: 32 per SM at 64 registers for the pose-only fields; 24 when
// mapping.
// Warps per tile of the masked backward.
__host__ __device__ inline int pw_warps(const Grid& g, bool ep) {
    return ep ? (g.tw * g.th + 31) >> 5 : tile_threads(g) >> 5;
}

template <int DT, int MODE, bool EP>
__global__ void __launch_bounds__(32, MODE == GS_TRACK ? 32 : 24)
    k_render_bwd_pw(gs_config cfg, Grid g, const void* __restrict__ splats, const uint32_t* __restrict__ vals,
                    const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ order,
                    const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                    const float* __restrict__ d_rgb, const float* __restrict__ d_depth, float* __restrict__ grad2d,
                    const uint32_t* __restrict__ bmask) {
    __shared__ RunStage R;
    const int wpt = pw_warps(g, EP);
    const int t = (int)blockIdx.x / wpt, w = (int)blockIdx.x % wpt;
    const int tile = order ? (int)__ldg(order + t) : t;
    bwd_pw<DT, MODE, PwPairs<MODE>::N, EP>(cfg, g, splats, vals, ranges, t_final, last_idx, d_rgb, d_depth,
                                           grad2d, bmask, tile, w, R);
}

// ---------------------------------------------------------------------------
// Entry-parallel compositing for the small tiles of downsampled frames
// ---------------------------------------------------------------------------
// With both strides >= 2 a tile holds at most 8x8 sampled pixels but covers
// the same full-resolution area, hence the same list length, as a 16x16
// tile: pixel-parallel warps would walk long lists with few (and far apart)
// pixels.  Here one CTA of W warps serves a tile (W = 8 for up to 32
// pixels, else 16) and warp w takes PPW = ceil(pixels / W) of its pixels
// (2 to 4), one at a time.  For its pixel the warp first compacts the staged
// entries whose pixel box contains it (a ballot per 32 entries, in list
// order), then lane l takes the l-th compacted entry.  Front-to-back
// compositing (Eq. 3) becomes a product scan: the transmittance before a
// valid entry is the pixel's T times the product of (1 - alpha) over the
// valid entries before it in the group of 32; the pixel stops at the first
// valid entry that would take T below t_eps.  The backward (Eq. 4, Eq. 5)
// compacts from the pixel's last blended entry back: T before an entry is T
// behind the group divided by the product of (1 - alpha) over it and the
// entries behind it, and the colour behind it is a prefix sum, so
//     dL/dalpha_k = T_k (c_k . g) - (sum_{j>k} w_j c_j . g + T_N bg . g) / (1 - alpha_k)
// with g the pixel's image gradient; each lane adds its entry's gradient to
// the tile's shared accumulators.  Entries are staged as four 16-byte arrays
// (lane l reading element l is conflict-free).
#define EP_B 256     // entries staged per batch (the forward of 64-pixel
                     // tiles stages 512: fewer CTA barriers per list)

template <int NB>
struct EpStageN {
    float4 a[NB];    // x, y, conic_a, conic_b
    float4 b[NB];    // conic_c, opacity, depth, -
    float4 c[NB];    // r, g, b, -
    int4 box[NB];    // pixel box
};
typedef EpStageN<EP_B> EpStage;

template <int W>
struct EpFwdBatch {
    static constexpr int N = W == 16 ? 2 * EP_B : EP_B;
};

template <int DT, int W, int NB>
__device__ __forceinline__ void ep_stage(const void* __restrict__ splats, const uint32_t* __restrict__ ids, int n_in,
                                         float alpha_min, EpStageN<NB>& S, uint32_t* sid) {
    for (int e = threadIdx.x; e < n_in; e += W * 32) {
        const uint32_t id = __ldg(ids + e);
        const Splat v = load_splat<DT>(splats, id);
        S.a[e] = make_float4(v.x, v.y, v.ca, v.cb);
        S.b[e] = make_float4(v.cc, v.op, v.depth, log2_opacity(v.op));
        float t2;
        S.box[e] = pixel_box(v, alpha_min, t2);
        S.c[e] = make_float4(v.r, v.g, v.b, 0.f);
        if (sid) sid[e] = id;
    }
}

// Whether staged entry e can blend at full-resolution pixel (px, py): inside
// its pixel box (a superset of the fragments the alpha test accepts, so
// compacting by it changes no result).  Testing the alpha ellipse here as
// well was measured slower: the extra loads cost more than the groups saved.
template <int NB>
__device__ __forceinline__ bool ep_may_blend(const EpStageN<NB>& S, int e, int px, int py) {
    const int4 box = S.box[e];
    return px >= box.x && px <= box.y && py >= box.z && py <= box.w;
}


// Pixel-to-warp assignment of a tile (the pairing of Sec. 5.2's workload
// scheduling unit): the tile's npix = W * ppw pixels are ranked by their
// expected work h (heaviest first, ties by index) and dealt to the W warps
// in snake order, round r going to warps 0..W-1 for even r and W-1..0 for
// odd r, so each warp gets a heavy pixel with a light one in every pair of
// rounds.  h is the pixel's list position of the last blended entry (the
// backward's input, or the previous iteration's for the forward); pixels
// outside the image have h = 0.  perm[w * ppw + j] is warp w's j-th pixel.
// Any h gives a valid permutation; it only changes which warp does what.
template <int W>
__device__ __forceinline__ void ep_pair(const Grid& g, int tile, int q0, int npix, const uint32_t* hint,
                                        uint32_t* s_h, uint8_t* perm) {
    const int ppw = (npix + W - 1) / W;
    const int q = (int)threadIdx.x;
    if (q < npix) {
        int i, j;
        uint32_t h = 0;
        if (hint && ep_pixel(g, tile, q0 + q, i, j)) h = hint[(size_t)j * g.Ws + i];
        s_h[q] = h;
    }
    __syncthreads();
    if (q < npix) {
        const uint32_t h = s_h[q];
        int r = 0;
        for (int o = 0; o < npix; ++o) {
            const uint32_t v = s_h[o];
            r += (v > h || (v == h && o < q)) ? 1 : 0;
        }
        const int round = r / W, pos = r % W;
        const int w = (round & 1) ? W - 1 - pos : pos;
        perm[w * ppw + round] = (uint8_t)q;
    }
    __syncthreads();
}

// Forward compositing of pixels q0 .. q0 + npix - 1 of `tile` by the CTA's W
// warps, entry-parallel (S: staging; cbuf_all: W compaction buffers).
template <int DT, int W>
__device__ __forceinline__ void fwd_ep(const gs_config& cfg, const Grid& g, const void* __restrict__ splats,
                                       const uint32_t* __restrict__ vals, const uint32_t* __restrict__ ranges,
                                       const FwdOut& O, int tile, int q0, int npix, EpStageN<EpFwdBatch<W>::N>& S,
                                       int (*cbuf_all)[64], uint32_t* s_h, uint8_t* perm,
                                       uint32_t (*bm_all)[EpFwdBatch<W>::N / 32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    int* cbuf = cbuf_all[warp];
    const int ppw = (npix + W - 1) / W;
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    // out_last still holds the previous iteration's positions (read before any write)
    ep_pair<W>(g, tile, q0, npix, cfg.balance ? O.last : nullptr, s_h, perm);
    // lane j < ppw holds the state of the warp's pixel j
    int mi, mj;
    const bool mine = lane < ppw && warp * ppw + lane < npix && ep_pixel(g, tile, q0 + perm[warp * ppw + lane], mi, mj);
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    uint32_t last = 0, nb = 0;
    bool done = !mine;
    constexpr int NB = EpFwdBatch<W>::N;
    uint32_t* bmw = bm_all[warp];  // the pixel's blend mask over the batch
    const uint32_t nw = (end - start + 31) >> 5;
    const size_t bm_tile = blend_mask_base_ep(tile, start);
    for (uint32_t b = start; b < end; b += NB) {
        if (__syncthreads_count(!done) == 0) break;
        const int n_in = (int)min((uint32_t)NB, end - b);
        ep_stage<DT, W, NB>(splats, vals + b, n_in, cfg.alpha_min, S, nullptr);
        __syncthreads();
        for (int j = 0; j < ppw; ++j) {
            if (__shfl_sync(0xffffffffu, done, j)) continue;
            int pi, pj;
            ep_pixel(g, tile, q0 + perm[warp * ppw + j], pi, pj);
            const int px = pi * g.sx, py = pj * g.sy;
            const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
            float Tj = __shfl_sync(0xffffffffu, T, j);
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, pd = 0.f;
            uint32_t lastj = 0, nbj = 0;
            bool stopped = false;
            if (O.bmask) {
                if (lane < NB / 32) bmw[lane] = 0u;
                __syncwarp();
            }
            // composite the k compacted entries cbuf[0, k), in list order
            auto composite = [&](int k) {
                const int e = lane < k ? cbuf[lane] : -1;
                float alpha = -1.f;
                if (e >= 0) {
                    const float4 A = S.a[e];
                    const float4 Bv = S.b[e];
                    const Quad Qd = quad_form(A.z, A.w, Bv.x, pxc - A.x, pyc - A.y);
                    const float al = fminf(cfg.alpha_max, raw_alpha(Qd.q, Bv.w));
                    if (!(Qd.q < 0.f)) alpha = al;
                }
                const bool valid = alpha >= cfg.alpha_min;
                if (__ballot_sync(0xffffffffu, valid) == 0u) return;
                const float f = valid ? 1.f - alpha : 1.f;
                float P = f;  // inclusive product over lanes 0..l
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y = __shfl_up_sync(0xffffffffu, P, o);
                    if (lane >= o) P *= y;
                }
                float Tb = __shfl_up_sync(0xffffffffu, P, 1);  // T before this entry
                Tb = lane == 0 ? Tj : Tj * Tb;
                const float Tn = Tb * f;
                const unsigned stop = __ballot_sync(0xffffffffu, valid && Tn < cfg.t_eps);
                const int lstar = stop ? __ffs(stop) - 1 : 32;
                const bool ok = valid && lane < lstar;
                if (ok) {
                    const float w = alpha * Tb;
                    const float4 Cc = S.c[e];
                    p0 += w * Cc.x;
                    p1 += w * Cc.y;
                    p2 += w * Cc.z;
                    pd += w * S.b[e].z;
                }
                const unsigned okm = __ballot_sync(0xffffffffu, ok);
                nbj += __popc(okm);
                if (O.bmask && ok) atomicOr(&bmw[e >> 5], 1u << (e & 31));
                const int ehi = __shfl_sync(0xffffffffu, e, okm ? 31 - __clz(okm) : 0);
                if (okm) lastj = b - start + (uint32_t)ehi + 1u;
                if (lstar < 32) {
                    Tj = __shfl_sync(0xffffffffu, Tb, lstar);
                    stopped = true;
                } else {
                    Tj = __shfl_sync(0xffffffffu, Tn, 31);
                }
            };
            int cnt = 0;
            for (int c = 0; c < n_in && !stopped; c += 32) {
                const int e = c + lane;
                const bool in = e < n_in && ep_may_blend(S, e, px, py);
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (in) cbuf[cnt + __popc(m & lt_mask)] = e;
                cnt += __popc(m);
                __syncwarp();
                if (cnt >= 32) {
                    composite(32);
                    const int rest = cnt - 32;
                    const int v = lane < rest ? cbuf[32 + lane] : 0;
                    __syncwarp();
                    if (lane < rest) cbuf[lane] = v;
                    __syncwarp();
                    cnt = rest;
                }
            }
            if (!stopped && cnt > 0) composite(cnt);
            __syncwarp();
            if (O.bmask && lane < ((n_in + 31) >> 5))
                O.bmask[bm_tile + (size_t)(q0 + perm[warp * ppw + j]) * nw + ((b - start) >> 5) + lane] = bmw[lane];
            p0 = warp_sum(p0);
            p1 = warp_sum(p1);
            p2 = warp_sum(p2);
            pd = warp_sum(pd);
            if (lane == j) {
                C0 += p0;
                C1 += p1;
                C2 += p2;
                D += pd;
                T = Tj;
                if (lastj) last = lastj;
                nb += nbj;
                done = stopped;
            }
        }
        __syncthreads();
    }
    float lpart = 0.f;
    if (mine) lpart = write_pixel(cfg, g, O, mi, mj, C0, C1, C2, D, T, last, nb);
    add_loss(O, lpart);
}

template <int DT, int W>
__global__ void __launch_bounds__(W * 32, W == 8 ? 4 : 2)
    k_render_fwd_ep(gs_config cfg, Grid g, const void* __restrict__ splats, const uint32_t* __restrict__ vals,
                    const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ order, FwdOut O) {
    __shared__ EpStageN<EpFwdBatch<W>::N> S;
    __shared__ int cbuf_all[W][64];
    __shared__ uint32_t s_h[64];
    __shared__ uint8_t perm[64];
    __shared__ uint32_t bm_all[W][EpFwdBatch<W>::N / 32];
    const int tile = order ? (int)__ldg(order + blockIdx.x) : (int)blockIdx.x;
    fwd_ep<DT, W>(cfg, g, splats, vals, ranges, O, tile, 0, g.tw * g.th, S, cbuf_all, s_h, perm, bm_all);
}

// Fields merged per entry: GS_TRACK du dv dA dB dC dd, GS_MAP du dv dA dB dC
// dop dd dr dg db; ep_col gives their grad2d columns.
template <int MODE>
struct EpFields {
    static constexpr int N = MODE == GS_MAP ? 10 : 6;
};
template <int MODE>
__device__ __forceinline__ int ep_col(int f) {
    if (MODE == GS_MAP) return f < 7 ? f : f + 1;
    return f < 5 ? f : 6;
}

// Shared memory of the entry-parallel backward (batches of NB entries;
// dynamic: above 48 KB for 16 warps and 512 entries).
template <int MODE, int W, int NB = EpFwdBatch<W>::N>
struct EpBwdSmem {
    EpStageN<NB> S;
    uint32_t sid[NB];
    float acc[EpFields<MODE>::N][NB];
    int cbuf[W][64];
    uint32_t s_h[64];
    uint8_t perm[64];
    uint32_t s_max;
};

// Backward compositing of pixels q0 .. q0 + npix - 1 of `tile` by the CTA's
// W warps, entry-parallel.
template <int DT, int MODE, int W>
__device__ __forceinline__ void bwd_ep(const gs_config& cfg, const Grid& g, const void* __restrict__ splats,
                                       const uint32_t* __restrict__ vals, const uint32_t* __restrict__ ranges,
                                       const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                                       const float* __restrict__ d_rgb, const float* __restrict__ d_depth,
                                       float* __restrict__ grad2d, const uint32_t* __restrict__ bmask, int tile,
                                       int q0, int npix, EpBwdSmem<MODE, W>& M) {
    constexpr int NF = EpFields<MODE>::N;
    constexpr int NB = EpFwdBatch<W>::N;
    EpStageN<NB>& S = M.S;
    uint32_t* sid = M.sid;
    float(&acc)[NF][NB] = M.acc;
    uint32_t& s_max = M.s_max;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned gt_mask = lane == 31 ? 0u : ~0u << (lane + 1);
    int* cbuf = M.cbuf[warp];
    const int ppw = (npix + W - 1) / W;
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    uint8_t* perm = M.perm;
    ep_pair<W>(g, tile, q0, npix, last_idx, M.s_h, perm);
    int mi, mj;
    const bool mine = lane < ppw && warp * ppw + lane < npix && ep_pixel(g, tile, q0 + perm[warp * ppw + lane], mi, mj);
    // state of pixel `lane`: T after the part already walked, the colour
    // behind it dotted with g, last blended position, image gradient g
    float T = 1.f, sdot = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, gd = 0.f;
    uint32_t last = 0;
    if (mine) {
        const size_t P = (size_t)g.Ws * g.Hs;
        const size_t pix = (size_t)mj * g.Ws + mi;
        T = t_final[pix];
        last = min(last_idx[pix], end - start);
        g0 = d_rgb[pix];
        g1 = d_rgb[P + pix];
        g2 = d_rgb[2 * P + pix];
        gd = d_depth[pix];
        sdot = T * (cfg.bg[0] * g0 + cfg.bg[1] * g1 + cfg.bg[2] * g2);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    uint32_t wl = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    if (lane == 0) atomicMax(&s_max, wl);
    __syncthreads();
    const uint32_t tile_last = s_max;
    const uint32_t nw = (end - start + 31) >> 5;
    const uint32_t* bm_tile = bmask ? bmask + blend_mask_base_ep(tile, start) : nullptr;
    // batches [start + k NB, start + (k + 1) NB) from the last one holding a
    // blended entry back to the first
    for (int kb = (int)((tile_last + NB - 1) / NB) - 1; kb >= 0; --kb) {
        const uint32_t lo = start + (uint32_t)kb * NB, hi = start + min(tile_last, (uint32_t)(kb + 1) * NB);
        const int n_in = (int)(hi - lo);
        ep_stage<DT, W, NB>(splats, vals + lo, n_in, cfg.alpha_min, S, sid);
        for (int q = threadIdx.x; q < NF * NB; q += W * 32) (&acc[0][0])[q] = 0.f;
        __syncthreads();
        const uint32_t base_pos = lo - start;
        for (int j = 0; j < ppw; ++j) {
            const uint32_t lastj = __shfl_sync(0xffffffffu, last, j);
            if (lastj <= base_pos) continue;  // nothing blended in this batch
            const int nj = (int)min((uint32_t)n_in, lastj - base_pos);
            const int qj = q0 + perm[warp * ppw + j];  // the pixel's index in the tile
            int pi, pj;
            ep_pixel(g, tile, qj, pi, pj);
            const int px = pi * g.sx, py = pj * g.sy;
            const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
            // the pixel's blend mask from the forward (entries it blended),
            // else its pixel box, selects the entries to compact
            const uint32_t* bmj = bm_tile ? bm_tile + (size_t)qj * nw + (base_pos >> 5) : nullptr;
            float Tj = __shfl_sync(0xffffffffu, T, j);
            float sj = __shfl_sync(0xffffffffu, sdot, j);
            // the pixel's image gradient
            const float h0 = __shfl_sync(0xffffffffu, g0, j), h1 = __shfl_sync(0xffffffffu, g1, j);
            const float h2 = __shfl_sync(0xffffffffu, g2, j), hd = __shfl_sync(0xffffffffu, gd, j);
            // the k compacted entries cbuf[0, k), last first: lane l's entry
            // has the entries of lanes < l behind it
            auto differentiate = [&](int k) {
                const int e = lane < k ? cbuf[lane] : -1;
                float4 Bv = make_float4(0.f, 0.f, 0.f, 0.f), Cc = Bv;
                float dx = 0.f, dy = 0.f, raw = 0.f, alpha = -1.f;
                Quad Qd = {0.f, 0.f, 0.f};
                bool valid = false;
                if (e >= 0) {
                    const float4 A = S.a[e];
                    Bv = S.b[e];
                    Cc = S.c[e];
                    dx = pxc - A.x;
                    dy = pyc - A.y;
                    Qd = quad_form(A.z, A.w, Bv.x, dx, dy);
                    raw = raw_alpha(Qd.q, Bv.w);
                    alpha = fminf(cfg.alpha_max, raw);
                    valid = !(Qd.q < 0.f) && !(alpha < cfg.alpha_min);
                }
                if (__ballot_sync(0xffffffffu, valid) == 0u) return;
                const float f = valid ? 1.f - alpha : 1.f;
                float Q = f;  // inclusive product over lanes 0..l (this entry and those behind it)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y = __shfl_up_sync(0xffffffffu, Q, o);
                    if (lane >= o) Q *= y;
                }
                const float Tb = __fdividef(Tj, Q);  // T before this entry (Eq. 5)
                const float w = valid ? alpha * Tb : 0.f;
                const float cg = Cc.x * h0 + Cc.y * h1 + Cc.z * h2 + Bv.z * hd;
                const float wcg = w * cg;
                float Sin = wcg;  // inclusive prefix sum of w (c . g)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y = __shfl_up_sync(0xffffffffu, Sin, o);
                    if (lane >= o) Sin += y;
                }
                if (valid) {
                    const float behind = sj + (Sin - wcg);
                    const float dLda = Tb * cg - __fdividef(behind, f);
                    float ga[NF];
#pragma unroll
                    for (int q = 0; q < NF; ++q) ga[q] = 0.f;
                    if (MODE == GS_MAP) {
                        ga[6] = w * hd;
                        ga[7] = w * h0;
                        ga[8] = w * h1;
                        ga[9] = w * h2;
                    } else {
                        ga[5] = w * hd;
                    }
                    if (!(raw > cfg.alpha_max)) {  // the clamp passes no gradient
                        if (MODE == GS_MAP) ga[5] = exp2_sfu(__fmul_rn(Qd.q, R_NEG_HALF_LOG2E)) * dLda;
                        const float dp = alpha * dLda;
                        ga[2] = -0.5f * dx * dx * dp;
                        ga[3] = -dx * dy * dp;
                        ga[4] = -0.5f * dy * dy * dp;
                        ga[0] = Qd.a * dp;
                        ga[1] = Qd.b * dp;
                    }
#pragma unroll
                    for (int q = 0; q < NF; ++q)
                        if (ga[q] != 0.f) atomicAdd(&acc[q][e], ga[q]);
                }
                // state in front of these entries
                Tj = __shfl_sync(0xffffffffu, __fdividef(Tj, Q), 31);
                sj = sj + __shfl_sync(0xffffffffu, Sin, 31);
            };
            int cnt = 0;
            for (int c = (nj - 1) & ~31; c >= 0; c -= 32) {
                const int e = c + lane;
                const bool in = e < nj && (bmj ? ((__ldg(bmj + (c >> 5)) >> lane) & 1u) != 0u : ep_may_blend(S, e, px, py));
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (in) cbuf[cnt + __popc(m & gt_mask)] = e;
                cnt += __popc(m);
                __syncwarp();
                if (cnt >= 32) {
                    differentiate(32);
                    const int rest = cnt - 32;
                    const int v = lane < rest ? cbuf[32 + lane] : 0;
                    __syncwarp();
                    if (lane < rest) cbuf[lane] = v;
                    __syncwarp();
                    cnt = rest;
                }
            }
            if (cnt > 0) differentiate(cnt);
            __syncwarp();
            if (lane == j) {
                T = Tj;
                sdot = sj;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n_in; e += W * 32) {
            float* dst = grad2d + (size_t)sid[e] * GS_GRAD2D_STRIDE;
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                const float v = acc[k][e];
                if (v != 0.f) atomicAdd(dst + ep_col<MODE>(k), v);
            }
        }
        __syncthreads();
    }
}

template <int DT, int MODE, int W>
__global__ void __launch_bounds__(W * 32, W == 8 ? 4 : 2)
    k_render_bwd_ep(gs_config cfg, Grid g, const void* __restrict__ splats, const uint32_t* __restrict__ vals,
                    const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ order,
                    const float* __restrict__ t_final, const uint32_t* __restrict__ last_idx,
                    const float* __restrict__ d_rgb, const float* __restrict__ d_depth,
                    float* __restrict__ grad2d, const uint32_t* __restrict__ bmask) {
    extern __shared__ __align__(16) unsigned char r_smem[];
    EpBwdSmem<MODE, W>& M = *reinterpret_cast<EpBwdSmem<MODE, W>*>(r_smem);
    const int tile = order ? (int)__ldg(order + blockIdx.x) : (int)blockIdx.x;
    bwd_ep<DT, MODE, W>(cfg, g, splats, vals, ranges, t_final, last_idx, d_rgb, d_depth, grad2d, bmask, tile, 0,
                        g.tw * g.th, M);
}

// ---------------------------------------------------------------------------
// Multi-session waves: forward compositing with the loss and backward
// compositing (GS_TRACK) over every job of a wave, one launch per kernel form
// ---------------------------------------------------------------------------
struct WaveFwdJob {
    Grid g;
    const void* splats;
    const uint32_t* vals;
    const uint32_t* ranges;
    const uint32_t* order;
    FwdOut O;
    int B;
};

template <int KST>
__global__ void __launch_bounds__(R_THREADS, KST == 1 ? 4 : 2)
    k_wave_render_fwd(const gs_config cfg, const __grid_constant__ Wave<WaveFwdJob> W) {
    extern __shared__ __align__(16) unsigned char r_smem[];
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveFwdJob& J = W.job[j];
    const Group G = make_group(J.g, J.order, J.B, (int)blockIdx.x - W.start[j]);
    if (G.tile < 0) return;
    fwd_pp<GS_F32, KST>(cfg, J.g, J.splats, J.vals, J.ranges, J.O, G, reinterpret_cast<StagedSplat*>(r_smem));
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 4 : 2)
    k_wave_render_fwd_ep(const gs_config cfg, const __grid_constant__ Wave<WaveFwdJob> W) {
    __shared__ EpStageN<EpFwdBatch<NW>::N> S;
    __shared__ int cbuf_all[NW][64];
    __shared__ uint32_t s_h[64];
    __shared__ uint8_t perm[64];
    __shared__ uint32_t bm_all[NW][EpFwdBatch<NW>::N / 32];
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveFwdJob& J = W.job[j];
    const int blk = (int)blockIdx.x - W.start[j];
    const int tile = J.order ? (int)__ldg(J.order + blk) : blk;
    fwd_ep<GS_F32, NW>(cfg, J.g, J.splats, J.vals, J.ranges, J.O, tile, 0, J.g.tw * J.g.th, S, cbuf_all, s_h, perm,
                       bm_all);
}

struct WaveBwdJob {
    Grid g;
    const void* splats;
    const uint32_t* vals;
    const uint32_t* ranges;
    const uint32_t* order;
    const float* t_final;
    const uint32_t* last_idx;
    const float* d_rgb;
    const float* d_depth;
    float* grad2d;
    const uint32_t* bmask;
    int B;
};

template <int KST>
__global__ void __launch_bounds__(R_THREADS, KST == 1 ? 4 : 2)
    k_wave_render_bwd(const gs_config cfg, const __grid_constant__ Wave<WaveBwdJob> W) {
    extern __shared__ __align__(16) unsigned char r_smem[];
    __shared__ uint32_t s_max_all[R_THREADS / 32];
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveBwdJob& J = W.job[j];
    const Group G = make_group(J.g, J.order, J.B, (int)blockIdx.x - W.start[j]);
    if (G.tile < 0) return;
    bwd_pp<GS_F32, GS_TRACK, KST>(cfg, J.g, J.splats, J.vals, J.ranges, J.t_final, J.last_idx, J.d_rgb, J.d_depth,
                                  J.grad2d, G, r_smem, s_max_all);
}

// Jobs with blend masks: one-warp CTAs over (job, tile, warp).
template <bool EP>
__global__ void __launch_bounds__(32, 32) k_wave_render_bwd_pw(const gs_config cfg,
                                                                const __grid_constant__ Wave<WaveBwdJob> W) {
    __shared__ RunStage R;
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveBwdJob& J = W.job[j];
    const int blk = (int)blockIdx.x - W.start[j];
    const int wpt = pw_warps(J.g, EP);
    const int t = blk / wpt, w = blk % wpt;
    const int tile = J.order ? (int)__ldg(J.order + t) : t;
    bwd_pw<GS_F32, GS_TRACK, PwPairs<GS_TRACK>::N, EP>(cfg, J.g, J.splats, J.vals, J.ranges, J.t_final, J.last_idx,
                                                        J.d_rgb, J.d_depth, J.grad2d, J.bmask, tile, w, R);
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 4 : 2)
    k_wave_render_bwd_ep(const gs_config cfg, const __grid_constant__ Wave<WaveBwdJob> W) {
    extern __shared__ __align__(16) unsigned char r_smem[];
    EpBwdSmem<GS_TRACK, NW>& M = *reinterpret_cast<EpBwdSmem<GS_TRACK, NW>*>(r_smem);
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveBwdJob& J = W.job[j];
    const int blk = (int)blockIdx.x - W.start[j];
    const int tile = J.order ? (int)__ldg(J.order + blk) : blk;
    bwd_ep<GS_F32, GS_TRACK, NW>(cfg, J.g, J.splats, J.vals, J.ranges, J.t_final, J.last_idx, J.d_rgb, J.d_depth,
                                 J.grad2d, J.bmask, tile, 0, J.g.tw * J.g.th, M);
}

}  // namespace gs

using namespace gs;

// Entries a tile stages per batch: R_BATCH, halved while the CTA's tiles
// would need more than `budget` bytes of shared memory.
static int group_batch(int gpc, int bytes_per_entry, int budget) {
    int B = R_BATCH;
    while (B > 32 && gpc * B * bytes_per_entry > budget) B >>= 1;
    return B;
}

// The forward's batch: the most entries (a multiple of 32, at most R_BATCH)
// whose records fit the forward budget for the CTA's gpc tiles.
static int fwd_batch(int gpc) {
    const int B = R_FWD_SMEM / (gpc * (int)sizeof(StagedSplat)) / 32 * 32;
    return B < 32 ? 32 : (B > R_BATCH ? R_BATCH : B);
}

// Raises a kernel's dynamic shared-memory limit once per device and
// instantiation (not repeated while a graph is being captured).
static gs_status smem_once(const void* fn, int id, int bytes) {
    static bool done[64][48] = {};  // ids: fwd 0-5, bwd 6-17, entry-parallel bwd 18-33, waves 40-45
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && done[dev][id]) return GS_OK;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "cudaFuncSetAttribute(render kernel %d)", id);
    if (dev >= 0 && dev < 64) done[dev][id] = true;
    return GS_OK;
}

// Kernel choice per frame (the results agree to float32 summation order):
// both strides >= 2 (tiles of at most 64 sampled pixels): entry-parallel,
// one CTA of 8 or 16 warps per tile; otherwise pixel-parallel groups.
template <int DT>
static gs_status launch_fwd(const gs_config& cfg, const Grid& g, const void* splats, const uint32_t* vals,
                            const uint32_t* ranges, const uint32_t* order, const FwdOut& O, cudaStream_t st) {
    const int ntiles = g.TX * g.TY;
    if (g.tw * g.th <= 64) {
        if (g.tw * g.th <= 32)
            k_render_fwd_ep<DT, 8><<<ntiles, 8 * 32, 0, st>>>(cfg, g, splats, vals, ranges, order, O);
        else
            k_render_fwd_ep<DT, 16><<<ntiles, 16 * 32, 0, st>>>(cfg, g, splats, vals, ranges, order, O);
        return check_launch("k_render_fwd_ep");
    }
    const int gpc = R_THREADS / tile_threads(g);
    const unsigned nt = (unsigned)((ntiles + gpc - 1) / gpc);
    const int B = fwd_batch(gpc);
    const size_t smem = (size_t)gpc * (B / 32 * 33) * sizeof(StagedSplat);  // + a dummy per 32
    gs_status s;
    if (gpc == 1) {
        if ((s = smem_once((const void*)k_render_fwd<DT, 1>, 2 * DT, R_FWD_SMEM / 32 * 33)) != GS_OK) return s;
        k_render_fwd<DT, 1><<<nt, R_THREADS, smem, st>>>(cfg, g, splats, vals, ranges, order, O, B);
    } else {
        if ((s = smem_once((const void*)k_render_fwd<DT, 4>, 2 * DT + 1, R_FWD_SMEM / 32 * 33)) != GS_OK) return s;
        k_render_fwd<DT, 4><<<nt, R_THREADS, smem, st>>>(cfg, g, splats, vals, ranges, order, O, B);
    }
    return check_launch("k_render_fwd");
}

static gs_status dispatch_fwd(const gs_config& cfg, const Grid& g, int rec_dtype, const void* splats,
                              const uint32_t* vals, const uint32_t* ranges, const uint32_t* order, const FwdOut& O,
                              cudaStream_t st) {
    if (rec_dtype == GS_F32) return launch_fwd<GS_F32>(cfg, g, splats, vals, ranges, order, O, st);
    if (rec_dtype == GS_BF16) return launch_fwd<GS_BF16>(cfg, g, splats, vals, ranges, order, O, st);
    return launch_fwd<GS_F16>(cfg, g, splats, vals, ranges, order, O, st);
}

template <int DT, int MD>
static gs_status launch_bwd(const gs_config& cfg, const Grid& g, const void* splats, const uint32_t* vals,
                            const uint32_t* ranges, const uint32_t* order, const float* t_final,
                            const uint32_t* last_idx, const float* d_rgb, const float* d_depth, float* grad2d,
                            const uint32_t* bmask, cudaStream_t st) {
    const int ntiles = g.TX * g.TY;
    const bool ep = g.tw * g.th <= 64;
    // with masks: one-warp CTAs for pixel-parallel tiles and for the 64-pixel
    // tiles of strided frames (stride 2: 64 -> 90 us in the entry-parallel
    // kernel; the 16- and 32-pixel tiles of larger strides half-fill or
    // spread a warp and stay entry-parallel: 38 against 60 us at 4x4)
    if (bmask && (!ep || g.tw * g.th == 64)) {
        const unsigned nw = (unsigned)ntiles * (unsigned)pw_warps(g, ep);
        if (ep)
            k_render_bwd_pw<DT, MD, true><<<nw, 32, 0, st>>>(cfg, g, splats, vals, ranges, order, t_final, last_idx,
                                                              d_rgb, d_depth, grad2d, bmask);
        else
            k_render_bwd_pw<DT, MD, false><<<nw, 32, 0, st>>>(cfg, g, splats, vals, ranges, order, t_final, last_idx,
                                                               d_rgb, d_depth, grad2d, bmask);
        return check_launch("k_render_bwd_pw");
    }
    if (ep) {
        gs_status s;
        const int id = 18 + 4 * (MD == GS_MAP) + DT;  // + 0 or 8 below: W
        if (g.tw * g.th <= 32) {
            const int sm = (int)sizeof(EpBwdSmem<MD, 8>);
            if ((s = smem_once((const void*)k_render_bwd_ep<DT, MD, 8>, id, sm)) != GS_OK) return s;
            k_render_bwd_ep<DT, MD, 8><<<ntiles, 8 * 32, sm, st>>>(cfg, g, splats, vals, ranges, order, t_final,
                                                                    last_idx, d_rgb, d_depth, grad2d, bmask);
        } else {
            const int sm = (int)sizeof(EpBwdSmem<MD, 16>);
            if ((s = smem_once((const void*)k_render_bwd_ep<DT, MD, 16>, id + 8, sm)) != GS_OK) return s;
            k_render_bwd_ep<DT, MD, 16><<<ntiles, 16 * 32, sm, st>>>(cfg, g, splats, vals, ranges, order,
                                                                      t_final, last_idx, d_rgb, d_depth, grad2d,
                                                                      bmask);
        }
        return check_launch("k_render_bwd_ep");
    }
    const int gpc = R_THREADS / tile_threads(g);
    const unsigned nt = (unsigned)((ntiles + gpc - 1) / gpc);
    const int per_entry = (int)(sizeof(StagedSplat) + sizeof(uint32_t) + sizeof(float) * Fields<MD>::N);
    const int B = group_batch(gpc, per_entry, R_BWD_SMEM);
    const size_t smem = (size_t)gpc * B * per_entry;
    const int id = 6 + 6 * (MD == GS_MAP) + 2 * DT;
    gs_status s;
    if (gpc == 1) {
        if ((s = smem_once((const void*)k_render_bwd<DT, MD, 1>, id, R_BWD_SMEM)) != GS_OK) return s;
        k_render_bwd<DT, MD, 1><<<nt, R_THREADS, smem, st>>>(cfg, g, splats, vals, ranges, order, t_final,
                                                             last_idx, d_rgb, d_depth, grad2d, B);
    } else {
        if ((s = smem_once((const void*)k_render_bwd<DT, MD, 4>, id + 1, R_BWD_SMEM)) != GS_OK) return s;
        k_render_bwd<DT, MD, 4><<<nt, R_THREADS, smem, st>>>(cfg, g, splats, vals, ranges, order, t_final,
                                                             last_idx, d_rgb, d_depth, grad2d, B);
    }
    return check_launch("k_render_bwd");
}

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
                                   uint32_t* last_idx, uint32_t* n_blended, uint32_t* blend_masks,
                                   gs_stream stream) {
    gs_status s;
    if ((s = render_checks(cfg, cam, rec_dtype, splats, n)) != GS_OK) return s;
    if (!tile_ranges || !rgb || !depth || !t_final || !last_idx)
        return set_error(GS_ERR_INVALID_ARG, "an image or range pointer is NULL");
    const FwdOut O = {rgb, depth, t_final, last_idx, n_blended, nullptr, nullptr, nullptr, nullptr, nullptr,
                      blend_masks};
    return dispatch_fwd(*cfg, make_grid(*cam), rec_dtype, splats, vals, tile_ranges, tile_order, O,
                        (cudaStream_t)stream);
}

extern "C" gs_status gs_render_fwd_loss(const gs_config* cfg, const gs_camera* cam, int rec_dtype,
                                        const void* splats, int64_t n, const uint32_t* vals,
                                        const uint32_t* tile_ranges, const uint32_t* tile_order, float* rgb,
                                        float* depth, float* t_final, uint32_t* last_idx, uint32_t* n_blended,
                                        uint32_t* blend_masks, const float* target_rgb, const float* target_depth,
                                        float* d_rgb, float* d_depth, double* loss_out, gs_stream stream) {
    gs_status s;
    if ((s = render_checks(cfg, cam, rec_dtype, splats, n)) != GS_OK) return s;
    if (!tile_ranges || !rgb || !depth || !t_final || !last_idx)
        return set_error(GS_ERR_INVALID_ARG, "an image or range pointer is NULL");
    if (!target_rgb || !target_depth || !d_rgb || !d_depth || !loss_out)
        return set_error(GS_ERR_INVALID_ARG, "a target, gradient or loss pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss_out, 0, sizeof(double), st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset loss");
    const FwdOut O = {rgb, depth, t_final, last_idx, n_blended, target_rgb, target_depth, d_rgb, d_depth, loss_out,
                      blend_masks};
    return dispatch_fwd(*cfg, make_grid(*cam), rec_dtype, splats, vals, tile_ranges, tile_order, O, st);
}

extern "C" size_t gs_blend_mask_words(const gs_camera* cam, int64_t key_capacity) {
    if (!cam || cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1 || key_capacity < 0) return 0;
    const Grid g = make_grid(*cam);
    if (g.tw * g.th <= 64)  // entry-parallel tiles: a run per pixel
        return blend_mask_base_ep(g.TX * g.TY, 0) + (size_t)64 * ((size_t)(key_capacity >> 5) + 1);
    return blend_mask_base(g.TX * g.TY, 0) + (size_t)256 * ((size_t)(key_capacity >> 5) + 1);
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
                                   const uint32_t* last_idx, const uint32_t* blend_masks, const float* d_rgb,
                                   const float* d_depth, int mode,
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
    if (n > 0) {
#define GS_LB(DT, MD) \
    launch_bwd<DT, MD>(*cfg, g, splats, vals, tile_ranges, tile_order, t_final, last_idx, d_rgb, d_depth, grad2d, \
                       blend_masks, st)
        if (mode == GS_MAP)
            s = rec_dtype == GS_F32 ? GS_LB(GS_F32, GS_MAP) : rec_dtype == GS_BF16 ? GS_LB(GS_BF16, GS_MAP)
                                                                                   : GS_LB(GS_F16, GS_MAP);
        else
            s = rec_dtype == GS_F32 ? GS_LB(GS_F32, GS_TRACK) : rec_dtype == GS_BF16 ? GS_LB(GS_BF16, GS_TRACK)
                                                                                     : GS_LB(GS_F16, GS_TRACK);
#undef GS_LB
        if (s != GS_OK) return s;
    }
    if (chain) {
        size_t wb = *workspace_bytes;
        return gs_project_bwd(cfg, cam, gsn, grad2d, grads, pose_grad6, score_terms, workspace, &wb, stream);
    }
    return GS_OK;
}

// ---------------------------------------------------------------------------
// Wave launcher (gs_track_wave): the compositing of every job, grouped by
// kernel form (0: full tiles, one per CTA; 1: smaller pixel-parallel tiles,
// several per CTA; 2, 3: entry-parallel tiles of up to 32 or 64 pixels)
// ---------------------------------------------------------------------------
namespace gs {

static int render_form(const Grid& g) {
    if (g.tw * g.th <= 64) return g.tw * g.th <= 32 ? 2 : 3;
    return R_THREADS / tile_threads(g) == 1 ? 0 : 1;
}

gs_status wave_render(const gs_config& cfg, const gs_track_job* jobs, int n, cudaStream_t st) {
    gs_status s;
    // forward compositing with the fused loss
    int present = 0;
    for (int j = 0; j < n; ++j) present |= 1 << render_form(make_grid(jobs[j].cam));
    for (int form = 0; form < 4; ++form) {
        if (!(present & (1 << form))) continue;
        Wave<WaveFwdJob> W;
        W.n = 0;
        int blocks = 0;
        size_t smem = 0;
        for (int j = 0; j < n; ++j) {
            const gs_track_job& t = jobs[j];
            const Grid g = make_grid(t.cam);
            if (render_form(g) != form) continue;
            const int ntiles = g.TX * g.TY;
            const int gpc = form < 2 ? R_THREADS / tile_threads(g) : 1;
            const int B = form < 2 ? fwd_batch(gpc) : 0;
            const FwdOut O = {t.rgb, t.depth, t.t_final, t.last_idx, t.n_blended, t.target_rgb, t.target_depth,
                              t.d_rgb, t.d_depth, t.loss, t.blend_masks};
            W.start[W.n] = blocks;
            W.job[W.n] = WaveFwdJob{g, t.splats, t.vals, t.tile_ranges, t.tile_order, O, B};
            ++W.n;
            blocks += (ntiles + gpc - 1) / gpc;
            if (form < 2) smem = std::max(smem, (size_t)gpc * (B / 32 * 33) * sizeof(StagedSplat));
        }
        W.start[W.n] = blocks;
        if (form == 0) {
            if ((s = smem_once((const void*)k_wave_render_fwd<1>, 40, R_FWD_SMEM / 32 * 33)) != GS_OK) return s;
            k_wave_render_fwd<1><<<(unsigned)blocks, R_THREADS, smem, st>>>(cfg, W);
        } else if (form == 1) {
            if ((s = smem_once((const void*)k_wave_render_fwd<4>, 41, R_FWD_SMEM / 32 * 33)) != GS_OK) return s;
            k_wave_render_fwd<4><<<(unsigned)blocks, R_THREADS, smem, st>>>(cfg, W);
        } else if (form == 2) {
            k_wave_render_fwd_ep<8><<<(unsigned)blocks, 8 * 32, 0, st>>>(cfg, W);
        } else {
            k_wave_render_fwd_ep<16><<<(unsigned)blocks, 16 * 32, 0, st>>>(cfg, W);
        }
        if ((s = check_launch("k_wave_render_fwd")) != GS_OK) return s;
    }
    // backward compositing, pose-only fields; jobs with blend masks go to the
    // one-warp kernel as in launch_bwd (kind 4: pixel-parallel tiles, 5:
    // 64-pixel entry-parallel tiles)
    auto bwd_kind = [](const gs_track_job& t) {
        const int form = render_form(make_grid(t.cam));
        if (!t.blend_masks) return form;
        return form < 2 ? 4 : (form == 3 ? 5 : form);
    };
    int kinds = 0;
    for (int j = 0; j < n; ++j) kinds |= 1 << bwd_kind(jobs[j]);
    for (int kind = 0; kind < 6; ++kind) {
        if (!(kinds & (1 << kind))) continue;
        Wave<WaveBwdJob> W;
        W.n = 0;
        int blocks = 0;
        size_t smem = 0;
        const int per_entry = (int)(sizeof(StagedSplat) + sizeof(uint32_t) + sizeof(float) * Fields<GS_TRACK>::N);
        for (int j = 0; j < n; ++j) {
            const gs_track_job& t = jobs[j];
            const Grid g = make_grid(t.cam);
            if (bwd_kind(t) != kind) continue;
            const int ntiles = g.TX * g.TY;
            const int gpc = kind < 2 ? R_THREADS / tile_threads(g) : 1;
            const int B = kind < 2 ? group_batch(gpc, per_entry, R_BWD_SMEM) : 0;
            W.start[W.n] = blocks;
            W.job[W.n] = WaveBwdJob{g, t.splats, t.vals, t.tile_ranges, t.tile_order, t.t_final, t.last_idx, t.d_rgb,
                                    t.d_depth, t.grad2d, t.blend_masks, B};
            ++W.n;
            blocks += kind >= 4 ? ntiles * pw_warps(g, kind == 5) : (ntiles + gpc - 1) / gpc;
            if (kind < 2) smem = std::max(smem, (size_t)gpc * B * per_entry);
        }
        W.start[W.n] = blocks;
        if (kind == 0) {
            if ((s = smem_once((const void*)k_wave_render_bwd<1>, 42, R_BWD_SMEM)) != GS_OK) return s;
            k_wave_render_bwd<1><<<(unsigned)blocks, R_THREADS, smem, st>>>(cfg, W);
        } else if (kind == 1) {
            if ((s = smem_once((const void*)k_wave_render_bwd<4>, 43, R_BWD_SMEM)) != GS_OK) return s;
            k_wave_render_bwd<4><<<(unsigned)blocks, R_THREADS, smem, st>>>(cfg, W);
        } else if (kind == 2) {
            const int sm = (int)sizeof(EpBwdSmem<GS_TRACK, 8>);
            if ((s = smem_once((const void*)k_wave_render_bwd_ep<8>, 44, sm)) != GS_OK) return s;
            k_wave_render_bwd_ep<8><<<(unsigned)blocks, 8 * 32, sm, st>>>(cfg, W);
        } else if (kind == 3) {
            const int sm = (int)sizeof(EpBwdSmem<GS_TRACK, 16>);
            if ((s = smem_once((const void*)k_wave_render_bwd_ep<16>, 45, sm)) != GS_OK) return s;
            k_wave_render_bwd_ep<16><<<(unsigned)blocks, 16 * 32, sm, st>>>(cfg, W);
        } else {
            if (kind == 4)
                k_wave_render_bwd_pw<false><<<(unsigned)blocks, 32, 0, st>>>(cfg, W);
            else
                k_wave_render_bwd_pw<true><<<(unsigned)blocks, 32, 0, st>>>(cfg, W);
        }
        if ((s = check_launch("k_wave_render_bwd")) != GS_OK) return s;
    }
    return GS_OK;
}

}  // namespace gs
