// Internal helpers shared by the sm_103a kernels of the rasterizer.
// Not part of the C ABI (see include/gs.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

#define GS_TILE 16
#define GS_TILE_PIX (GS_TILE * GS_TILE)

namespace gs {

// ---------------------------------------------------------------------------
// Host-side error plumbing (defined in gs_api.cu)
// ---------------------------------------------------------------------------
gs_status set_error(gs_status code, const char* fmt, ...);
// gs_project's argument checks (gs_project.cu).
gs_status project_checks(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g, int rec_dtype);
// Projection fused with the binning's per-CTA tile rows (gs_project.cu).
gs_status launch_project_hist(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g, int rec_dtype,
                              void* splats, int64_t per, unsigned nb, int ntiles, uint32_t* hist, void* rects,
                              cudaStream_t st);
gs_status check_launch(const char* what);
int num_sms();

// Device address of the status word of the current device (defined in
// gs_api.cu).  Kernels that can raise a condition receive it as an argument
// and set it with raise_status (the first condition wins).
unsigned int* status_ptr();

__device__ __forceinline__ void raise_status(unsigned int* st, unsigned int code) {
    atomicCAS(st, 0u, code);
}

// Replaces R and t by the device pose when the camera carries one.
__device__ __forceinline__ void resolve_pose(gs_camera& cam) {
    if (cam.pose) {
#pragma unroll
        for (int i = 0; i < 9; ++i) cam.R[i] = __ldg(cam.pose + i);
#pragma unroll
        for (int i = 0; i < 3; ++i) cam.t[i] = __ldg(cam.pose + 9 + i);
    }
}

// ---------------------------------------------------------------------------
// Sampled grid of a camera (Sec. 4.2 strides)
// ---------------------------------------------------------------------------
struct Grid {
    int W, H;        // full resolution
    int sx, sy;      // strides
    int Ws, Hs;      // sampled image
    int tw, th;      // tile size in sampled pixels (powers of two)
    int lw, lh;      // log2 of tw, th
    int TX, TY;      // tiles
};

// Tile side in sampled pixels for stride s: 16 / p2(s), at least 4, where
// p2(s) is the smallest power of two >= s.  The tile's full-resolution
// footprint stays ~16 pixels (the paper's tile), so a sampled pixel's tile
// list does not grow with the stride.
__host__ __device__ inline int tile_dim(int s) {
    int p = 1;
    while (p < s && p < 16) p <<= 1;
    const int t = GS_TILE / p;
    return t < 4 ? 4 : t;
}

__host__ __device__ inline Grid make_grid(const gs_camera& c) {
    Grid g;
    g.W = c.width;
    g.H = c.height;
    g.sx = c.sx;
    g.sy = c.sy;
    // (integer division is a long instruction sequence on the GPU: stride 1
    // and the power-of-two tile sides take the direct forms)
    g.Ws = c.sx == 1 ? c.width : (c.width + c.sx - 1) / c.sx;
    g.Hs = c.sy == 1 ? c.height : (c.height + c.sy - 1) / c.sy;
    g.tw = tile_dim(c.sx);
    g.th = tile_dim(c.sy);
    g.lw = g.tw == 16 ? 4 : (g.tw == 8 ? 3 : 2);
    g.lh = g.th == 16 ? 4 : (g.th == 8 ? 3 : 2);
    g.TX = (g.Ws + g.tw - 1) >> g.lw;
    g.TY = (g.Hs + g.th - 1) >> g.lh;
    return g;
}

__host__ __device__ inline int floor_div(int a, int b) {
    if (b == 1) return a;
    int q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}
__host__ __device__ inline int ceil_div_i(int a, int b) { return -floor_div(-a, b); }
__host__ __device__ inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Integer pixel position of a 2D mean: floor of the coordinate, clamped so
// that it fits an int far outside any image.
__device__ __forceinline__ int pix_floor(float u) {
    return (int)floorf(fminf(fmaxf(u, -1.0e9f), 1.0e9f));
}

// Tile rect [x0,x1) x [y0,y1) of a 2D Gaussian with mean (u, v) and integer
// radius r: the sampled pixels inside the image whose full-resolution
// position lies in the box [floor(u)-r, floor(u)+r] x [floor(v)-r, floor(v)+r]
// (Sec. 2.1, Step 1-2; strides of Sec. 4.2), in tiles of tw x th sampled
// pixels.  Returns the tile count.
// Geometry a tile rect needs: mean, depth, radius, conic and opacity.
struct Geom {
    float x, y, depth;
    int radius;
    float ca, cb, cc, op;
};

// Half extents (ex, ey) of the pixel box where alpha = op exp(-d^T Q d / 2)
// can reach alpha_min (Q = conic; fragments below alpha_min are skipped,
// Sec. 2.1): |d_x| <= sqrt(2 ln(op / alpha_min) (Q^-1)_xx).  ln is bounded
// above by 64 (x^(1/64) - 1) (from e^t >= 1 + t), computed with six
// correctly rounded square roots and fixed float32 operations, so the FP64
// oracle evaluates the very same float32 numbers; 1e-3 added to the bound
// and the factor 1.002 + 2e-3 px cover the rounding of the per-pixel alpha
// test.  Returns false when no pixel can reach alpha_min (op < alpha_min);
// (ex, ey) = +inf when the conic is degenerate (no shrinking).
__device__ __forceinline__ bool alpha_extent(float ca, float cb, float cc, float op, float alpha_min, float& ex,
                                             float& ey) {
    if (!(op >= alpha_min)) return false;
    ex = ey = __int_as_float(0x7f800000);
    const float det = __fsub_rn(__fmul_rn(ca, cc), __fmul_rn(cb, cb));
    if (!(det > 0.f)) return true;
    float q = __fdiv_rn(op, alpha_min);
#pragma unroll
    for (int i = 0; i < 6; ++i) q = __fsqrt_rn(q);
    const float L = __fmul_rn(64.f, __fsub_rn(q, 1.f));
    const float t2 = __fmul_rn(2.f, __fadd_rn(fmaxf(L, 0.f), 1e-3f));
    ex = __fadd_rn(__fmul_rn(__fsqrt_rn(__fdiv_rn(__fmul_rn(t2, cc), det)), 1.002f), 2e-3f);
    ey = __fadd_rn(__fmul_rn(__fsqrt_rn(__fdiv_rn(__fmul_rn(t2, ca), det)), 1.002f), 2e-3f);
    return true;
}

// Tiles of a Gaussian (Sec. 2.1, Step 1-2): those holding a sampled in-image
// pixel of its integer box [floor(x) - r, floor(x) + r] x [...] shrunk to the
// pixels whose centre lies within the alpha extent (pixel p when
// |p + 0.5 - x| <= ex).  Returns the tile count and [x0, x1) x [y0, y1).
__device__ __forceinline__ int tile_rect(const Grid& g, const Geom& G, float alpha_min, int& x0, int& x1,
                                         int& y0, int& y1) {
    x0 = x1 = y0 = y1 = 0;
    const int r = G.radius;
    if (r <= 0) return 0;
    float ex, ey;
    if (!alpha_extent(G.ca, G.cb, G.cc, G.op, alpha_min, ex, ey)) return 0;
    int xi = pix_floor(G.x), yi = pix_floor(G.y);
    // 64-bit guard against xi +- r overflow is unnecessary: |xi| <= 1e9, r < 2^30
    long long bx0 = (long long)xi - r, bx1 = (long long)xi + r;
    long long by0 = (long long)yi - r, by1 = (long long)yi + r;
    if (ex < 1e8f && fabsf(G.x) < 1e8f) {
        bx0 = max(bx0, (long long)ceilf(__fsub_rn(__fsub_rn(G.x, ex), 0.5f)));
        bx1 = min(bx1, (long long)floorf(__fsub_rn(__fadd_rn(G.x, ex), 0.5f)));
    }
    if (ey < 1e8f && fabsf(G.y) < 1e8f) {
        by0 = max(by0, (long long)ceilf(__fsub_rn(__fsub_rn(G.y, ey), 0.5f)));
        by1 = min(by1, (long long)floorf(__fsub_rn(__fadd_rn(G.y, ey), 0.5f)));
    }
    if (bx1 < bx0 || by1 < by0) return 0;
    if (bx1 < 0 || by1 < 0 || bx0 > (long long)(g.W - 1) || by0 > (long long)(g.H - 1)) return 0;
    int i0 = ceil_div_i((int)max(bx0, -1LL), g.sx);
    int i1 = floor_div((int)min(bx1, (long long)g.W), g.sx);
    int j0 = ceil_div_i((int)max(by0, -1LL), g.sy);
    int j1 = floor_div((int)min(by1, (long long)g.H), g.sy);
    i0 = clampi(i0, 0, g.Ws);
    i1 = clampi(i1, -1, g.Ws - 1);
    j0 = clampi(j0, 0, g.Hs);
    j1 = clampi(j1, -1, g.Hs - 1);
    if (i0 > i1 || j0 > j1) return 0;
    x0 = i0 >> g.lw;  // i0, j0 >= 0 here
    x1 = (i1 >> g.lw) + 1;
    y0 = j0 >> g.lh;
    y1 = (j1 >> g.lh) + 1;
    return (x1 - x0) * (y1 - y0);
}

// ---------------------------------------------------------------------------
// 2D records
// ---------------------------------------------------------------------------
// Unpacked 2D Gaussian as the compositing kernels use it.
struct Splat {
    float x, y, ca, cb, cc, op, depth;
    int radius;
    float r, g, b;
};

__device__ __forceinline__ float h2f(uint16_t h, int dt) {
    if (dt == GS_BF16) return __bfloat162float(__ushort_as_bfloat16(h));
    return __half2float(__ushort_as_half(h));
}
__device__ __forceinline__ uint16_t f2h(float f, int dt) {
    if (dt == GS_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(f));
    return __half_as_ushort(__float2half_rn(f));
}

template <int DT>
__device__ __forceinline__ Splat load_splat(const void* base, uint32_t k) {
    Splat s;
    if (DT == GS_F32) {
        const float4* p = reinterpret_cast<const float4*>(base) + 3 * (size_t)k;
        float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
        s.x = a.x; s.y = a.y; s.ca = a.z; s.cb = a.w;
        s.cc = b.x; s.op = b.y; s.depth = b.z; s.radius = __float_as_int(b.w);
        s.r = c.x; s.g = c.y; s.b = c.z;
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(base) + 2 * (size_t)k;
        uint4 a = __ldg(p), b = __ldg(p + 1);
        s.x = __uint_as_float(a.x); s.y = __uint_as_float(a.y);
        s.depth = __uint_as_float(a.z); s.radius = (int)a.w;
        s.ca = h2f((uint16_t)(b.x & 0xffff), DT); s.cb = h2f((uint16_t)(b.x >> 16), DT);
        s.cc = h2f((uint16_t)(b.y & 0xffff), DT); s.op = h2f((uint16_t)(b.y >> 16), DT);
        s.r = h2f((uint16_t)(b.z & 0xffff), DT); s.g = h2f((uint16_t)(b.z >> 16), DT);
        s.b = h2f((uint16_t)(b.w & 0xffff), DT);
    }
    return s;
}

// What the binning reads of a record: mean, depth, radius, conic, opacity.
template <int DT>
__device__ __forceinline__ Geom load_geom(const void* base, uint32_t k) {
    Geom G;
    if (DT == GS_F32) {
        const float4* p = reinterpret_cast<const float4*>(base) + 3 * (size_t)k;
        const float4 a = __ldg(p), b = __ldg(p + 1);
        G.x = a.x; G.y = a.y; G.ca = a.z; G.cb = a.w;
        G.cc = b.x; G.op = b.y; G.depth = b.z; G.radius = __float_as_int(b.w);
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(base) + 2 * (size_t)k;
        const uint4 a = __ldg(p), b = __ldg(p + 1);
        G.x = __uint_as_float(a.x); G.y = __uint_as_float(a.y);
        G.depth = __uint_as_float(a.z); G.radius = (int)a.w;
        G.ca = h2f((uint16_t)(b.x & 0xffff), DT); G.cb = h2f((uint16_t)(b.x >> 16), DT);
        G.cc = h2f((uint16_t)(b.y & 0xffff), DT); G.op = h2f((uint16_t)(b.y >> 16), DT);
    }
    return G;
}

// ---------------------------------------------------------------------------
// Adam (the map update of a mapping iteration; the paper fixes no optimizer)
// ---------------------------------------------------------------------------
// One element: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
// p <- p - lr (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t.
// Every operation rounded on its own (no contraction), so gs_adam and the
// Adam step fused into the backward projection give the same bits.
__device__ __forceinline__ void adam_elem(float& p, float& m, float& v, float g, float lr, float b1, float b2,
                                          float c1, float c2, float eps) {
    m = __fadd_rn(__fmul_rn(b1, m), __fmul_rn(__fsub_rn(1.f, b1), g));
    v = __fadd_rn(__fmul_rn(b2, v), __fmul_rn(__fmul_rn(__fsub_rn(1.f, b2), g), g));
    p = __fsub_rn(p, __fdiv_rn(__fmul_rn(lr, __fdiv_rn(m, c1)), __fadd_rn(__fsqrt_rn(__fdiv_rn(v, c2)), eps)));
}

// ---------------------------------------------------------------------------
// Multi-session waves (gs_track_wave)
// ---------------------------------------------------------------------------
// A wave launch's descriptor table: job j owns blocks [start[j], start[j+1])
// of the grid.  It is passed by value as a __grid_constant__ kernel
// parameter (constant bank), so every CTA reads it without a copy.
template <typename J>
struct Wave {
    int n;
    int start[GS_WAVE_MAX + 1];
    J job[GS_WAVE_MAX];
};

// Job of block b: the largest j with start[j] <= b (binary search).
__device__ __forceinline__ int wave_find(const int* start, int n, int b) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Where a job's binning state lives in its gs_project_bin_sort workspace.
struct WaveBin {
    int64_t per;          // Gaussians per projection / scatter CTA
    unsigned nb;          // projection CTAs (rows of hist)
    int ntiles;
    uint32_t* count;      // tile totals
    uint32_t* start;      // bucket starts
    uint32_t* hist;       // per-CTA tile rows
    unsigned int* ticket; // the column scan's ticket
    uint32_t* n_big;
    void* tmp;            // sort scratch
    void* rects;          // kept tile rects
};
gs_status wave_bin_layout(const gs_track_job& j, WaveBin* out);
unsigned int* wave_bwd_ticket(const gs_track_job& j);
// The stages of a wave, in launch order.
gs_status wave_project_hist(const gs_config& cfg, const gs_track_job* jobs, const WaveBin* bins, int n,
                            cudaStream_t st);
gs_status wave_bin_sort(const gs_track_job* jobs, const WaveBin* bins, int n, cudaStream_t st);
gs_status wave_render(const gs_config& cfg, const gs_track_job* jobs, int n, cudaStream_t st);
gs_status wave_project_bwd(const gs_config& cfg, const gs_track_job* jobs, int n, cudaStream_t st);

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sum of NF values, scattered over the lanes: at each butterfly level
// (lane offsets 16, 8, ..., 1) the C values a lane still carries are paired,
// the lower lanes keeping the first C/2 and the upper lanes the second C/2
// (a lane sends the half it gives up and combines it with what its partner
// sends), and an odd one out is combined whole; once one value is left, the
// remaining levels combine it with the partner's.  NF = 6 takes 8 exchanges,
// NF = 10 takes 12, NF = 12 takes 13 (instead of 5 per value).  Value f ends
// up summed over all 32 lanes on the lanes whose merge_owner<NF> is f.
// Op::swap(x, off) exchanges x with the lane `off` away; Op::join(mine,
// theirs, up) combines the value a lane keeps with the one its partner sent
// (up: this lane is the upper partner), in an operand order that makes both
// partners of a level compute the same bits.
struct MergeFloat {
    static __device__ __forceinline__ float swap(float x, int off) { return __shfl_xor_sync(0xffffffffu, x, off); }
    static __device__ __forceinline__ float join(float mine, float theirs, bool) { return mine + theirs; }
};
struct MergeIds {  // the pairing alone, on value numbers
    static __device__ __forceinline__ int swap(int x, int) { return x; }
    static __device__ __forceinline__ int join(int mine, int, bool) { return mine; }
};

template <int C, int OFF>
struct MergeLevel {
    template <typename T, int NF, typename Op>
    static __device__ __forceinline__ void run(T (&v)[NF], int lane) {
        if constexpr (OFF > 0) {
            const bool up = (lane & OFF) != 0;
            if constexpr (C > 1) {
                constexpr int H = C / 2;
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    const T send = up ? v[i] : v[i + H];
                    const T keep = up ? v[i + H] : v[i];
                    v[i] = Op::join(keep, Op::swap(send, OFF), up);
                }
                if constexpr ((C & 1) != 0) v[H] = Op::join(v[C - 1], Op::swap(v[C - 1], OFF), up);
                MergeLevel<H + (C & 1), OFF / 2>::template run<T, NF, Op>(v, lane);
            } else {
                v[0] = Op::join(v[0], Op::swap(v[0], OFF), up);
                MergeLevel<1, OFF / 2>::template run<T, NF, Op>(v, lane);
            }
        }
    }
};

template <int NF, typename T = float, typename Op = MergeFloat>
__device__ __forceinline__ T warp_merge(T (&v)[NF]) {
    static_assert(NF >= 1 && NF <= 32, "at most one merged value per lane");
    MergeLevel<NF, 16>::template run<T, NF, Op>(v, threadIdx.x & 31);
    return v[0];
}

// The value this lane holds after warp_merge<NF>, or -1: the same pairing on
// value numbers; of the lanes left holding the same value, the lowest owns it.
template <int NF>
__device__ __forceinline__ int merge_owner() {
    const int lane = threadIdx.x & 31;
    int id[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) id[i] = i;
    MergeLevel<NF, 16>::template run<int, NF, MergeIds>(id, lane);
    const unsigned same = __match_any_sync(0xffffffffu, id[0]);
    return lane == __ffs(same) - 1 ? id[0] : -1;
}

}  // namespace gs
