// A-1 projection (Sec. 2.1, Step 1-1) and A-8 backward projection + camera
// pose gradient (Sec. 2.2, Step 5) on sm_103a.
//
// One thread per Gaussian.  Both passes call project_core(), so the backward
// differentiates exactly the float32 arithmetic of the forward.  These
// kernels stream the 56-byte parameter record once (forward: plus a 48-byte
// or 32-byte 2D record write; backward: plus the 48-byte 2D gradient) and are
// HBM-bound at large n.
#include <stdio.h>

#include <algorithm>
#include <atomic>

#include "gs_internal.cuh"

namespace gs {

struct Proj {
    bool visible;
    float p[3];          // camera-frame mean
    float qn[4];         // normalised quaternion (w, x, y, z)
    float qinv;          // 1/|q|
    float scale[3];      // exp(log_scale)
    float M[9];          // Rq diag(scale), row-major
    float Sc[9];         // camera-frame covariance R M M^T R^T
    bool clx, cly;       // x/z or y/z hit the clamp
    float lx, ly;        // signed clamp value when clamped
    float J00, J02, J11, J12;
    float a, b, c;       // 2D covariance + dilation
    float ca, cb, cc;    // conic
    float u, v;
    int radius;
    float op;
};

__device__ __forceinline__ void project_core(const gs_camera& cam, const gs_config& cfg,
                                             const float* mu, const float* ls, const float* q,
                                             float ologit, Proj& o) {
    const float* R = cam.R;
    o.visible = false;
    o.radius = 0;
    for (int i = 0; i < 3; ++i)
        o.p[i] = fmaf(R[3 * i], mu[0], fmaf(R[3 * i + 1], mu[1], fmaf(R[3 * i + 2], mu[2], cam.t[i])));
    const float x = o.p[0], y = o.p[1], z = o.p[2];
    if (!(z >= cfg.near_z)) return;

    float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    o.qinv = 1.0f / sqrtf(qq);
    for (int i = 0; i < 4; ++i) o.qn[i] = q[i] * o.qinv;
    const float w = o.qn[0], qx = o.qn[1], qy = o.qn[2], qz = o.qn[3];
    float Rq[9];
    Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); Rq[1] = 2.f * (qx * qy - w * qz); Rq[2] = 2.f * (qx * qz + w * qy);
    Rq[3] = 2.f * (qx * qy + w * qz); Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); Rq[5] = 2.f * (qy * qz - w * qx);
    Rq[6] = 2.f * (qx * qz - w * qy); Rq[7] = 2.f * (qy * qz + w * qx); Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
    for (int i = 0; i < 3; ++i) o.scale[i] = expf(ls[i]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) o.M[3 * i + j] = Rq[3 * i + j] * o.scale[j];
    // W = R M  ->  Sc = W W^T
    float Wm[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Wm[3 * i + j] = R[3 * i] * o.M[j] + R[3 * i + 1] * o.M[3 + j] + R[3 * i + 2] * o.M[6 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            float s = Wm[3 * i] * Wm[3 * j] + Wm[3 * i + 1] * Wm[3 * j + 1] + Wm[3 * i + 2] * Wm[3 * j + 2];
            o.Sc[3 * i + j] = s;
            o.Sc[3 * j + i] = s;
        }

    const float limx = 1.3f * (0.5f * (float)cam.width) / cam.fx;
    const float limy = 1.3f * (0.5f * (float)cam.height) / cam.fy;
    const float zi = 1.0f / z;
    float xz = x * zi, yz = y * zi;
    o.clx = o.cly = false;
    o.lx = o.ly = 0.f;
    if (xz > limx) { xz = limx; o.clx = true; o.lx = limx; }
    else if (xz < -limx) { xz = -limx; o.clx = true; o.lx = -limx; }
    if (yz > limy) { yz = limy; o.cly = true; o.ly = limy; }
    else if (yz < -limy) { yz = -limy; o.cly = true; o.ly = -limy; }
    o.J00 = cam.fx * zi;
    o.J02 = -cam.fx * xz * zi;
    o.J11 = cam.fy * zi;
    o.J12 = -cam.fy * yz * zi;
    // Sigma2 = J Sc J^T with J = [[J00, 0, J02], [0, J11, J12]]
    const float* S = o.Sc;
    float T0x = o.J00 * S[0] + o.J02 * S[6], T0y = o.J00 * S[1] + o.J02 * S[7], T0z = o.J00 * S[2] + o.J02 * S[8];
    float T1y = o.J11 * S[4] + o.J12 * S[7], T1z = o.J11 * S[5] + o.J12 * S[8];
    o.a = T0x * o.J00 + T0z * o.J02 + cfg.dilation;
    o.b = T0y * o.J11 + T0z * o.J12;
    o.c = T1y * o.J11 + T1z * o.J12 + cfg.dilation;
    const float det = o.a * o.c - o.b * o.b;
    if (!(det > 0.f)) return;
    const float di = 1.0f / det;
    o.ca = o.c * di;
    o.cb = -o.b * di;
    o.cc = o.a * di;
    const float mid = 0.5f * (o.a + o.c);
    const float lmax = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    const float r = ceilf(3.0f * sqrtf(lmax));
    o.radius = (int)fminf(r, 1073741824.0f);
    o.u = cam.fx * x * zi + cam.cx;
    o.v = cam.fy * y * zi + cam.cy;
    o.op = 1.0f / (1.0f + expf(-ologit));
    o.visible = true;
}

// Projects Gaussian k and writes its 2D record; returns its tile count and
// rect [x0, x1) x [y0, y1) (the binning's, from the values as the record
// stores them).  `cam` has its pose resolved.
template <int DT>
__device__ __forceinline__ int project_write(const gs_camera& cam, const gs_config& cfg, const gs_gaussians& g,
                                             const Grid& grid, int64_t k, void* out, int& x0, int& x1, int& y0,
                                             int& y1) {
    float mu[3], ls[3], q[4];
    for (int i = 0; i < 3; ++i) { mu[i] = __ldg(g.means + 3 * k + i); ls[i] = __ldg(g.log_scales + 3 * k + i); }
    for (int i = 0; i < 4; ++i) q[i] = __ldg(g.quats + 4 * k + i);
    const float ol = __ldg(g.opacity_logit + k);
    const bool masked = g.mask && __ldg(g.mask + k);
    Proj o;
    if (!masked) project_core(cam, cfg, mu, ls, q, ol, o);
    else { o.visible = false; o.radius = 0; }
    float cr = __ldg(g.rgb + 3 * k), cg = __ldg(g.rgb + 3 * k + 1), cb = __ldg(g.rgb + 3 * k + 2);
    int touched = 0;
    x0 = x1 = y0 = y1 = 0;
    if (o.visible) {
        Geom G;
        G.x = o.u; G.y = o.v; G.depth = o.p[2]; G.radius = o.radius;
        G.ca = DT == GS_F32 ? o.ca : h2f(f2h(o.ca, DT), DT);
        G.cb = DT == GS_F32 ? o.cb : h2f(f2h(o.cb, DT), DT);
        G.cc = DT == GS_F32 ? o.cc : h2f(f2h(o.cc, DT), DT);
        G.op = DT == GS_F32 ? o.op : h2f(f2h(o.op, DT), DT);
        touched = tile_rect(grid, G, cfg.alpha_min, x0, x1, y0, y1);
    } else {
        o.u = o.v = o.ca = o.cb = o.cc = o.op = 0.f;
        o.p[2] = 0.f;
        o.radius = 0;
    }
    if (DT == GS_F32) {
        float4* dst = reinterpret_cast<float4*>(out) + 3 * k;
        dst[0] = make_float4(o.u, o.v, o.ca, o.cb);
        dst[1] = make_float4(o.cc, o.op, o.p[2], __int_as_float(o.radius));
        dst[2] = make_float4(cr, cg, cb, __uint_as_float((uint32_t)touched));
    } else {
        uint4* dst = reinterpret_cast<uint4*>(out) + 2 * k;
        dst[0] = make_uint4(__float_as_uint(o.u), __float_as_uint(o.v), __float_as_uint(o.p[2]),
                            (uint32_t)o.radius);
        uint32_t t16 = (uint32_t)min(touched, 65535);
        dst[1] = make_uint4((uint32_t)f2h(o.ca, DT) | ((uint32_t)f2h(o.cb, DT) << 16),
                            (uint32_t)f2h(o.cc, DT) | ((uint32_t)f2h(o.op, DT) << 16),
                            (uint32_t)f2h(cr, DT) | ((uint32_t)f2h(cg, DT) << 16),
                            (uint32_t)f2h(cb, DT) | (t16 << 16));
    }
    return touched;
}

template <int DT>
__global__ void __launch_bounds__(256) k_project(gs_camera cam, gs_config cfg, gs_gaussians g,
                                                 void* out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    resolve_pose(cam);
    const Grid grid = make_grid(cam);
    int x0, x1, y0, y1;
    project_write<DT>(cam, cfg, g, grid, k, out, x0, x1, y0, y1);
}

// Projection fused with the binning's first pass: CTA c projects Gaussians
// [c per, (c + 1) per), counts their tiles in a shared row that becomes row
// c of `hist` (the per-CTA tile rows of the binning), and keeps each rect
// (x0 | x1 << 16, y0 | y1 << 16; zero: no tile) for the scatter.
template <int DT>
__device__ __forceinline__ void project_hist_body(gs_camera cam, const gs_config& cfg, const gs_gaussians& g,
                                                  void* out, int64_t per, int ntiles, uint32_t* __restrict__ hist,
                                                  uint2* __restrict__ rects, int blk) {
    extern __shared__ uint32_t h_row[];
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) h_row[t] = 0;
    __syncthreads();
    resolve_pose(cam);
    const Grid grid = make_grid(cam);
    const int64_t k0 = (int64_t)blk * per, k1 = min(g.n, k0 + per);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        int x0, x1, y0, y1;
        const int touched = project_write<DT>(cam, cfg, g, grid, k, out, x0, x1, y0, y1);
        rects[k] = touched ? make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16))
                           : make_uint2(0u, 0u);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) atomicAdd(h_row + ty * grid.TX + tx, 1u);
    }
    __syncthreads();
    uint32_t* row = hist + (size_t)blk * ntiles;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) row[t] = h_row[t];
}

template <int DT>
__global__ void __launch_bounds__(256) k_project_hist(gs_camera cam, gs_config cfg, gs_gaussians g, void* out,
                                                      int64_t per, int ntiles, uint32_t* __restrict__ hist,
                                                      uint2* __restrict__ rects) {
    project_hist_body<DT>(cam, cfg, g, out, per, ntiles, hist, rects, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------
// Backward projection (Sec. 2.2, Step 5)
// ---------------------------------------------------------------------------

#define PB_THREADS 256
#define PB_PER 2          // Gaussians per thread of the backward projection with the pose

// Blocks of the backward projection for n Gaussians, per Gaussians a thread.
static inline int64_t pb_blocks(int64_t n, int per) { return (n + per * PB_THREADS - 1) / (per * PB_THREADS); }

// The pose gradient is a sum over every Gaussian of terms of both signs
// (the Merging Tree of Sec. 5.1 reduces it in hardware).  Inside a block the
// sums carry a float32 pair (hi, lo) with hi + lo the value (about 48
// significant bits): additions are an error-free two-sum of the high parts
// (Knuth) plus the low parts, renormalised with a fast two-sum (Dekker), in
// float32 because GB300's float64 rate is a small fraction of it; the last
// block sums the blocks' pairs the same way, merges its 32 lane sums in a
// butterfly of pair additions and returns hi + lo as a float64.
// Fixed operation order throughout, so the reduction is deterministic.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bp = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, t);
    return DF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

// Pairs exchanged and added in warp_merge.
struct MergeDF {
    static __device__ __forceinline__ DF swap(DF x, int off) {
        return DF{__shfl_xor_sync(0xffffffffu, x.hi, off), __shfl_xor_sync(0xffffffffu, x.lo, off)};
    }
    static __device__ __forceinline__ DF join(DF mine, DF theirs, bool up) {
        return up ? df_add(theirs, mine) : df_add(mine, theirs);  // the lower lane's value first
    }
};

// ---------------------------------------------------------------------------
// Pose step: Adam on xi, then T <- exp(xi^) T
// ---------------------------------------------------------------------------
// Adam on component i of xi: its moments (m, v) are updated in place; returns
// the step xi_i (rho: lr_t, phi: lr_r).
__device__ __forceinline__ float pose_adam_component(int i, float g, float& m, float& v, float step, float lr_t,
                                                     float lr_r, float b1, float b2, float eps) {
    const float c1 = 1.f - powf(b1, step), c2 = 1.f - powf(b2, step);
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    return -(i < 3 ? lr_t : lr_r) * (m / c1) / (sqrtf(v / c2) + eps);
}

// T <- exp(xi^) T for a pose (R row-major, t); pose_in may be pose_out.
__device__ __forceinline__ void pose_exp_apply(const float* xi, const float* pose_in, float* pose_out) {
    // exp of (rho, phi): R_d = Rodrigues(phi), V = I + (1-cos)/th^2 K + (th-sin)/th^3 K^2
    const float px = xi[3], py = xi[4], pz = xi[5];
    const float th2 = px * px + py * py + pz * pz, th = sqrtf(th2);
    float A, B, Cc;
    if (th < 1e-4f) {
        A = 1.f - th2 / 6.f;
        B = 0.5f - th2 / 24.f;
        Cc = 1.f / 6.f - th2 / 120.f;
    } else {
        A = sinf(th) / th;
        B = (1.f - cosf(th)) / th2;
        Cc = (th - sinf(th)) / (th2 * th);
    }
    const float K[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
    float K2[9], Rd[9], V[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
    for (int i = 0; i < 9; ++i) {
        const float I = (i % 4 == 0) ? 1.f : 0.f;
        Rd[i] = I + A * K[i] + B * K2[i];
        V[i] = I + B * K[i] + Cc * K2[i];
    }
    float R[9], t[3], Rn[9], tn[3];
    for (int i = 0; i < 9; ++i) R[i] = pose_in[i];
    for (int i = 0; i < 3; ++i) t[i] = pose_in[9 + i];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Rn[3 * i + j] = Rd[3 * i] * R[j] + Rd[3 * i + 1] * R[3 + j] + Rd[3 * i + 2] * R[6 + j];
        tn[i] = Rd[3 * i] * t[0] + Rd[3 * i + 1] * t[1] + Rd[3 * i + 2] * t[2] +
                V[3 * i] * xi[0] + V[3 * i + 1] * xi[1] + V[3 * i + 2] * xi[2];
    }
    for (int i = 0; i < 9; ++i) pose_out[i] = Rn[i];
    for (int i = 0; i < 3; ++i) pose_out[9 + i] = tn[i];
}

// The pose step by one block (every thread calls it, at least 6 of them):
// thread i < 6 takes component i of the Adam step, thread 0 the exp map.
// g6 = dL/dxi; the moments and step count are read from adam_in and written
// to adam_out, the pose read from pose_in and written to pose_out (in and out
// may be the same memory).  Not inlined, so that the separate pose update and
// the one fused into the backward projection run the same code.
__device__ __noinline__ void pose_step_block(const double* g6, const float* adam_in, float* adam_out,
                                             const float* pose_in, float* pose_out, float lr_t, float lr_r,
                                             float b1, float b2, float eps) {
    __shared__ float s_xi[6];
    const int i = threadIdx.x;
    const float step = adam_in[12] + 1.f;
    if (i < 6) {
        float m = adam_in[i], v = adam_in[6 + i];
        s_xi[i] = pose_adam_component(i, (float)g6[i], m, v, step, lr_t, lr_r, b1, b2, eps);
        adam_out[i] = m;
        adam_out[6 + i] = v;
    }
    __syncthreads();
    if (i == 0) {
        adam_out[12] = step;
        pose_exp_apply(s_xi, pose_in, pose_out);
    }
}

__global__ void k_pose_update(float* __restrict__ pose, const double* __restrict__ grad, float* __restrict__ adam,
                              float lr_t, float lr_r, float b1, float b2, float eps) {
    pose_step_block(grad, adam, adam, pose, pose, lr_t, lr_r, b1, b2, eps);
}

// Final combination of the per-block pose partials (float32 pairs) by the
// last block to finish (no spin: the block that takes the last ticket sees
// every other block's partial, published before its ticket).  Warp w < 6 sums
// component w, each lane its strided share of the blocks (16 loads in flight
// before the dependent additions), then the 32 lane sums meet in a fixed
// butterfly of pair additions; warp 7 meanwhile reads the pose step's inputs.
// float64 appears only in the result: on GB300 a float64 butterfly took
// 2.7 us of this block's tail, the pairs a small fraction of it.
__device__ void pose_final_last_block(const float2* __restrict__ part, int nblk, double* __restrict__ out,
                                      unsigned int* __restrict__ ticket, const gs_pose_step& step) {
    static_assert(PB_THREADS >= 256, "the last block uses warps 0-5 and 7");
    __shared__ bool s_last;
    __shared__ float s_pose[12], s_adam[13];
    __shared__ double s_g[6];
    __threadfence();
    __syncwarp();  // lanes 0-5 of warp 0 wrote the partials: their fences precede the ticket
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)nblk - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (step.pose && w == 7) {
        if (lane < 12) s_pose[lane] = step.pose[lane];
        else if (lane < 25) s_adam[lane - 12] = step.adam[lane - 12];
    }
    if (w < 6) {
        DF d{0.f, 0.f};
        for (int b0 = lane; b0 < nblk; b0 += 16 * 32) {
            float2 v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int b = b0 + 32 * j;
                v[j] = b < nblk ? __ldcg(part + (size_t)b * 6 + w) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (b0 + 32 * j < nblk) d = df_add(d, DF{v[j].x, v[j].y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DF t{__shfl_xor_sync(0xffffffffu, d.hi, o), __shfl_xor_sync(0xffffffffu, d.lo, o)};
            d = (lane & o) ? df_add(t, d) : df_add(d, t);  // the same operand order on both partners
        }
        if (lane == 0) {
            const double g = (double)d.hi + (double)d.lo;
            out[w] = g;
            s_g[w] = g;
        }
    }
    if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch
    if (step.pose) {  // the fused pose step (every block has read the pose by now)
        __syncthreads();
        pose_step_block(s_g, s_adam, step.adam, s_pose, step.pose, step.lr_trans, step.lr_rot, step.beta1,
                        step.beta2, step.eps);
    }
}

// The map's Adam step fused into the backward projection (mapping): each
// thread updates its Gaussian's parameters and moments from the gradients it
// just formed.  p[t] are the parameter arrays of the map (means, log_scales,
// quats, opacity_logit, rgb), m[t] and v[t] their moments.
struct AdamMap {
    float* p[5];
    float* m[5];
    float* v[5];
    float lr, b1, b2, eps, c1, c2;
};

// PER Gaussians per thread: two when the pose is reduced (391 blocks of 256
// fit one wave on the tracking frame: 21.5 -> 19.5 us), one otherwise (the
// mapping step's per-Gaussian gradients and Adam update are memory-bound and
// want every thread: 0.936 against 0.979 ms per mapping iteration).
template <bool WANT_GRADS, bool WANT_POSE, bool WANT_SCORE, bool ADAM = false, int PER = WANT_POSE ? PB_PER : 1>
__device__ __forceinline__ void project_bwd_body(gs_camera cam, const gs_config& cfg, const gs_gaussians& g,
                                                 const float* __restrict__ grad2d, const gs_grads& grads,
                                                 float* __restrict__ score, float2* __restrict__ pose_part,
                                                 double* __restrict__ pose_out, unsigned int* __restrict__ ticket,
                                                 const gs_pose_step& step, int blk, int nblk,
                                                 const AdamMap* adam = nullptr) {
    // the thread's pose terms, summed as float32 pairs over its Gaussians
    DF pacc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) pacc[i] = DF{0.f, 0.f};
    resolve_pose(cam);
#pragma unroll 1
    for (int rep = 0; rep < PER; ++rep) {
        const int64_t k = ((int64_t)blk * PER + rep) * blockDim.x + threadIdx.x;
        float pose[6] = {0, 0, 0, 0, 0, 0};
        if (k < g.n) {
            float mu[3], ls[3], q[4];
            for (int i = 0; i < 3; ++i) { mu[i] = __ldg(g.means + 3 * k + i); ls[i] = __ldg(g.log_scales + 3 * k + i); }
            for (int i = 0; i < 4; ++i) q[i] = __ldg(g.quats + 4 * k + i);
            const float ol = __ldg(g.opacity_logit + k);
            const bool masked = g.mask && __ldg(g.mask + k);
            // With the pose reduced (a latency-bound launch of one wave) the
            // 2D gradient is read with the parameters, so the two loads'
            // latencies overlap instead of following the projection (grad2d
            // holds n rows; the values count only for a visible Gaussian).
            // Otherwise it is read after it, keeping fewer values live.
            const float4* g4 = reinterpret_cast<const float4*>(grad2d) + 3 * k;
            float4 ga, gb, gc;
            if (WANT_POSE) { ga = __ldg(g4); gb = __ldg(g4 + 1); gc = __ldg(g4 + 2); }
            Proj o;
            o.visible = false;
            if (!masked) project_core(cam, cfg, mu, ls, q, ol, o);
            float gmu[3] = {0, 0, 0}, gls[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gol = 0.f, grgb[3] = {0, 0, 0};
            float t_mu = 0.f, t_sig = 0.f;
            if (o.visible) {
                if (!WANT_POSE) { ga = __ldg(g4); gb = __ldg(g4 + 1); gc = __ldg(g4 + 2); }
                const float gu = ga.x, gv = ga.y, gA = ga.z, gB = ga.w, gC = gb.x, gop = gb.y, gd = gb.z;
                grgb[0] = gc.x; grgb[1] = gc.y; grgb[2] = gc.z;
                const float x = o.p[0], y = o.p[1], z = o.p[2];
                const float fx = cam.fx, fy = cam.fy;
                // conic Q = S2^{-1}: G2 = -Q Gq Q with Gq = [[gA, gB/2], [gB/2, gC]]
                const float Q00 = o.ca, Q01 = o.cb, Q11 = o.cc;
                const float hB = 0.5f * gB;
                const float M00 = Q00 * gA + Q01 * hB, M01 = Q00 * hB + Q01 * gC;
                const float M10 = Q01 * gA + Q11 * hB, M11 = Q01 * hB + Q11 * gC;
                const float G00 = -(M00 * Q00 + M01 * Q01);
                const float G01 = -(M00 * Q01 + M01 * Q11);
                const float G11 = -(M10 * Q01 + M11 * Q11);
                // dL/dSc = J^T G2 J (J rows: (J00, 0, J02), (0, J11, J12))
                const float J00 = o.J00, J02 = o.J02, J11 = o.J11, J12 = o.J12;
                float Gc[9];
                {
                    // columns of J: c0 = (J00, 0), c1 = (0, J11), c2 = (J02, J12)
                    const float c0x = J00, c1y = J11, c2x = J02, c2y = J12;
                    // G2 c_j
                    const float g0x = G00 * c0x;
                    const float g1x = G01 * c1y, g1y = G11 * c1y;
                    const float g2x = G00 * c2x + G01 * c2y, g2y = G01 * c2x + G11 * c2y;
                    Gc[0] = c0x * g0x;
                    Gc[1] = c0x * g1x;
                    Gc[2] = c0x * g2x;
                    Gc[4] = c1y * g1y;
                    Gc[5] = c1y * g2y;
                    Gc[8] = c2x * g2x + c2y * g2y;
                    Gc[3] = Gc[1]; Gc[6] = Gc[2]; Gc[7] = Gc[5];
                }
                // dL/dJ = 2 G2 J Sc ; only entries (0,0), (0,2), (1,1), (1,2) matter
                const float* S = o.Sc;
                // J Sc rows
                const float JS0x = J00 * S[0] + J02 * S[6], JS0y = J00 * S[1] + J02 * S[7], JS0z = J00 * S[2] + J02 * S[8];
                const float JS1x = J11 * S[3] + J12 * S[6], JS1y = J11 * S[4] + J12 * S[7], JS1z = J11 * S[5] + J12 * S[8];
                const float GJ00 = 2.f * (G00 * JS0x + G01 * JS1x);
                const float GJ02 = 2.f * (G00 * JS0z + G01 * JS1z);
                const float GJ11 = 2.f * (G01 * JS0y + G11 * JS1y);
                const float GJ12 = 2.f * (G01 * JS0z + G11 * JS1z);
                const float zi = 1.f / z, zi2 = zi * zi, zi3 = zi2 * zi;
                float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f;
                gp2 += GJ00 * (-fx * zi2) + GJ11 * (-fy * zi2);
                if (o.clx) gp2 += GJ02 * (fx * o.lx * zi2);
                else { gp0 += GJ02 * (-fx * zi2); gp2 += GJ02 * (2.f * fx * x * zi3); }
                if (o.cly) gp2 += GJ12 * (fy * o.ly * zi2);
                else { gp1 += GJ12 * (-fy * zi2); gp2 += GJ12 * (2.f * fy * y * zi3); }
                gp0 += gu * fx * zi;
                gp1 += gv * fy * zi;
                gp2 += -(gu * fx * x + gv * fy * y) * zi2 + gd;
                const float* R = cam.R;
                gmu[0] = R[0] * gp0 + R[3] * gp1 + R[6] * gp2;
                gmu[1] = R[1] * gp0 + R[4] * gp1 + R[7] * gp2;
                gmu[2] = R[2] * gp0 + R[5] * gp1 + R[8] * gp2;
                // GS = R^T Gc R
                float tmp[9], GS[9];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        tmp[3 * i + j] = R[i] * Gc[j] + R[3 + i] * Gc[3 + j] + R[6 + i] * Gc[6 + j];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        GS[3 * i + j] = tmp[3 * i] * R[j] + tmp[3 * i + 1] * R[3 + j] + tmp[3 * i + 2] * R[6 + j];
                if (WANT_SCORE) {
                    t_mu = sqrtf(gmu[0] * gmu[0] + gmu[1] * gmu[1] + gmu[2] * gmu[2]);
                    float fr = 0.f;
                    for (int i = 0; i < 9; ++i) fr += GS[i] * GS[i];
                    t_sig = sqrtf(fr);
                }
                if (WANT_GRADS) {
                    // Sigma = M M^T: dL/dM = 2 GS M
                    float GM[9];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j)
                            GM[3 * i + j] = 2.f * (GS[3 * i] * o.M[j] + GS[3 * i + 1] * o.M[3 + j] + GS[3 * i + 2] * o.M[6 + j]);
                    float GR[9];
                    for (int j = 0; j < 3; ++j) {
                        gls[j] = GM[j] * o.M[j] + GM[3 + j] * o.M[3 + j] + GM[6 + j] * o.M[6 + j];
                        for (int i = 0; i < 3; ++i) GR[3 * i + j] = GM[3 * i + j] * o.scale[j];
                    }
                    const float w = o.qn[0], qx = o.qn[1], qy = o.qn[2], qz = o.qn[3];
                    float gqn[4];
                    gqn[0] = 2.f * (-qz * GR[1] + qy * GR[2] + qz * GR[3] - qx * GR[5] - qy * GR[6] + qx * GR[7]);
                    gqn[1] = 2.f * (qy * GR[1] + qz * GR[2] + qy * GR[3] - 2.f * qx * GR[4] - w * GR[5] + qz * GR[6] + w * GR[7] - 2.f * qx * GR[8]);
                    gqn[2] = 2.f * (-2.f * qy * GR[0] + qx * GR[1] + w * GR[2] + qx * GR[3] + qz * GR[5] - w * GR[6] + qz * GR[7] - 2.f * qy * GR[8]);
                    gqn[3] = 2.f * (-2.f * qz * GR[0] - w * GR[1] + qx * GR[2] + w * GR[3] - 2.f * qz * GR[4] + qy * GR[5] + qx * GR[6] + qy * GR[7]);
                    const float dq = o.qn[0] * gqn[0] + o.qn[1] * gqn[1] + o.qn[2] * gqn[2] + o.qn[3] * gqn[3];
                    for (int i = 0; i < 4; ++i) gq[i] = (gqn[i] - o.qn[i] * dq) * o.qinv;
                    gol = gop * o.op * (1.f - o.op);
                }
                if (WANT_POSE) {
                    pose[0] = gp0; pose[1] = gp1; pose[2] = gp2;
                    // p x gp
                    pose[3] = y * gp2 - z * gp1;
                    pose[4] = z * gp0 - x * gp2;
                    pose[5] = x * gp1 - y * gp0;
                    // <Gc, [e_i]x S - S [e_i]x>: for the symmetric Gc and S it
                    // is tr([e_i]x (W - W^T)) with W = S Gc, i.e.
                    // 2 (W_jk - W_kj) for (i, j, k) a cyclic order of (0, 1, 2)
                    const float* Sm = o.Sc;
                    auto Wij = [&](int i, int j) {
                        return Sm[3 * i] * Gc[j] + Sm[3 * i + 1] * Gc[3 + j] + Sm[3 * i + 2] * Gc[6 + j];
                    };
                    pose[3] += 2.f * (Wij(1, 2) - Wij(2, 1));
                    pose[4] += 2.f * (Wij(2, 0) - Wij(0, 2));
                    pose[5] += 2.f * (Wij(0, 1) - Wij(1, 0));
                }
            } else if (!masked && WANT_GRADS) {
                // rgb gradient is independent of visibility only through grad2d,
                // which is zero for culled Gaussians; keep zeros.
            }
            if (ADAM) {
                const AdamMap& A = *adam;
                float* const gv[5] = {gmu, gls, gq, &gol, grgb};
                const int width[5] = {3, 3, 4, 1, 3};
    #pragma unroll
                for (int t = 0; t < 5; ++t)
    #pragma unroll
                    for (int i = 0; i < width[t]; ++i) {
                        const size_t e = (size_t)width[t] * k + i;
                        float pp = A.p[t][e], mm = A.m[t][e], vv = A.v[t][e];
                        adam_elem(pp, mm, vv, gv[t][i], A.lr, A.b1, A.b2, A.c1, A.c2, A.eps);
                        A.p[t][e] = pp;
                        A.m[t][e] = mm;
                        A.v[t][e] = vv;
                    }
            }
            if (WANT_GRADS) {
                if (grads.means) for (int i = 0; i < 3; ++i) grads.means[3 * k + i] = gmu[i];
                if (grads.log_scales) for (int i = 0; i < 3; ++i) grads.log_scales[3 * k + i] = gls[i];
                if (grads.quats) for (int i = 0; i < 4; ++i) grads.quats[4 * k + i] = gq[i];
                if (grads.opacity_logit) grads.opacity_logit[k] = gol;
                if (grads.rgb) for (int i = 0; i < 3; ++i) grads.rgb[3 * k + i] = o.visible ? grgb[i] : 0.f;
            }
            if (WANT_SCORE) {
                score[2 * k] = t_mu;
                score[2 * k + 1] = t_sig;
            }
        }
        if (WANT_POSE) {
    #pragma unroll
            for (int i = 0; i < 6; ++i) pacc[i] = df_add(pacc[i], DF{pose[i], 0.f});
        }
    }
    if (WANT_POSE) {
        // warp sums as float32 pairs (error-free two-sums, a reduce-scatter
        // of the six components), then the block's 8 warp pairs in order
        __shared__ float2 ws[PB_THREADS / 32][6];
        const int wid = threadIdx.x >> 5;
        DF v[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = pacc[i];
        const DF tot = warp_merge<6, DF, MergeDF>(v);  // 8 pair exchanges for the six components
        const int owner = merge_owner<6>();
        if (owner >= 0) ws[wid][owner] = make_float2(tot.hi, tot.lo);
        __syncthreads();
        if (threadIdx.x < 6) {
            DF s{0.f, 0.f};
            for (int w = 0; w < PB_THREADS / 32; ++w) {
                const float2 v = ws[w][threadIdx.x];
                s = df_add(s, DF{v.x, v.y});
            }
            pose_part[(size_t)blk * 6 + threadIdx.x] = make_float2(s.hi, s.lo);
        }
        pose_final_last_block(pose_part, nblk, pose_out, ticket, step);
    }
}

template <bool WANT_GRADS, bool WANT_POSE, bool WANT_SCORE>
__global__ void __launch_bounds__(PB_THREADS) k_project_bwd(gs_camera cam, gs_config cfg,
                                                            gs_gaussians g, const float* __restrict__ grad2d,
                                                            gs_grads grads, float* __restrict__ score,
                                                            float2* __restrict__ pose_part,
                                                            double* __restrict__ pose_out,
                                                            unsigned int* __restrict__ ticket, gs_pose_step step) {
    project_bwd_body<WANT_GRADS, WANT_POSE, WANT_SCORE>(cam, cfg, g, grad2d, grads, score, pose_part, pose_out,
                                                        ticket, step, (int)blockIdx.x, (int)gridDim.x);
}

// ---------------------------------------------------------------------------
// Multi-session waves: the projection with the binning's tile rows, and the
// backward projection with the pose step, over every job of a wave
// ---------------------------------------------------------------------------
struct WaveProjJob {
    gs_camera cam;
    gs_gaussians g;
    float* splats;
    int64_t per;
    int ntiles;
    uint32_t* hist;
    uint2* rects;
    // zeroed here for the later stages of the wave: the column scan's ticket,
    // the backward projection's ticket, the loss and the 2D gradients
    unsigned int* bin_ticket;
    unsigned int* bwd_ticket;
    double* loss;
    float* grad2d;
};

__global__ void __launch_bounds__(256) k_wave_project_hist(const gs_config cfg,
                                                           const __grid_constant__ Wave<WaveProjJob> W) {
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveProjJob& J = W.job[j];
    const int blk = (int)blockIdx.x - W.start[j];
    if (blk == 0 && threadIdx.x == 0) {
        *J.bin_ticket = 0u;
        *J.bwd_ticket = 0u;
        *J.loss = 0.0;
    }
    // this CTA's Gaussians' 2D gradient rows (the backward accumulates into them)
    const int64_t k0 = (int64_t)blk * J.per, k1 = min(J.g.n, k0 + J.per);
    float4* g4 = reinterpret_cast<float4*>(J.grad2d);
    for (int64_t q = 3 * k0 + threadIdx.x; q < 3 * k1; q += blockDim.x) g4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    project_hist_body<GS_F32>(J.cam, cfg, J.g, J.splats, J.per, J.ntiles, J.hist, J.rects, blk);
}

struct WavePbJob {
    gs_camera cam;
    gs_gaussians g;
    const float* grad2d;
    float* score;
    float2* part;
    double* pose_out;
    unsigned int* ticket;
    gs_pose_step step;
};

template <bool WANT_SCORE>
__global__ void __launch_bounds__(PB_THREADS) k_wave_project_bwd(const gs_config cfg,
                                                                 const __grid_constant__ Wave<WavePbJob> W) {
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WavePbJob& J = W.job[j];
    const gs_grads none = {nullptr, nullptr, nullptr, nullptr, nullptr};
    project_bwd_body<false, true, WANT_SCORE>(J.cam, cfg, J.g, J.grad2d, none, J.score, J.part, J.pose_out,
                                              J.ticket, J.step, (int)blockIdx.x - W.start[j],
                                              W.start[j + 1] - W.start[j]);
}

// Launches k_project_hist (nb CTAs of `per` Gaussians; ntiles words of
// dynamic shared memory).
gs_status launch_project_hist(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g, int rec_dtype,
                              void* splats, int64_t per, unsigned nb, int ntiles, uint32_t* hist, void* rects,
                              cudaStream_t st) {
    const size_t sm = sizeof(uint32_t) * (size_t)ntiles;
    uint2* r = (uint2*)rects;
    if (rec_dtype == GS_F32) k_project_hist<GS_F32><<<nb, 256, sm, st>>>(*cam, *cfg, *g, splats, per, ntiles, hist, r);
    else if (rec_dtype == GS_BF16) k_project_hist<GS_BF16><<<nb, 256, sm, st>>>(*cam, *cfg, *g, splats, per, ntiles, hist, r);
    else k_project_hist<GS_F16><<<nb, 256, sm, st>>>(*cam, *cfg, *g, splats, per, ntiles, hist, r);
    return check_launch("k_project_hist");
}

}  // namespace gs

using namespace gs;

static gs_status check_camera(const gs_camera* cam) {
    if (!cam) return set_error(GS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1)
        return set_error(GS_ERR_INVALID_ARG, "bad camera size %d x %d or stride %d,%d", cam->width,
                         cam->height, cam->sx, cam->sy);
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return set_error(GS_ERR_INVALID_ARG, "focal length must be > 0");
    if (cam->width > (1 << 20) || cam->height > (1 << 20))
        return set_error(GS_ERR_INVALID_ARG, "image larger than 2^20 pixels per side");
    return GS_OK;
}

static gs_status check_gaussians(const gs_gaussians* g) {
    if (!g) return set_error(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0 || g->n > (int64_t)0xFFFFFFF0LL) return set_error(GS_ERR_INVALID_ARG, "bad Gaussian count");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->rgb))
        return set_error(GS_ERR_INVALID_ARG, "a Gaussian parameter array is NULL");
    return GS_OK;
}

namespace gs {
// gs_project's argument checks (the record pointer aside).
gs_status project_checks(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g, int rec_dtype) {
    if (!cfg) return set_error(GS_ERR_INVALID_ARG, "config is NULL");
    gs_status s;
    if ((s = check_camera(cam)) != GS_OK) return s;
    if ((s = check_gaussians(g)) != GS_OK) return s;
    if (rec_dtype != GS_F32 && rec_dtype != GS_BF16 && rec_dtype != GS_F16)
        return set_error(GS_ERR_INVALID_ARG, "bad record dtype %d", rec_dtype);
    return GS_OK;
}
}  // namespace gs

extern "C" gs_status gs_project(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                int rec_dtype, void* splats, gs_stream stream) {
    if (!cfg) return set_error(GS_ERR_INVALID_ARG, "config is NULL");
    gs_status s;
    if ((s = check_camera(cam)) != GS_OK) return s;
    if ((s = check_gaussians(g)) != GS_OK) return s;
    if (rec_dtype != GS_F32 && rec_dtype != GS_BF16 && rec_dtype != GS_F16)
        return set_error(GS_ERR_INVALID_ARG, "bad record dtype %d", rec_dtype);
    if (g->n == 0) return GS_OK;
    if (!splats || ((uintptr_t)splats & 15)) return set_error(GS_ERR_INVALID_ARG, "splats NULL or not 16-byte aligned");
    const int th = 256;
    const unsigned blocks = (unsigned)((g->n + th - 1) / th);
    if (rec_dtype == GS_F32) k_project<GS_F32><<<blocks, th, 0, (cudaStream_t)stream>>>(*cam, *cfg, *g, splats);
    else if (rec_dtype == GS_BF16) k_project<GS_BF16><<<blocks, th, 0, (cudaStream_t)stream>>>(*cam, *cfg, *g, splats);
    else k_project<GS_F16><<<blocks, th, 0, (cudaStream_t)stream>>>(*cam, *cfg, *g, splats);
    return check_launch("k_project");
}

size_t gs_project_bwd_ws(int64_t n) {
    const size_t nblk = (size_t)pb_blocks(n, PB_PER);
    return ((nblk * 6 * sizeof(double)) + 255 + 256) & ~(size_t)255;  // partials + ticket
}

extern "C" gs_status gs_project_bwd(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                    const float* grad2d, gs_grads* grads, double* pose_grad6,
                                    float* score_terms, void* workspace, size_t* workspace_bytes,
                                    gs_stream stream) {
    return gs_project_bwd_step(cfg, cam, g, grad2d, grads, pose_grad6, score_terms, nullptr, workspace,
                               workspace_bytes, stream);
}

extern "C" gs_status gs_project_bwd_step(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                         const float* grad2d, gs_grads* grads, double* pose_grad6,
                                         float* score_terms, const gs_pose_step* step, void* workspace,
                                         size_t* workspace_bytes, gs_stream stream) {
    if (!cfg || !workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "config or workspace_bytes is NULL");
    if (step) {
        if (!pose_grad6) return set_error(GS_ERR_INVALID_ARG, "a pose step needs pose_grad6");
        if (!step->pose || !step->adam) return set_error(GS_ERR_INVALID_ARG, "pose step: NULL pose or adam");
        if (!(step->beta1 >= 0.f && step->beta1 < 1.f) || !(step->beta2 >= 0.f && step->beta2 < 1.f) ||
            !(step->eps > 0.f))
            return set_error(GS_ERR_INVALID_ARG, "pose step: bad Adam constants");
    }
    const gs_pose_step no_step = {nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 0.f};
    const gs_pose_step ps = step ? *step : no_step;
    gs_status s;
    if ((s = check_camera(cam)) != GS_OK) return s;
    if ((s = check_gaussians(g)) != GS_OK) return s;
    const size_t need = gs_project_bwd_ws(g->n);
    if (!workspace) { *workspace_bytes = need; return GS_OK; }
    if (*workspace_bytes < need) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu bytes", *workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    const bool want_grads = grads && (grads->means || grads->log_scales || grads->quats ||
                                      grads->opacity_logit || grads->rgb);
    const bool want_pose = pose_grad6 != nullptr;
    const bool want_score = score_terms != nullptr;
    if (g->n == 0) {
        if (want_pose && cudaMemsetAsync(pose_grad6, 0, 6 * sizeof(double), st) != cudaSuccess)
            return set_error(GS_ERR_CUDA, "memset pose");
        if (step) return gs_pose_update(ps.pose, pose_grad6, ps.adam, ps.lr_trans, ps.lr_rot, ps.beta1, ps.beta2,
                                        ps.eps, stream);
        return GS_OK;
    }
    if (!grad2d) return set_error(GS_ERR_INVALID_ARG, "grad2d is NULL");
    gs_grads gg = grads ? *grads : gs_grads{nullptr, nullptr, nullptr, nullptr, nullptr};
    const unsigned nblk = (unsigned)pb_blocks(g->n, want_pose ? PB_PER : 1);
    float2* part = (float2*)workspace;
    unsigned int* ticket = (unsigned int*)((char*)workspace + need - 256);
    if (want_pose && cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "memset ticket");
#define GS_PB_LAUNCH(A, B, C_) \
    k_project_bwd<A, B, C_><<<nblk, PB_THREADS, 0, st>>>(*cam, *cfg, *g, grad2d, gg, score_terms, part, pose_grad6, \
                                                         ticket, ps)
    if (want_grads) {
        if (want_pose) { if (want_score) GS_PB_LAUNCH(true, true, true); else GS_PB_LAUNCH(true, true, false); }
        else { if (want_score) GS_PB_LAUNCH(true, false, true); else GS_PB_LAUNCH(true, false, false); }
    } else {
        if (want_pose) { if (want_score) GS_PB_LAUNCH(false, true, true); else GS_PB_LAUNCH(false, true, false); }
        else { if (want_score) GS_PB_LAUNCH(false, false, true); else return GS_OK; }
    }
#undef GS_PB_LAUNCH
    return check_launch("k_project_bwd");
}

extern "C" gs_status gs_pose_update(float* pose, const double* pose_grad6, float* adam, float lr_trans, float lr_rot,
                                    float beta1, float beta2, float eps, gs_stream stream) {
    if (!pose || !pose_grad6 || !adam) return set_error(GS_ERR_INVALID_ARG, "NULL pointer");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return set_error(GS_ERR_INVALID_ARG, "bad Adam constants");
    k_pose_update<<<1, 32, 0, (cudaStream_t)stream>>>(pose, pose_grad6, adam, lr_trans, lr_rot, beta1, beta2, eps);
    return check_launch("k_pose_update");
}

// ---------------------------------------------------------------------------
// Allocation-free variant of gs_project_bwd (see include/gs.h)
// ---------------------------------------------------------------------------
// Fixed scratch for gs_project_bwd_noalloc: room for the per-block pose
// partials of GS_NOALLOC_MAX_GAUSSIANS Gaussians plus the ticket word.  In
// host code this name is only a stand-in: the kernel gets the device address
// looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];
// the size: one float2 pose partial per component (6) and block of PB_THREADS
// Gaussians, plus the ticket word, rounded to 256 bytes (an upper bound: a
// block takes PB_PER x PB_THREADS Gaussians)
static_assert(PB_THREADS == 256 && PB_PER >= 1 && 6 * sizeof(float2) == 48,
              "GS_NOALLOC_SCRATCH_BYTES assumes at least 256 Gaussians and 48 bytes of pose partials per block");

static gs_status noalloc_scratch(void** out) {
    // One entry per device, written by a host thread's first call.  Threads
    // that race on an entry store the same address (relaxed atomics keep
    // that race defined).  cudaDeviceReset invalidates the entry: the
    // address is not looked up again until the process restarts.
    static std::atomic<void*> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return set_error(GS_ERR_CUDA, "no current device");
    void* p = cache[dev].load(std::memory_order_relaxed);
    if (!p) {
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return set_error(GS_ERR_CUDA, "scratch address: %s", cudaGetErrorString(e));
        cache[dev].store(p, std::memory_order_relaxed);
    }
    *out = p;
    return GS_OK;
}

extern "C" gs_status gs_project_bwd_noalloc(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                            const float* grad2d, gs_grads* grads, double* pose_grad6,
                                            float* score_terms, gs_stream stream) {
    if (!g) return set_error(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n > (int64_t)GS_NOALLOC_MAX_GAUSSIANS)
        return set_error(GS_ERR_INVALID_ARG, "n = %lld exceeds GS_NOALLOC_MAX_GAUSSIANS = %d", (long long)g->n,
                         GS_NOALLOC_MAX_GAUSSIANS);
    size_t need = 0;
    gs_status s = gs_project_bwd(cfg, cam, g, grad2d, grads, pose_grad6, score_terms, nullptr, &need, stream);
    if (s != GS_OK) return s;
    if (need > (size_t)GS_NOALLOC_SCRATCH_BYTES)
        return set_error(GS_ERR_INVALID_ARG, "scratch of %zu bytes exceeds the static %d", need, GS_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    if ((s = noalloc_scratch(&scratch)) != GS_OK) return s;
    size_t have = (size_t)GS_NOALLOC_SCRATCH_BYTES;
    return gs_project_bwd(cfg, cam, g, grad2d, grads, pose_grad6, score_terms, scratch, &have, stream);
}

// ---------------------------------------------------------------------------
// Backward projection with the map's Adam step (mapping iteration)
// ---------------------------------------------------------------------------
namespace gs {
template <bool WANT_SCORE>
__global__ void __launch_bounds__(PB_THREADS) k_project_bwd_adam(gs_camera cam, gs_config cfg, gs_gaussians g,
                                                                 const float* __restrict__ grad2d, gs_grads grads,
                                                                 float* __restrict__ score, AdamMap A,
                                                                 float* __restrict__ state) {
    // the step count: read by every block, advanced by the last (as gs_adam)
    const float step = __ldcg(state) + 1.f;
    A.c1 = 1.f - powf(A.b1, step);
    A.c2 = 1.f - powf(A.b2, step);
    const gs_pose_step none = {nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 0.f};
    project_bwd_body<true, false, WANT_SCORE, true>(cam, cfg, g, grad2d, grads, score, nullptr, nullptr, nullptr,
                                                    none, (int)blockIdx.x, (int)gridDim.x, &A);
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(reinterpret_cast<unsigned int*>(state + 1), 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        state[0] = step;
        *reinterpret_cast<unsigned int*>(state + 1) = 0u;
    }
}
}  // namespace gs

extern "C" gs_status gs_project_bwd_adam(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                         const float* grad2d, const gs_map_adam* adam, gs_grads* grads,
                                         float* score_terms, gs_stream stream) {
    if (!cfg || !adam) return set_error(GS_ERR_INVALID_ARG, "config or adam is NULL");
    gs_status s;
    if ((s = check_camera(cam)) != GS_OK) return s;
    if ((s = check_gaussians(g)) != GS_OK) return s;
    if (!(adam->beta1 >= 0.f && adam->beta1 < 1.f) || !(adam->beta2 >= 0.f && adam->beta2 < 1.f) ||
        !(adam->eps > 0.f))
        return set_error(GS_ERR_INVALID_ARG, "bad Adam constants");
    if (!adam->state) return set_error(GS_ERR_INVALID_ARG, "Adam state is NULL");
    for (int t = 0; t < 5; ++t)
        if (g->n > 0 && (!adam->m[t] || !adam->v[t])) return set_error(GS_ERR_INVALID_ARG, "moment array %d is NULL", t);
    if (g->n == 0) return GS_OK;
    if (!grad2d) return set_error(GS_ERR_INVALID_ARG, "grad2d is NULL");
    AdamMap A;
    float* const P[5] = {(float*)g->means, (float*)g->log_scales, (float*)g->quats, (float*)g->opacity_logit,
                         (float*)g->rgb};
    for (int t = 0; t < 5; ++t) {
        A.p[t] = P[t];
        A.m[t] = adam->m[t];
        A.v[t] = adam->v[t];
    }
    A.lr = adam->lr;
    A.b1 = adam->beta1;
    A.b2 = adam->beta2;
    A.eps = adam->eps;
    A.c1 = A.c2 = 1.f;
    const gs_grads gg = grads ? *grads : gs_grads{nullptr, nullptr, nullptr, nullptr, nullptr};
    const unsigned nblk = (unsigned)pb_blocks(g->n, 1);
    cudaStream_t st = (cudaStream_t)stream;
    if (score_terms)
        k_project_bwd_adam<true><<<nblk, PB_THREADS, 0, st>>>(*cam, *cfg, *g, grad2d, gg, score_terms, A, adam->state);
    else
        k_project_bwd_adam<false><<<nblk, PB_THREADS, 0, st>>>(*cam, *cfg, *g, grad2d, gg, nullptr, A, adam->state);
    return check_launch("k_project_bwd_adam");
}

// ---------------------------------------------------------------------------
// Wave launchers (gs_track_wave)
// ---------------------------------------------------------------------------
namespace gs {

unsigned int* wave_bwd_ticket(const gs_track_job& j) {
    const size_t need = gs_project_bwd_ws(j.g.n);
    return (unsigned int*)((char*)j.bwd_workspace + need - 256);
}

gs_status wave_project_hist(const gs_config& cfg, const gs_track_job* jobs, const WaveBin* bins, int n,
                            cudaStream_t st) {
    Wave<WaveProjJob> W;  // the launch's parameter block (copied at launch)
    W.n = n;
    int blocks = 0, smax = 1;
    for (int j = 0; j < n; ++j) {
        const gs_track_job& t = jobs[j];
        const WaveBin& b = bins[j];
        W.start[j] = blocks;
        blocks += (int)b.nb;
        smax = std::max(smax, b.ntiles);
        W.job[j] = WaveProjJob{t.cam, t.g, t.splats, b.per, b.ntiles, b.hist, (uint2*)b.rects, b.ticket,
                               wave_bwd_ticket(t), t.loss, t.grad2d};
    }
    W.start[n] = blocks;
    k_wave_project_hist<<<(unsigned)blocks, 256, sizeof(uint32_t) * (size_t)smax, st>>>(cfg, W);
    return check_launch("k_wave_project_hist");
}

gs_status wave_project_bwd(const gs_config& cfg, const gs_track_job* jobs, int n, cudaStream_t st) {
    Wave<WavePbJob> W;
    W.n = n;
    int blocks = 0;
    bool score = false;
    for (int j = 0; j < n; ++j) score = score || jobs[j].score_terms;
    for (int j = 0; j < n; ++j) {
        const gs_track_job& t = jobs[j];
        W.start[j] = blocks;
        blocks += (int)pb_blocks(t.g.n, PB_PER);
        W.job[j] = WavePbJob{t.cam, t.g, t.grad2d, t.score_terms, (float2*)t.bwd_workspace, t.pose_grad6,
                             wave_bwd_ticket(t), t.step};
    }
    W.start[n] = blocks;
    if (score) {  // (gs_track_wave checked that every job has one)
        k_wave_project_bwd<true><<<(unsigned)blocks, PB_THREADS, 0, st>>>(cfg, W);
    } else {
        k_wave_project_bwd<false><<<(unsigned)blocks, PB_THREADS, 0, st>>>(cfg, W);
    }
    return check_launch("k_wave_project_bwd");
}

}  // namespace gs
