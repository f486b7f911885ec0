// A-9 gradient-reuse pruning (Sec. 4.1, Eq. 7), the change ratio of
// tile-Gaussian intersections, compaction, and A-10 keyframe-driven dynamic
// downsampling (Sec. 4.2) on sm_103a.
//
// Selection is a radix select on the unique 64-bit key (score bits << 32 |
// id): eight 8-bit digit passes, each CTA re-deriving the prefix chosen so
// far from the previous passes' histograms (a few hundred integer ops), so
// no pass needs a separate pick launch or a host round trip.  Scores are
// non-negative, so their float bits order like their values.
#include "gs_internal.cuh"

namespace gs {

typedef unsigned long long u64;

#define PR_THREADS 256
#define PR_CHUNK 2048

struct PruneState {
    u64 n_active;  // unmasked Gaussians
};

__device__ __forceinline__ u64 score_key(const float* __restrict__ st, int64_t k, float lam) {
    // Eq. 7 in float32: product rounded, then sum rounded (no fused multiply-add)
    const float s = __fadd_rn(st[2 * k], __fmul_rn(lam, st[2 * k + 1]));
    return ((u64)__float_as_uint(s) << 32) | (u64)(uint32_t)k;
}

__global__ void __launch_bounds__(PR_THREADS) k_prune_count(const uint8_t* __restrict__ mask, int64_t n,
                                                            PruneState* __restrict__ state) {
    __shared__ unsigned int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    unsigned int c = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        c += mask[k] == 0 ? 1u : 0u;
    atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&state->n_active, (u64)s_cnt);
}

// m = min(floor(frac * n_active), max_select): rank (1-based) of the largest
// selected key.
__device__ __forceinline__ u64 select_count(const PruneState* st, float frac, int64_t max_select) {
    const double m = floor((double)frac * (double)st->n_active);
    u64 mm = (u64)m;
    if ((int64_t)mm > max_select) mm = (u64)(max_select < 0 ? 0 : max_select);
    return mm;
}

// Re-derives the key prefix fixed by passes [0, p) from their histograms.
__device__ __forceinline__ void derive_prefix(const unsigned int* __restrict__ hist, int p, u64 m, u64& prefix,
                                              u64& remaining) {
    prefix = 0;
    remaining = m;
    for (int q = 0; q < p; ++q) {
        const unsigned int* h = hist + q * 256;
        u64 cum = 0;
        int b = 0;
        for (; b < 256; ++b) {
            const u64 c = h[b];
            if (cum + c >= remaining) break;
            cum += c;
        }
        if (b == 256) b = 255;  // only reachable if m exceeds the candidates
        remaining -= cum;
        prefix |= (u64)b << (56 - 8 * q);
    }
}

__global__ void __launch_bounds__(PR_THREADS) k_select_pass(const float* __restrict__ st, const uint8_t* __restrict__ mask,
                                                            int64_t n, float lam, float frac, int64_t max_select,
                                                            const PruneState* __restrict__ state,
                                                            unsigned int* __restrict__ hist, int p) {
    __shared__ unsigned int sh[256];
    __shared__ u64 s_prefix;
    __shared__ int s_skip;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
    if (threadIdx.x == 0) {
        const u64 m = select_count(state, frac, max_select);
        u64 prefix, rem;
        derive_prefix(hist, p, m, prefix, rem);
        s_prefix = prefix;
        s_skip = (m == 0);
    }
    __syncthreads();
    if (s_skip) return;
    const u64 prefix = s_prefix;
    const int shift = 56 - 8 * p;
    const u64 hi_mask = p == 0 ? 0ull : (~0ull << (64 - 8 * p));
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (mask[k]) continue;
        const u64 key = score_key(st, k, lam);
        if ((key & hi_mask) != prefix) continue;
        atomicAdd(&sh[(key >> shift) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (sh[i]) atomicAdd(hist + p * 256 + i, sh[i]);
}

__global__ void __launch_bounds__(PR_THREADS) k_select_mask(const float* __restrict__ st, uint8_t* __restrict__ mask,
                                                            int64_t n, float lam, float frac, int64_t max_select,
                                                            const PruneState* __restrict__ state,
                                                            const unsigned int* __restrict__ hist) {
    __shared__ u64 s_kth;
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        const u64 m = select_count(state, frac, max_select);
        u64 prefix, rem;
        derive_prefix(hist, 8, m, prefix, rem);
        s_kth = prefix;
        s_skip = (m == 0);
    }
    __syncthreads();
    if (s_skip) return;
    const u64 kth = s_kth;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (mask[k]) continue;
        if (score_key(st, k, lam) <= kth) mask[k] = 1;
    }
}

// Compaction map: exclusive scan of (mask == 0) in id order.
__global__ void __launch_bounds__(PR_THREADS) k_keep_count(const uint8_t* __restrict__ mask, int64_t n,
                                                           u64* __restrict__ partial) {
    __shared__ unsigned int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * PR_CHUNK;
    unsigned int c = 0;
    for (int j = threadIdx.x; j < PR_CHUNK; j += PR_THREADS) {
        const int64_t k = base + j;
        if (k < n && mask[k] == 0) ++c;
    }
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_keep_scan(u64* __restrict__ partial, int nchunk, int64_t* __restrict__ n_kept) {
    __shared__ u64 s_warp[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u64 carry = 0;
    for (int base = 0; base < nchunk; base += 1024) {
        const int i = base + threadIdx.x;
        const u64 v = i < nchunk ? partial[i] : 0ull;
        u64 x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        if (wid == 0) {
            u64 w = s_warp[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const u64 y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const u64 before = wid > 0 ? s_warp[wid - 1] : 0ull;
        const u64 total = s_warp[31];
        if (i < nchunk) partial[i] = carry + before + x - v;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_kept = (int64_t)carry;
}

__global__ void __launch_bounds__(PR_THREADS) k_keep_write(const uint8_t* __restrict__ mask, int64_t n,
                                                           const u64* __restrict__ partial, uint32_t* __restrict__ map) {
    // each warp takes 64 consecutive ids (2 per lane) of the chunk, in order
    __shared__ unsigned int s_warp[PR_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * PR_CHUNK;
    u64 off = partial[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int seg = 0; seg < PR_CHUNK; seg += PR_THREADS) {
        const int64_t k = base + seg + threadIdx.x;
        const bool keep = k < n && mask[k] == 0;
        const unsigned int bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[wid] = __popc(bal);
        __syncthreads();
        unsigned int before = 0, total = 0;
        for (int w = 0; w < PR_THREADS / 32; ++w) {
            if (w < wid) before += s_warp[w];
            total += s_warp[w];
        }
        if (k < n) map[k] = keep ? (uint32_t)(off + before + __popc(bal & ((1u << lane) - 1u))) : 0xFFFFFFFFu;
        off += total;
        __syncthreads();
    }
}

// |rect_a| + |rect_b| - 2 |rect_a & rect_b| and |rect_a| summed over Gaussians.
template <int DT>
__global__ void __launch_bounds__(PR_THREADS) k_change(gs_camera cam, float alpha_min, const void* __restrict__ sa,
                                                       const void* __restrict__ sb, int64_t n, u64* __restrict__ acc) {
    const Grid grid = make_grid(cam);
    u64 sym = 0, na = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int ax0, ax1, ay0, ay1, bx0, bx1, by0, by1;
        const int ca = tile_rect(grid, load_geom<DT>(sa, (uint32_t)k), alpha_min, ax0, ax1, ay0, ay1);
        const int cb = tile_rect(grid, load_geom<DT>(sb, (uint32_t)k), alpha_min, bx0, bx1, by0, by1);
        int inter = 0;
        if (ca > 0 && cb > 0) {
            const int ix = min(ax1, bx1) - max(ax0, bx0), iy = min(ay1, by1) - max(ay0, by0);
            if (ix > 0 && iy > 0) inter = ix * iy;
        }
        sym += (u64)(ca + cb - 2 * inter);
        na += (u64)ca;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sym += __shfl_xor_sync(0xffffffffu, sym, o);
        na += __shfl_xor_sync(0xffffffffu, na, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, sym);
        atomicAdd(acc + 1, na);
    }
}

__global__ void k_change_final(const u64* __restrict__ acc, float* __restrict__ out) {
    const double na = (double)acc[1];
    *out = (float)((double)acc[0] / (na > 1.0 ? na : 1.0));
}

__global__ void __launch_bounds__(256) k_compact(const float* __restrict__ src, int64_t n, int width,
                                                 const uint32_t* __restrict__ map, float* __restrict__ dst) {
    const int64_t total = n * (int64_t)width;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = q / width;
        const uint32_t to = map[k];
        if (to != 0xFFFFFFFFu) dst[(int64_t)to * width + (q - k * width)] = src[q];
    }
}

__global__ void __launch_bounds__(256) k_gather(const float* __restrict__ full, int C, int W, int H, int sx, int sy,
                                                float* __restrict__ out) {
    const int Ws = (W + sx - 1) / sx, Hs = (H + sy - 1) / sy;
    const int64_t total = (int64_t)C * Ws * Hs;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % Ws);
        const int64_t r = q / Ws;
        const int j = (int)(r % Hs);
        const int c = (int)(r / Hs);
        out[q] = full[((int64_t)c * H + (int64_t)j * sy) * W + (int64_t)i * sx];
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace gs

using namespace gs;

extern "C" int32_t gs_next_interval(const gs_config* cfg, int32_t K, float change_ratio) {
    if (!cfg || K < 1) return 1;
    int32_t nk = change_ratio > cfg->change_thr ? K / 2 : 2 * K;
    if (nk < 1) nk = 1;
    if (nk > cfg->k_max) nk = cfg->k_max;
    return nk;
}

extern "C" gs_status gs_prune(const gs_config* cfg, const float* score_terms, int64_t n, uint8_t* mask_inout,
                              int iter_in_interval, int* k_inout, float change_ratio, int64_t max_select,
                              uint32_t* compact_map_out, int64_t* n_kept_out, void* workspace,
                              size_t* workspace_bytes, gs_stream stream) {
    if (!cfg || !workspace_bytes || !k_inout) return set_error(GS_ERR_INVALID_ARG, "config, k_inout or workspace_bytes NULL");
    if (n < 0 || n > (int64_t)0xFFFFFFF0LL) return set_error(GS_ERR_INVALID_ARG, "bad Gaussian count");
    if (*k_inout < 1) return set_error(GS_ERR_INVALID_ARG, "interval K must be >= 1");
    const int64_t nchunk = (n + PR_CHUNK - 1) / PR_CHUNK;
    const size_t off_hist = 0, off_state = a256(8 * 256 * sizeof(unsigned int));
    const size_t off_part = a256(off_state + sizeof(PruneState));
    const size_t need = a256(off_part + sizeof(u64) * (size_t)(nchunk > 0 ? nchunk : 1));
    if (!workspace) { *workspace_bytes = need; return GS_OK; }
    if (*workspace_bytes < need) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    const int sms = num_sms();
    const int64_t want = (n + PR_THREADS - 1) / PR_THREADS;
    const unsigned nb = (unsigned)(want < 4 * sms ? (want > 0 ? want : 1) : 4 * sms);
    gs_status s;
    if (iter_in_interval == 0) {
        if (n == 0) return GS_OK;
        if (!score_terms || !mask_inout) return set_error(GS_ERR_INVALID_ARG, "score_terms or mask NULL");
        if (cudaMemsetAsync(ws, 0, off_part, st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset prune state");
        unsigned int* hist = (unsigned int*)(ws + off_hist);
        PruneState* state = (PruneState*)(ws + off_state);
        k_prune_count<<<nb, PR_THREADS, 0, st>>>(mask_inout, n, state);
        if ((s = check_launch("k_prune_count")) != GS_OK) return s;
        for (int p = 0; p < 8; ++p) {
            k_select_pass<<<nb, PR_THREADS, 0, st>>>(score_terms, mask_inout, n, cfg->lambda_score, cfg->prune_frac,
                                                     max_select, state, hist, p);
            if ((s = check_launch("k_select_pass")) != GS_OK) return s;
        }
        k_select_mask<<<nb, PR_THREADS, 0, st>>>(score_terms, mask_inout, n, cfg->lambda_score, cfg->prune_frac,
                                                 max_select, state, hist);
        return check_launch("k_select_mask");
    }
    if (iter_in_interval == *k_inout) {
        if (!compact_map_out || !n_kept_out || (n > 0 && !mask_inout))
            return set_error(GS_ERR_INVALID_ARG, "compact map, n_kept or mask NULL");
        if (n == 0) {
            if (cudaMemsetAsync(n_kept_out, 0, sizeof(int64_t), st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset");
        } else {
            u64* part = (u64*)(ws + off_part);
            k_keep_count<<<(unsigned)nchunk, PR_THREADS, 0, st>>>(mask_inout, n, part);
            if ((s = check_launch("k_keep_count")) != GS_OK) return s;
            k_keep_scan<<<1, 1024, 0, st>>>(part, (int)nchunk, n_kept_out);
            if ((s = check_launch("k_keep_scan")) != GS_OK) return s;
            k_keep_write<<<(unsigned)nchunk, PR_THREADS, 0, st>>>(mask_inout, n, part, compact_map_out);
            if ((s = check_launch("k_keep_write")) != GS_OK) return s;
        }
        *k_inout = gs_next_interval(cfg, *k_inout, change_ratio);
        return GS_OK;
    }
    return GS_OK;
}

extern "C" gs_status gs_change_ratio(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats_a,
                                     const void* splats_b,
                                     int64_t n, void* workspace, size_t* workspace_bytes, float* ratio_out,
                                     gs_stream stream) {
    if (!cfg || !cam || !workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "config, camera or workspace_bytes NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1)
        return set_error(GS_ERR_INVALID_ARG, "bad camera size or stride");
    if (rec_dtype != GS_F32 && rec_dtype != GS_BF16 && rec_dtype != GS_F16)
        return set_error(GS_ERR_INVALID_ARG, "bad record dtype");
    if (n < 0) return set_error(GS_ERR_INVALID_ARG, "bad Gaussian count");
    const size_t need = 256;
    if (!workspace) { *workspace_bytes = need; return GS_OK; }
    if (*workspace_bytes < need) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, need);
    if (!ratio_out || (n > 0 && (!splats_a || !splats_b))) return set_error(GS_ERR_INVALID_ARG, "NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    u64* acc = (u64*)workspace;
    if (cudaMemsetAsync(acc, 0, 2 * sizeof(u64), st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset");
    gs_status s;
    if (n > 0) {
        const int sms = num_sms();
        const int64_t want = (n + PR_THREADS - 1) / PR_THREADS;
        const unsigned nb = (unsigned)(want < 4 * sms ? want : 4 * sms);
        if (rec_dtype == GS_F32) k_change<GS_F32><<<nb, PR_THREADS, 0, st>>>(*cam, cfg->alpha_min, splats_a, splats_b, n, acc);
        else if (rec_dtype == GS_BF16) k_change<GS_BF16><<<nb, PR_THREADS, 0, st>>>(*cam, cfg->alpha_min, splats_a, splats_b, n, acc);
        else k_change<GS_F16><<<nb, PR_THREADS, 0, st>>>(*cam, cfg->alpha_min, splats_a, splats_b, n, acc);
        if ((s = check_launch("k_change")) != GS_OK) return s;
    }
    k_change_final<<<1, 1, 0, st>>>(acc, ratio_out);
    return check_launch("k_change_final");
}

extern "C" gs_status gs_compact(const float* src, int64_t n, int32_t width, const uint32_t* compact_map, float* dst,
                                gs_stream stream) {
    if (n < 0 || width < 1) return set_error(GS_ERR_INVALID_ARG, "bad size");
    if (n == 0) return GS_OK;
    if (!src || !compact_map || !dst) return set_error(GS_ERR_INVALID_ARG, "NULL pointer");
    const int sms = num_sms();
    const int64_t want = (n * width + 255) / 256;
    const unsigned nb = (unsigned)(want < 8 * sms ? want : 8 * sms);
    k_compact<<<nb, 256, 0, (cudaStream_t)stream>>>(src, n, width, compact_map, dst);
    return check_launch("k_compact");
}

extern "C" gs_status gs_downsample(int64_t frame_idx, int64_t last_kf_idx, int is_keyframe, int m, int32_t* sx,
                                   int32_t* sy, const float* target_full, int32_t channels, int32_t W, int32_t H,
                                   float* target_out, gs_stream stream) {
    if (!sx || !sy) return set_error(GS_ERR_INVALID_ARG, "sx or sy NULL");
    if (is_keyframe) {
        *sx = 1;
        *sy = 1;
    } else {
        if (m < 2 || (m & (m - 1)) != 0) return set_error(GS_ERR_INVALID_ARG, "m must be a power of two >= 2");
        if (frame_idx <= last_kf_idx) return set_error(GS_ERR_INVALID_ARG, "frame must follow its keyframe");
        // R0/R = max(16 / m^(n-k-1), 4)
        const int64_t e = frame_idx - last_kf_idx - 1;
        int64_t ratio = 16;
        for (int64_t q = 0; q < e && ratio > 4; ++q) ratio /= m;
        if (ratio < 4) ratio = 4;
        if (ratio == 16) { *sx = 4; *sy = 4; }
        else if (ratio == 8) { *sx = 4; *sy = 2; }
        else { *sx = 2; *sy = 2; }
    }
    if (!target_full) return GS_OK;
    if (!target_out || channels < 1 || W < 1 || H < 1) return set_error(GS_ERR_INVALID_ARG, "bad gather arguments");
    const int64_t total = (int64_t)channels * ((W + *sx - 1) / *sx) * ((H + *sy - 1) / *sy);
    const int sms = num_sms();
    const int64_t want = (total + 255) / 256;
    const unsigned nb = (unsigned)(want < 8 * sms ? want : 8 * sms);
    k_gather<<<nb, 256, 0, (cudaStream_t)stream>>>(target_full, channels, W, H, *sx, *sy, target_out);
    return check_launch("k_gather");
}
