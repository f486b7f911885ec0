// A-2..A-4: tile intersection, key duplication, 64-bit radix sort and tile
// ranges (Sec. 2.1, Step 1-2 and Step 2) on sm_103a.
//
// Pipeline (all on the caller's stream, no host synchronisation; the key
// count stays on the device and the sort kernels read it):
//   k_bin_count  per 2048-Gaussian chunk: sum of tiles touched
//   k_bin_scan   one CTA: exclusive scan of the chunk sums -> key count
//   k_bin_dup    per chunk: block scan, then each Gaussian writes its
//                (tile << 32 | depth bits, id) pairs in id order
//   k_sort_hist  digit histograms of every pass in one read of the keys
//   k_sort_pass  one per 8-bit digit: persistent CTAs take 4096-key tiles in
//                ticket order, rank keys with warp match-any, find each
//                digit's global offset by decoupled look-back over the
//                previous tiles (bounded spins), and scatter through shared
//                memory so that each digit run is written contiguously
//   k_ranges     first/last index of every tile in the sorted keys
// Every pass is stable, so keys with equal (tile, depth) keep id order.
#include "gs_internal.cuh"

namespace gs {

#define BIN_THREADS 256
#define BIN_PER_THREAD 8
#define BIN_CHUNK (BIN_THREADS * BIN_PER_THREAD)

#define SORT_THREADS 512
#define SORT_KPT 8
#define SORT_TILE (SORT_THREADS * SORT_KPT)
#define SORT_WARPS (SORT_THREADS / 32)
#define RADIX 256

#define FLAG_AGG (1u << 30)
#define FLAG_PREFIX (2u << 30)
#define COUNT_MASK ((1u << 30) - 1u)
#define SPIN_LIMIT (1 << 22)

typedef unsigned long long u64;

// ---------------------------------------------------------------------------
// Block-level exclusive scan of 64-bit values (blockDim.x multiple of 32,
// at most 1024 threads).
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 block_excl_scan_u64(u64 v, u64* s_warp, u64& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u64 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        u64 w = lane < nw ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u64 y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[nw - 1];
    u64 before = wid > 0 ? s_warp[wid - 1] : 0ull;
    __syncthreads();
    return before + x - v;
}

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_bin_count(gs_camera cam, const void* __restrict__ splats,
                                                           int64_t n, u64* __restrict__ partial) {
    __shared__ u64 s_warp[32];
    const Grid grid = make_grid(cam);
    const int64_t k0 = (int64_t)blockIdx.x * BIN_CHUNK + (int64_t)threadIdx.x * BIN_PER_THREAD;
    u64 sum = 0;
#pragma unroll
    for (int j = 0; j < BIN_PER_THREAD; ++j) {
        const int64_t k = k0 + j;
        if (k < n) {
            float x, y, d;
            int r;
            load_geom<DT>(splats, (uint32_t)k, x, y, d, r);
            int a, b, c, e;
            sum += (u64)tile_rect(grid, x, y, r, a, b, c, e);
        }
    }
    u64 total;
    block_excl_scan_u64(sum, s_warp, total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Exclusive scan of the chunk sums in place; writes the total key count.
__global__ void __launch_bounds__(1024) k_bin_scan(u64* __restrict__ partial, int nchunk,
                                                   int64_t* __restrict__ n_keys, int64_t cap,
                                                   unsigned int* __restrict__ status) {
    __shared__ u64 s_warp[32];
    u64 carry = 0;
    for (int base = 0; base < nchunk; base += 1024) {
        const int i = base + threadIdx.x;
        const u64 v = i < nchunk ? partial[i] : 0ull;
        u64 total;
        const u64 ex = block_excl_scan_u64(v, s_warp, total);
        if (i < nchunk) partial[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        *n_keys = (int64_t)carry;
        if ((int64_t)carry > cap) raise_status(status, GS_ERR_CAPACITY);
    }
}

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_bin_dup(gs_camera cam, const void* __restrict__ splats,
                                                         int64_t n, const u64* __restrict__ partial,
                                                         int64_t cap, u64* __restrict__ keys,
                                                         uint32_t* __restrict__ vals) {
    __shared__ u64 s_warp[32];
    const Grid grid = make_grid(cam);
    const int64_t k0 = (int64_t)blockIdx.x * BIN_CHUNK + (int64_t)threadIdx.x * BIN_PER_THREAD;
    u64 sum = 0;
#pragma unroll
    for (int j = 0; j < BIN_PER_THREAD; ++j) {
        const int64_t k = k0 + j;
        if (k < n) {
            float x, y, d;
            int r;
            load_geom<DT>(splats, (uint32_t)k, x, y, d, r);
            int a, b, c, e;
            sum += (u64)tile_rect(grid, x, y, r, a, b, c, e);
        }
    }
    u64 total;
    u64 off = partial[blockIdx.x] + block_excl_scan_u64(sum, s_warp, total);
    for (int j = 0; j < BIN_PER_THREAD; ++j) {
        const int64_t k = k0 + j;
        if (k >= n) break;
        float x, y, d;
        int r;
        load_geom<DT>(splats, (uint32_t)k, x, y, d, r);
        int x0, x1, y0, y1;
        if (tile_rect(grid, x, y, r, x0, x1, y0, y1) == 0) continue;
        const u64 dbits = (u64)__float_as_uint(d);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) {
                if ((int64_t)off < cap) {
                    keys[off] = ((u64)(ty * grid.TX + tx) << 32) | dbits;
                    vals[off] = (uint32_t)k;
                }
                ++off;
            }
    }
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t key_count(const int64_t* n_keys, int64_t cap) {
    const int64_t n = *n_keys;
    return n < cap ? n : cap;
}

__global__ void __launch_bounds__(256) k_sort_hist(const u64* __restrict__ keys, const int64_t* n_keys,
                                                   int64_t cap, int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t sh[8][RADIX];
    for (int i = threadIdx.x; i < 8 * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const int64_t N = key_count(n_keys, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const u64 k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct SortSmem {
    u64 keys[SORT_TILE];
    uint32_t vals[SORT_TILE];
    uint32_t whist[SORT_WARPS][RADIX];
    uint32_t dstart[RADIX];
    uint32_t gbase[RADIX];
    uint32_t gdigit[RADIX];
    uint32_t scan_tmp[SORT_WARPS];
    int tile;
};

// Exclusive scan of 256 values held by threads 0..255 (others pass 0).
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t* tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31 && wid < 8) tmp[wid] = x;
    __syncthreads();
    uint32_t before = 0;
    if (threadIdx.x < RADIX)
        for (int w = 0; w < wid; ++w) before += tmp[w];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_pass(const u64* __restrict__ src_k,
                                                            const uint32_t* __restrict__ src_v,
                                                            u64* __restrict__ dst_k, uint32_t* __restrict__ dst_v,
                                                            const int64_t* n_keys, int64_t cap,
                                                            const uint32_t* __restrict__ hist,
                                                            uint32_t* __restrict__ status,
                                                            uint32_t* __restrict__ ticket, int shift,
                                                            unsigned int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t N = key_count(n_keys, cap);
    const int ntiles = (int)((N + SORT_TILE - 1) / SORT_TILE);
    {
        const uint32_t h = tid < RADIX ? hist[tid] : 0u;
        const uint32_t ex = scan256(h, sm.scan_tmp);
        if (tid < RADIX) sm.gdigit[tid] = ex;
    }
    const uint32_t lt_mask = (1u << lane) - 1u;
    while (true) {
        if (tid == 0) sm.tile = (int)atomicAdd(ticket, 1u);
        for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&sm.whist[0][0])[i] = 0;
        __syncthreads();
        const int t = sm.tile;
        if (t >= ntiles) break;
        const int64_t base = (int64_t)t * SORT_TILE;
        const int cnt = (int)min((int64_t)SORT_TILE, N - base);
        u64 key[SORT_KPT];
        uint32_t val[SORT_KPT], rank[SORT_KPT], dig[SORT_KPT];
#pragma unroll
        for (int k = 0; k < SORT_KPT; ++k) {
            const int li = wid * (32 * SORT_KPT) + k * 32 + lane;
            const bool valid = li < cnt;
            key[k] = valid ? src_k[base + li] : 0ull;
            val[k] = valid ? src_v[base + li] : 0u;
            dig[k] = valid ? (uint32_t)((key[k] >> shift) & 0xff) : RADIX;
        }
#pragma unroll
        for (int k = 0; k < SORT_KPT; ++k) {
            const uint32_t d = dig[k];
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t prior = 0;
            if (d < RADIX) prior = sm.whist[wid][d];
            __syncwarp();
            if (d < RADIX && lane == __ffs(peers) - 1) sm.whist[wid][d] = prior + __popc(peers);
            __syncwarp();
            rank[k] = prior + __popc(peers & lt_mask);
        }
        __syncthreads();
        // per digit: exclusive offsets across warps, tile count, look-back
        uint32_t count = 0;
        if (tid < RADIX) {
            for (int w = 0; w < SORT_WARPS; ++w) {
                const uint32_t c = sm.whist[w][tid];
                sm.whist[w][tid] = count;
                count += c;
            }
            uint32_t* my = status + (size_t)t * RADIX + tid;
            if (t == 0) st_relaxed(my, FLAG_PREFIX | count);
            else st_relaxed(my, FLAG_AGG | count);
        }
        const uint32_t dstart = scan256(count, sm.scan_tmp);
        if (tid < RADIX) {
            sm.dstart[tid] = dstart;
            uint32_t excl = 0;
            if (t > 0) {
                for (int j = t - 1; j >= 0; --j) {
                    const uint32_t* ps = status + (size_t)j * RADIX + tid;
                    uint32_t v = ld_relaxed(ps);
                    int spins = 0;
                    while ((v >> 30) == 0u) {
                        if (++spins > SPIN_LIMIT) {
                            raise_status(err, GS_ERR_TIMEOUT);
                            v = FLAG_PREFIX;
                            break;
                        }
                        __nanosleep(32);
                        v = ld_relaxed(ps);
                    }
                    excl += v & COUNT_MASK;
                    if ((v & FLAG_PREFIX) != 0u) break;
                }
                st_relaxed(status + (size_t)t * RADIX + tid, FLAG_PREFIX | (excl + count));
            }
            sm.gbase[tid] = sm.gdigit[tid] + excl;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SORT_KPT; ++k) {
            const uint32_t d = dig[k];
            if (d < RADIX) {
                const uint32_t pos = sm.dstart[d] + sm.whist[wid][d] + rank[k];
                sm.keys[pos] = key[k];
                sm.vals[pos] = val[k];
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += SORT_THREADS) {
            const u64 k = sm.keys[i];
            const uint32_t d = (uint32_t)((k >> shift) & 0xff);
            const uint32_t dst = sm.gbase[d] + (uint32_t)i - sm.dstart[d];
            dst_k[dst] = k;
            dst_v[dst] = sm.vals[i];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_ranges(const u64* __restrict__ keys, const int64_t* n_keys,
                                                int64_t cap, uint32_t* __restrict__ ranges) {
    const int64_t N = key_count(n_keys, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)i;
        if (i == N - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
    }
}

// Heavy-first tile order: tiles grouped by floor(log2(length + 1)), longest
// group first (32 groups; order inside a group is whatever the atomics give,
// which only affects scheduling, never results).
__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t* __restrict__ ranges, int ntiles,
                                                     uint32_t* __restrict__ order) {
    __shared__ uint32_t cnt[33], cur[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        atomicAdd(&cnt[31 - (31 - __clz(len + 1u))], 1u);  // bucket 0 = longest
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < 33; ++b) { cur[b] = run; run += cnt[b]; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        const uint32_t pos = atomicAdd(&cur[31 - (31 - __clz(len + 1u))], 1u);
        order[pos] = (uint32_t)t;
    }
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
struct SortLayout {
    int passes;
    int64_t nchunk;
    int64_t max_tiles;
    size_t off_partial, off_altk, off_altv, off_zero, zero_bytes, off_hist, off_status, off_ticket, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static SortLayout sort_layout(int64_t n, int64_t cap, int ntiles_img) {
    SortLayout L;
    int tb = 0;
    while ((1ll << tb) < (long long)ntiles_img) ++tb;
    L.passes = (32 + tb + 7) / 8;
    L.nchunk = (n + BIN_CHUNK - 1) / BIN_CHUNK;
    L.max_tiles = (cap + SORT_TILE - 1) / SORT_TILE;
    size_t o = 0;
    L.off_partial = o; o = align256(o + sizeof(u64) * (size_t)(L.nchunk > 0 ? L.nchunk : 1));
    L.off_altk = o; o = align256(o + sizeof(u64) * (size_t)(cap > 0 ? cap : 1));
    L.off_altv = o; o = align256(o + sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
    L.off_zero = o;
    L.off_hist = o; o = align256(o + sizeof(uint32_t) * RADIX * (size_t)L.passes);
    L.off_ticket = o; o = align256(o + sizeof(uint32_t) * (size_t)L.passes);
    L.off_status = o; o = align256(o + sizeof(uint32_t) * RADIX * (size_t)L.passes * (size_t)(L.max_tiles > 0 ? L.max_tiles : 1));
    L.zero_bytes = o - L.off_zero;
    L.total = o;
    return L;
}

static int sort_blocks_per_sm() {
    static int bps = 0;  // same on every GB300 device
    if (bps == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sort_pass, SORT_THREADS, sizeof(SortSmem)) != cudaSuccess || b < 1)
            b = 1;
        bps = b;
    }
    return bps;
}

}  // namespace gs

using namespace gs;

static gs_status bin_common_checks(const gs_camera* cam, int rec_dtype, const void* splats, int64_t n,
                                   bool size_query) {
    if (!cam) return set_error(GS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1 || cam->width > (1 << 20) ||
        cam->height > (1 << 20))
        return set_error(GS_ERR_INVALID_ARG, "bad camera size or stride");
    if (rec_dtype != GS_F32 && rec_dtype != GS_BF16 && rec_dtype != GS_F16)
        return set_error(GS_ERR_INVALID_ARG, "bad record dtype %d", rec_dtype);
    if (n < 0 || n > (int64_t)0xFFFFFFF0LL) return set_error(GS_ERR_INVALID_ARG, "bad Gaussian count");
    if (!size_query && n > 0 && (!splats || ((uintptr_t)splats & 15)))
        return set_error(GS_ERR_INVALID_ARG, "splats NULL or not 16-byte aligned");
    return GS_OK;
}

static gs_status launch_count_scan(const gs_camera* cam, int rec_dtype, const void* splats, int64_t n,
                                   u64* partial, int64_t nchunk, int64_t* n_keys_out, int64_t cap,
                                   cudaStream_t st) {
    if (n == 0) {
        if (cudaMemsetAsync(n_keys_out, 0, sizeof(int64_t), st) != cudaSuccess)
            return set_error(GS_ERR_CUDA, "memset n_keys");
        return GS_OK;
    }
    const unsigned nb = (unsigned)nchunk;
    if (rec_dtype == GS_F32) k_bin_count<GS_F32><<<nb, BIN_THREADS, 0, st>>>(*cam, splats, n, partial);
    else if (rec_dtype == GS_BF16) k_bin_count<GS_BF16><<<nb, BIN_THREADS, 0, st>>>(*cam, splats, n, partial);
    else k_bin_count<GS_F16><<<nb, BIN_THREADS, 0, st>>>(*cam, splats, n, partial);
    gs_status s;
    if ((s = check_launch("k_bin_count")) != GS_OK) return s;
    unsigned int* err = status_ptr();
    if (!err) return set_error(GS_ERR_CUDA, "status word address");
    k_bin_scan<<<1, 1024, 0, st>>>(partial, (int)nchunk, n_keys_out, cap, err);
    return check_launch("k_bin_scan");
}

extern "C" gs_status gs_bin_count(const gs_camera* cam, int rec_dtype, const void* splats, int64_t n,
                                  void* workspace, size_t* workspace_bytes, int64_t* n_keys_out,
                                  gs_stream stream) {
    gs_status s;
    if ((s = bin_common_checks(cam, rec_dtype, splats, n, workspace == nullptr)) != GS_OK) return s;
    if (!workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    const int64_t nchunk = (n + BIN_CHUNK - 1) / BIN_CHUNK;
    const size_t need = align256(sizeof(u64) * (size_t)(nchunk > 0 ? nchunk : 1));
    if (!workspace) { *workspace_bytes = need; return GS_OK; }
    if (*workspace_bytes < need) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, need);
    if (!n_keys_out) return set_error(GS_ERR_INVALID_ARG, "n_keys_out is NULL");
    return launch_count_scan(cam, rec_dtype, splats, n, (u64*)workspace, nchunk, n_keys_out,
                             (int64_t)1 << 62, (cudaStream_t)stream);
}

extern "C" gs_status gs_bin_sort(const gs_camera* cam, int rec_dtype, const void* splats, int64_t n,
                                 int64_t keys_capacity, void* workspace, size_t* workspace_bytes,
                                 uint64_t* keys_out, uint32_t* vals_out, int64_t* n_keys_out,
                                 uint32_t* tile_ranges, uint32_t* tile_order, gs_stream stream) {
    gs_status s;
    if ((s = bin_common_checks(cam, rec_dtype, splats, n, workspace == nullptr)) != GS_OK) return s;
    if (!workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    if (keys_capacity < 0 || keys_capacity >= (int64_t)COUNT_MASK)
        return set_error(GS_ERR_INVALID_ARG, "keys_capacity must be in [0, 2^30)");
    const Grid grid = make_grid(*cam);
    const int ntiles = grid.TX * grid.TY;
    const SortLayout L = sort_layout(n, keys_capacity, ntiles);
    if (!workspace) { *workspace_bytes = L.total; return GS_OK; }
    if (*workspace_bytes < L.total) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, L.total);
    if (((uintptr_t)workspace & 255) != 0) return set_error(GS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (!n_keys_out || !tile_ranges || (keys_capacity > 0 && (!keys_out || !vals_out)))
        return set_error(GS_ERR_INVALID_ARG, "an output pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    if (cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)ntiles, st) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "memset ranges");
    u64* partial = (u64*)(ws + L.off_partial);
    if ((s = launch_count_scan(cam, rec_dtype, splats, n, partial, L.nchunk, n_keys_out, keys_capacity, st)) != GS_OK)
        return s;
    if (n == 0 || keys_capacity == 0) {
        if (tile_order) {
            k_tile_order<<<1, 1024, 0, st>>>(tile_ranges, ntiles, tile_order);
            return check_launch("k_tile_order");
        }
        return GS_OK;
    }
    if (cudaMemsetAsync(ws + L.off_zero, 0, L.zero_bytes, st) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "memset sort state");
    // ping-pong so that the last pass writes keys_out / vals_out
    u64* bufk[2] = {(u64*)keys_out, (u64*)(ws + L.off_altk)};
    uint32_t* bufv[2] = {vals_out, (uint32_t*)(ws + L.off_altv)};
    int cur = (L.passes % 2 == 0) ? 0 : 1;
    const unsigned nb = (unsigned)L.nchunk;
    if (rec_dtype == GS_F32)
        k_bin_dup<GS_F32><<<nb, BIN_THREADS, 0, st>>>(*cam, splats, n, partial, keys_capacity, bufk[cur], bufv[cur]);
    else if (rec_dtype == GS_BF16)
        k_bin_dup<GS_BF16><<<nb, BIN_THREADS, 0, st>>>(*cam, splats, n, partial, keys_capacity, bufk[cur], bufv[cur]);
    else
        k_bin_dup<GS_F16><<<nb, BIN_THREADS, 0, st>>>(*cam, splats, n, partial, keys_capacity, bufk[cur], bufv[cur]);
    if ((s = check_launch("k_bin_dup")) != GS_OK) return s;
    uint32_t* hist = (uint32_t*)(ws + L.off_hist);
    uint32_t* status = (uint32_t*)(ws + L.off_status);
    uint32_t* ticket = (uint32_t*)(ws + L.off_ticket);
    const int sms = num_sms();
    unsigned int* err = status_ptr();
    if (!err) return set_error(GS_ERR_CUDA, "status word address");
    {
        const int64_t want = (keys_capacity + 255) / 256;
        const unsigned hb = (unsigned)(want < 2 * sms ? (want > 0 ? want : 1) : 2 * sms);
        k_sort_hist<<<hb, 256, 0, st>>>(bufk[cur], n_keys_out, keys_capacity, L.passes, hist);
        if ((s = check_launch("k_sort_hist")) != GS_OK) return s;
    }
    {
        // once per device (not repeated while a graph is being captured)
        static bool attr_done[64] = {false};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !attr_done[dev]) {
            if (cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem)) !=
                cudaSuccess)
                return set_error(GS_ERR_CUDA, "cudaFuncSetAttribute(k_sort_pass)");
            if (dev >= 0 && dev < 64) attr_done[dev] = true;
        }
    }
    const int64_t want = L.max_tiles;
    const int64_t cap_blocks = (int64_t)sms * sort_blocks_per_sm();
    const unsigned sb = (unsigned)(want < cap_blocks ? want : cap_blocks);
    for (int p = 0; p < L.passes; ++p) {
        k_sort_pass<<<sb, SORT_THREADS, sizeof(SortSmem), st>>>(
            bufk[cur], bufv[cur], bufk[cur ^ 1], bufv[cur ^ 1], n_keys_out, keys_capacity, hist + p * RADIX,
            status + (size_t)p * RADIX * (size_t)L.max_tiles, ticket + p, 8 * p, err);
        if ((s = check_launch("k_sort_pass")) != GS_OK) return s;
        cur ^= 1;
    }
    {
        const int64_t want2 = (keys_capacity + 255) / 256;
        const unsigned rb = (unsigned)(want2 < 4 * sms ? (want2 > 0 ? want2 : 1) : 4 * sms);
        k_ranges<<<rb, 256, 0, st>>>(bufk[cur], n_keys_out, keys_capacity, tile_ranges);
        if ((s = check_launch("k_ranges")) != GS_OK) return s;
    }
    if (tile_order) {
        k_tile_order<<<1, 1024, 0, st>>>(tile_ranges, ntiles, tile_order);
        if ((s = check_launch("k_tile_order")) != GS_OK) return s;
    }
    return GS_OK;
}
