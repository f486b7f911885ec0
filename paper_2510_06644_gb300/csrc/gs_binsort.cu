// A-2..A-4: tile intersection, key duplication, 64-bit key sort and tile
// ranges (Sec. 2.1, Step 1-2 and Step 2) on sm_103a.
//
// The key of a (tile, Gaussian) pair is tile_id << 32 | float32 bits of the
// depth, with the Gaussian id as the tie-break (equal depths keep id order).
// It is sorted as an MSD radix sort whose first digit is the whole tile id:
//   k_tile_hist     per-CTA tile counts of each Gaussian's rect, summed in
//                   shared memory and written as one row per CTA (grids of
//   k_col_scan      up to 8192 tiles); a column scan over the CTAs gives
//                   each CTA's offset inside every bucket and the tile
//                   totals.  Larger grids count with one global atomic per
//                   key (k_tile_count).
//   k_tile_scan     one CTA: exclusive scan of the tile counts -> bucket
//                   starts, tile ranges, key count, capacity check
//   k_tile_order    one CTA: heavy-first permutation of the tiles (stable)
//                   (with the per-CTA rows, the column scan's last CTA runs
//                   both: k_col_scan_tail)
//   k_tile_scatter  each pair takes a slot of its tile's bucket and writes
//                   the 64-bit remainder key depth_bits << 32 | id there (a
//                   CTA's slots start at its row offset and are dealt out
//                   with shared-memory atomics: no global atomics)
//   k_tile_sort     bucket sort, heavy first: the remainder keys are unique,
//                   so any correct sort of them gives the same result.
//                   One launch: buckets of up to 512 keys take one warp
//                   each, a merge sort with the keys in registers; up to
//                   4096 keys one CTA, each warp merge-sorting 256 (8 per
//                   lane) before the warps merge their runs, up to 8192 the
//                   same with 512 per warp; longer buckets sort
//                   8192-key runs in shared memory and merge them by rank
//                   in global memory.  The sort writes tile_id << 32 |
//                   depth_bits and the id.
// The scatter order inside a bucket depends on atomics, the output does not.
// Everything stays on the device: the key count is never read by the host.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

#define BIN_THREADS 256
#define TS_THREADS 512
#define TS_SMEM_KEYS 8192
#define SW_MAX 512               // buckets up to this length sort with one warp

typedef unsigned long long u64;

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_count(gs_camera cam, float alpha_min, const void* __restrict__ splats,
                                                            int64_t n, uint32_t* __restrict__ count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Grid grid = make_grid(cam);
    const Geom G = load_geom<DT>(splats, (uint32_t)k);
    int x0, x1, y0, y1;
    if (tile_rect(grid, G, alpha_min, x0, x1, y0, y1) == 0) return;
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) atomicAdd(count + ty * grid.TX + tx, 1u);
}

// Shared-memory aggregated forms of the two passes above, for grids of at
// most AGG_MAX_TILES tiles.  CTA c takes `per_cta` consecutive Gaussians:
//   k_tile_hist      counts its pairs per tile in shared memory and writes
//                    the row hist[c][0..T) (no global atomics);
//   k_col_scan       exclusive prefix of hist[.][t] over the CTAs (in place)
//                    and the tile totals;
//   k_tile_scatter_rows  CTA c starts tile t's slots at start[t] +
//                    hist[c][t] and deals them out with shared-memory atomics.
#define AGG_MAX_TILES 8192

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_hist(gs_camera cam, float alpha_min, const void* __restrict__ splats, int64_t n,
                                                           int64_t per_cta, int ntiles, uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t h[];
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const Grid grid = make_grid(cam);
    const int64_t k0 = (int64_t)blockIdx.x * per_cta, k1 = min(n, k0 + per_cta);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const Geom G = load_geom<DT>(splats, (uint32_t)k);
        int x0, x1, y0, y1;
        if (tile_rect(grid, G, alpha_min, x0, x1, y0, y1) == 0) continue;
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) atomicAdd(h + ty * grid.TX + tx, 1u);
    }
    __syncthreads();
    uint32_t* row = hist + (size_t)blockIdx.x * ntiles;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) row[t] = h[t];
}

// Column scan of the per-CTA rows: CTA b takes 32 tiles; its 32 warps split
// the rows into 32 consecutive ranges, sum them, scan the 32 partial sums in
// shared memory and write each row's exclusive prefix in place.
__device__ __forceinline__ void col_scan_body(uint32_t* __restrict__ hist, int nrows, int ntiles,
                                              uint32_t* __restrict__ total, int blk) {
    // CTA: CS_TILES tiles x (1024 / CS_TILES) row groups of consecutive rows
    constexpr int CS_TILES = 8, CS_GROUPS = 1024 / CS_TILES;
    __shared__ uint32_t part[CS_GROUPS][CS_TILES + 1];
    const int tx = threadIdx.x % CS_TILES, ty = threadIdx.x / CS_TILES;
    const int t = blk * CS_TILES + tx;
    const int per = (nrows + CS_GROUPS - 1) / CS_GROUPS;
    const int r0 = min(nrows, ty * per), r1 = min(nrows, r0 + per);
    // rows in groups of 8 loads issued back to back (a dependent sum per
    // load would wait out an L2 round trip per row); the first group stays
    // in registers for the prefix pass (the only group when a thread has at
    // most 8 rows: up to 1024 rows)
    uint32_t sum = 0, v0[8];
    if (t < ntiles)
        for (int r = r0; r < r1; r += 8) {
            uint32_t v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = r + k < r1 ? __ldcg(hist + (size_t)(r + k) * ntiles + t) : 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k) sum += v[k];
            if (r == r0) {
#pragma unroll
                for (int k = 0; k < 8; ++k) v0[k] = v[k];
            }
        }
    part[ty][tx] = sum;
    __syncthreads();
    // warp w < CS_TILES scans column w's CS_GROUPS partial sums (4 per lane)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < CS_TILES) {
        uint32_t v[CS_GROUPS / 32];
        uint32_t loc = 0;
#pragma unroll
        for (int k = 0; k < CS_GROUPS / 32; ++k) {
            v[k] = part[lane * (CS_GROUPS / 32) + k][w];
            loc += v[k];
        }
        uint32_t incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - loc;
#pragma unroll
        for (int k = 0; k < CS_GROUPS / 32; ++k) {
            part[lane * (CS_GROUPS / 32) + k][w] = run;
            run += v[k];
        }
        const int tc = blk * CS_TILES + w;
        if (lane == 31 && tc < ntiles) total[tc] = incl;
    }
    __syncthreads();
    uint32_t run = part[ty][tx];
    if (t < ntiles)
        for (int r = r0; r < r1; r += 8) {
            uint32_t v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                v[k] = r == r0 ? v0[k] : (r + k < r1 ? __ldcg(hist + (size_t)(r + k) * ntiles + t) : 0u);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (r + k < r1) {
                    hist[(size_t)(r + k) * ntiles + t] = run;
                    run += v[k];
                }
        }
}

__global__ void __launch_bounds__(1024) k_col_scan(uint32_t* __restrict__ hist, int nrows, int ntiles,
                                                   uint32_t* __restrict__ total) {
    col_scan_body(hist, nrows, ntiles, total, (int)blockIdx.x);
}

// Heavy-first tile order (defined below with the tile scan).
__device__ __forceinline__ void tile_order_body(const uint32_t* __restrict__ ranges, int ntiles,
                                                uint32_t* __restrict__ order, uint32_t* __restrict__ n_big);

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_scatter_rows(gs_camera cam, float alpha_min, const void* __restrict__ splats,
                                                                   int64_t n, int64_t per_cta, int ntiles,
                                                                   const uint32_t* __restrict__ start,
                                                                   const uint32_t* __restrict__ hist, int64_t cap,
                                                                   u64* __restrict__ keys,
                                                                   const uint32_t* __restrict__ ranges,
                                                                   uint32_t* __restrict__ order,
                                                                   uint32_t* __restrict__ n_big) {
    if (blockIdx.x == gridDim.x - 1) {  // the heavy-first order, beside the scatter
        tile_order_body(ranges, ntiles, order, n_big);
        return;
    }
    extern __shared__ uint32_t h[];
    uint32_t* base = h + ntiles;
    const uint32_t* row = hist + (size_t)blockIdx.x * ntiles;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        h[t] = 0;
        base[t] = start[t] + row[t];
    }
    __syncthreads();
    const Grid grid = make_grid(cam);
    const int64_t k0 = (int64_t)blockIdx.x * per_cta, k1 = min(n, k0 + per_cta);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const Geom G = load_geom<DT>(splats, (uint32_t)k);
        int x0, x1, y0, y1;
        if (tile_rect(grid, G, alpha_min, x0, x1, y0, y1) == 0) continue;
        const u64 rem = ((u64)__float_as_uint(G.depth) << 32) | (u64)(uint32_t)k;
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) {
                const int t = ty * grid.TX + tx;
                const u64 pos = (u64)base[t] + atomicAdd(h + t, 1u);
                if ((int64_t)pos < cap) keys[pos] = rem;
            }
    }
}

// Exclusive scan of the tile counts.  start[t] = min(bucket start, cap);
// ranges (if not NULL) = bucket clipped to the capacity; *n_keys = total.
__device__ __forceinline__ void tile_scan_body(const uint32_t* __restrict__ count, int ntiles, int64_t cap,
                                               uint32_t* __restrict__ start, uint32_t* __restrict__ ranges,
                                               int64_t* __restrict__ n_keys, unsigned int* __restrict__ status) {
    __shared__ u64 s_warp[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u64 carry = 0;
    // each chunk's counts are loaded while the previous chunk is scanned
    u64 v_nx = (int)threadIdx.x < ntiles ? (u64)__ldcg(count + threadIdx.x) : 0ull;
    for (int base = 0; base < ntiles; base += 1024) {
        const int t = base + threadIdx.x;
        const u64 v = v_nx;
        v_nx = t + 1024 < ntiles ? (u64)__ldcg(count + t + 1024) : 0ull;
        u64 x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        if (wid == 0) {
            u64 w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u64 y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const u64 excl = carry + (wid > 0 ? s_warp[wid - 1] : 0ull) + x - v;
        const u64 total = s_warp[31];
        if (t < ntiles) {
            const u64 b = excl < (u64)cap ? excl : (u64)cap;
            const u64 e = excl + v < (u64)cap ? excl + v : (u64)cap;
            if (start) start[t] = (uint32_t)b;
            if (ranges) {
                ranges[2 * t] = e > b ? (uint32_t)b : 0u;
                ranges[2 * t + 1] = e > b ? (uint32_t)e : 0u;
            }
        }
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *n_keys = (int64_t)carry;
        if ((int64_t)carry > cap) raise_status(status, GS_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(1024) k_tile_scan(const uint32_t* __restrict__ count, int ntiles, int64_t cap,
                                                    uint32_t* __restrict__ start, uint32_t* __restrict__ ranges,
                                                    int64_t* __restrict__ n_keys, unsigned int* __restrict__ status) {
    tile_scan_body(count, ntiles, cap, start, ranges, n_keys, status);
}

// Heavy-first tile order: tiles grouped by quarter octaves of their length
// -- x = length - 1 in [2^m + q 2^(m-2), 2^m + (q + 1) 2^(m-2)), q = 0..3
// (lengths 1 and 0 last) -- longest group first, ascending tile index inside
// a group: a stable counting sort, so the order is a function of the lists
// alone (the compositing kernels may treat the first tiles of the order
// differently, and their results must not depend on scheduling).  Finer than
// whole octaves, it launches the compositing CTAs closer to longest first
// (tracking step 231.6 -> 226.4 us against octaves).  n_big receives the
// number of tiles longer than SW_MAX keys, which are exactly the first n_big
// of the order (SW_MAX + 1 starts a group).
#define OG_N 133  // order groups: quarter octaves of the length, then length 1, then empty
__device__ __forceinline__ int order_group(uint32_t len) {
    if (len == 0) return OG_N - 1;
    const uint32_t x = len - 1u;
    if (x == 0) return OG_N - 2;
    const int msb = 31 - __clz(x);
    const int sub = msb >= 2 ? (int)((x >> (msb - 2)) & 3u) : (int)((x << (2 - msb)) & 3u);
    return (31 - msb) * 4 + (3 - sub);
}

__device__ __forceinline__ void tile_order_body(const uint32_t* __restrict__ ranges, int ntiles,
                                                uint32_t* __restrict__ order, uint32_t* __restrict__ n_big) {
    __shared__ uint32_t cnt[OG_N], cur[OG_N];
    __shared__ uint32_t wcnt[32][OG_N];  // per warp and group, within a 1024-tile chunk
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = threadIdx.x; b < OG_N; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        atomicAdd(&cnt[order_group(__ldcg(ranges + 2 * t + 1) - __ldcg(ranges + 2 * t))], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < OG_N; ++b) {
            if (b == order_group(SW_MAX + 1)) *n_big = run + cnt[b];
            cur[b] = run;
            run += cnt[b];
        }
    }
    const int nw = (int)(blockDim.x >> 5);
    for (int base = 0; base < ntiles; base += (int)blockDim.x) {
        for (int q = threadIdx.x; q < 32 * OG_N; q += blockDim.x) (&wcnt[0][0])[q] = 0;
        __syncthreads();
        const int t = base + (int)threadIdx.x;
        const int grp = t < ntiles ? order_group(__ldcg(ranges + 2 * t + 1) - __ldcg(ranges + 2 * t)) : OG_N;
        const unsigned same = __match_any_sync(0xffffffffu, grp);
        const unsigned rank = __popc(same & ((1u << lane) - 1u));
        if (grp < OG_N && rank == 0) wcnt[warp][grp] = __popc(same);
        __syncthreads();
        for (int b = threadIdx.x; b < OG_N; b += blockDim.x) {  // exclusive scan over the warps, per group
            uint32_t run = cur[b];
            for (int w = 0; w < nw; ++w) {
                const uint32_t v = wcnt[w][b];
                wcnt[w][b] = run;
                run += v;
            }
            cur[b] = run;
        }
        __syncthreads();
        if (grp < OG_N) order[wcnt[warp][grp] + rank] = (uint32_t)t;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t* __restrict__ ranges, int ntiles,
                                                     uint32_t* __restrict__ order, uint32_t* __restrict__ n_big) {
    tile_order_body(ranges, ntiles, order, n_big);
}

// The column scan followed, in the CTA that finishes last (ticket; every
// other CTA's totals are published before its ticket), by the tile scan and
// the heavy-first order: one launch instead of three.
struct ScanTail {
    unsigned int* ticket;  // zero on entry, zero again on exit
    int64_t cap;
    uint32_t* start;
    uint32_t* ranges;
    int64_t* n_keys;
    unsigned int* status;
    uint32_t* order;
    uint32_t* n_big;
};

__device__ __forceinline__ void col_scan_tail_body(uint32_t* __restrict__ hist, int nrows, int ntiles,
                                                   uint32_t* __restrict__ total, const ScanTail& T, int blk,
                                                   int nblk) {
    __shared__ bool s_last;
    col_scan_body(hist, nrows, ntiles, total, blk);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(T.ticket, 1u) == (unsigned)nblk - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    tile_scan_body(total, ntiles, T.cap, T.start, T.ranges, T.n_keys, T.status);
    __syncthreads();
    if (T.order) tile_order_body(T.ranges, ntiles, T.order, T.n_big);  // else the scatter's extra CTA
    if (threadIdx.x == 0) *T.ticket = 0u;
}

__global__ void __launch_bounds__(1024) k_col_scan_tail(uint32_t* __restrict__ hist, int nrows, int ntiles,
                                                        uint32_t* __restrict__ total, ScanTail T) {
    col_scan_tail_body(hist, nrows, ntiles, total, T, (int)blockIdx.x, (int)gridDim.x);
}

// k_tile_scatter_rows with the rects the fused projection kept (no
// geometry re-read, no tile-rect arithmetic): only the depth is loaded.
template <int DT>
__device__ __forceinline__ void scatter_rects_body(int TX, const void* __restrict__ splats, int64_t n,
                                                   int64_t per_cta, int ntiles, const uint32_t* __restrict__ start,
                                                   const uint32_t* __restrict__ hist,
                                                   const uint2* __restrict__ rects, int64_t cap,
                                                   u64* __restrict__ keys, const uint32_t* __restrict__ ranges,
                                                   uint32_t* __restrict__ order, uint32_t* __restrict__ n_big,
                                                   int blk, int nblk) {
    if (blk == nblk - 1) {  // the heavy-first order, beside the scatter
        tile_order_body(ranges, ntiles, order, n_big);
        return;
    }
    extern __shared__ uint32_t h[];
    uint32_t* base = h + ntiles;
    const uint32_t* row = hist + (size_t)blk * ntiles;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        h[t] = 0;
        base[t] = start[t] + row[t];
    }
    __syncthreads();
    const int64_t k0 = (int64_t)blk * per_cta, k1 = min(n, k0 + per_cta);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const uint2 r = __ldg(rects + k);
        const int x0 = (int)(r.x & 0xffffu), x1 = (int)(r.x >> 16), y0 = (int)(r.y & 0xffffu), y1 = (int)(r.y >> 16);
        if (x1 <= x0) continue;
        const float depth = DT == GS_F32 ? __ldg(reinterpret_cast<const float*>(splats) + 12 * (size_t)k + 6)
                                         : __ldg(reinterpret_cast<const float*>(splats) + 8 * (size_t)k + 2);
        const u64 rem = ((u64)__float_as_uint(depth) << 32) | (u64)(uint32_t)k;
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) {
                const int t = ty * TX + tx;
                const u64 pos = (u64)base[t] + atomicAdd(h + t, 1u);
                if ((int64_t)pos < cap) keys[pos] = rem;
            }
    }
}

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_scatter_rects(int TX, const void* __restrict__ splats, int64_t n,
                                                                    int64_t per_cta, int ntiles,
                                                                    const uint32_t* __restrict__ start,
                                                                    const uint32_t* __restrict__ hist,
                                                                    const uint2* __restrict__ rects, int64_t cap,
                                                                    u64* __restrict__ keys,
                                                                    const uint32_t* __restrict__ ranges,
                                                                    uint32_t* __restrict__ order,
                                                                    uint32_t* __restrict__ n_big) {
    scatter_rects_body<DT>(TX, splats, n, per_cta, ntiles, start, hist, rects, cap, keys, ranges, order, n_big,
                           (int)blockIdx.x, (int)gridDim.x);
}

template <int DT>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_scatter(gs_camera cam, float alpha_min, const void* __restrict__ splats,
                                                              int64_t n, const uint32_t* __restrict__ start,
                                                              uint32_t* __restrict__ fill, int64_t cap,
                                                              u64* __restrict__ keys) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Grid grid = make_grid(cam);
    const Geom G = load_geom<DT>(splats, (uint32_t)k);
    int x0, x1, y0, y1;
    if (tile_rect(grid, G, alpha_min, x0, x1, y0, y1) == 0) return;
    const u64 rem = ((u64)__float_as_uint(G.depth) << 32) | (u64)(uint32_t)k;
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) {
            const int t = ty * grid.TX + tx;
            const u64 pos = (u64)start[t] + atomicAdd(fill + t, 1u);
            if ((int64_t)pos < cap) keys[pos] = rem;
        }
}

// Bitonic sort of m (power of two) keys in shared memory, ascending.
__device__ __forceinline__ void bitonic_smem(u64* s, int m) {
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < (m >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (j - 1));
                const int hi = lo + j;
                const u64 a = s[lo], b = s[hi];
                const bool asc = (lo & k) == 0;
                if ((a > b) == asc) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Number of keys in sorted run r[0, len) that are < x (lower bound).
__device__ __forceinline__ int rank_in(const u64* r, int len, u64 x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(r + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Merge sort of a bucket with the keys in registers.  Thread t of the
// sorting group holds positions [t KPT, (t+1) KPT) (blocked layout).  Each
// thread first sorts its KPT keys with a register network; then rounds of
// merges double the sorted run length: each thread finds where its KPT
// outputs start in the pair of runs (merge path: a binary search on the
// diagonal) and merges KPT keys serially.  Runs go through shared memory,
// padded by one key per 16 so that the blocked accesses spread over the
// banks.  Padding keys are ~0 (above every real key: depth bits < 2^31).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad16(int x) { return x + (x >> 4); }

template <int KPT>
__device__ __forceinline__ void sort_regs(u64 (&v)[KPT]) {
#pragma unroll
    for (int k = 2; k <= KPT; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < KPT; ++i) {
                const int p = i ^ j;
                if (p > i) {
                    const u64 lo = v[i] < v[p] ? v[i] : v[p], hi = v[i] < v[p] ? v[p] : v[i];
                    const bool asc = (i & k) == 0;
                    v[i] = asc ? lo : hi;
                    v[p] = asc ? hi : lo;
                }
            }
}

__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Merge rounds from sorted runs of `run` keys up to one run of nthr * KPT
// keys.  t: the thread's index in the group; buf: the group's buffer
// (pad16 of nthr * KPT keys); the group synchronises with __syncwarp when
// it is one warp, else with named barrier 1 over nthr threads.
template <int KPT>
__device__ __forceinline__ void merge_rounds(u64 (&v)[KPT], u64* buf, int t, int nthr, int run) {
    const int M = nthr * KPT;
    for (; run < M; run <<= 1) {
#pragma unroll
        for (int k = 0; k < KPT; ++k) buf[pad16(t * KPT + k)] = v[k];
        if (nthr == 32) __syncwarp(); else named_bar(1, nthr);
        const int pair0 = (t * KPT) & ~(2 * run - 1);
        const int diag = t * KPT - pair0;
        const int a0 = pair0, b0 = pair0 + run;
        int lo = max(0, diag - run), hi = min(diag, run);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (buf[pad16(a0 + mid)] < buf[pad16(b0 + diag - 1 - mid)]) lo = mid + 1;
            else hi = mid;
        }
        int i = lo, j = diag - lo;
        u64 x = i < run ? buf[pad16(a0 + i)] : ~0ull;
        u64 y = j < run ? buf[pad16(b0 + j)] : ~0ull;
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const bool ta = x < y;
            v[k] = ta ? x : y;
            if (ta) {
                ++i;
                x = i < run ? buf[pad16(a0 + i)] : ~0ull;
            } else {
                ++j;
                y = j < run ? buf[pad16(b0 + j)] : ~0ull;
            }
        }
        if (nthr == 32) __syncwarp(); else named_bar(1, nthr);
    }
}

// Loads a bucket of n <= nthr * KPT keys into the blocked layout (coalesced
// through buf), padding with ~0.
template <int KPT>
__device__ __forceinline__ void load_blocked(const u64* key, int n, u64 (&v)[KPT], u64* buf, int t, int nthr) {
    // all KPT global loads are issued before the first shared store
#pragma unroll
    for (int r = 0; r < KPT; ++r) v[r] = t + r * nthr < n ? __ldcg(key + t + r * nthr) : ~0ull;
#pragma unroll
    for (int r = 0; r < KPT; ++r) buf[pad16(t + r * nthr)] = v[r];
    if (nthr == 32) __syncwarp(); else named_bar(1, nthr);
#pragma unroll
    for (int k = 0; k < KPT; ++k) v[k] = buf[pad16(t * KPT + k)];
    if (nthr == 32) __syncwarp(); else named_bar(1, nthr);
}

// Writes the sorted bucket (coalesced through buf): tile_id << 32 |
// depth_bits and the id.
template <int KPT>
__device__ __forceinline__ void store_sorted(u64* key, uint32_t* val, int n, u64 hi, const u64 (&v)[KPT], u64* buf,
                                             int t, int nthr) {
#pragma unroll
    for (int k = 0; k < KPT; ++k) buf[pad16(t * KPT + k)] = v[k];
    if (nthr == 32) __syncwarp(); else named_bar(1, nthr);
    for (int x = t; x < n; x += nthr) {
        const u64 w = buf[pad16(x)];
        key[x] = hi | (w >> 32);
        val[x] = (uint32_t)w;
    }
}

template <int KPT>
__device__ __forceinline__ void warp_sort_bucket(u64* key, uint32_t* val, int n, u64 hi, u64* buf) {
    const int lane = threadIdx.x & 31;
    u64 v[KPT];
    load_blocked<KPT>(key, n, v, buf, lane, 32);
    sort_regs<KPT>(v);
    merge_rounds<KPT>(v, buf, lane, 32, KPT);
    store_sorted<KPT>(key, val, n, hi, v, buf, lane, 32);
}


// One launch for all buckets.  CTAs below n_big take the long buckets
// (first in the order), one each; every later CTA takes 16 short buckets,
// one per warp (both kinds run at once).
__device__ __forceinline__ void tile_sort_body(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ order,
                                               const uint32_t* __restrict__ n_big_p, int ntiles,
                                               u64* __restrict__ keys, uint32_t* __restrict__ vals,
                                               u64* __restrict__ tmp, int blk) {
    extern __shared__ __align__(16) u64 s[];
    const int n_big = (int)*n_big_p;
    if (blk >= n_big) {
        const int warp = threadIdx.x >> 5;
        const int idx = n_big + (blk - n_big) * (TS_THREADS / 32) + warp;
        if (idx >= ntiles) return;
        const int t = (int)order[idx];
        const uint32_t b = ranges[2 * t], e = ranges[2 * t + 1];
        const int n = (int)(e - b);
        if (n <= 0 || n > SW_MAX) return;
        const u64 hi = (u64)(uint32_t)t << 32;
        u64* buf = s + pad16(warp * SW_MAX);
        if (n <= 32) warp_sort_bucket<1>(keys + b, vals + b, n, hi, buf);
        else if (n <= 64) warp_sort_bucket<2>(keys + b, vals + b, n, hi, buf);
        else if (n <= 128) warp_sort_bucket<4>(keys + b, vals + b, n, hi, buf);
        else if (n <= 256) warp_sort_bucket<8>(keys + b, vals + b, n, hi, buf);
        else warp_sort_bucket<16>(keys + b, vals + b, n, hi, buf);
        return;
    }
    const int t = (int)order[blk];
    const uint32_t b = ranges[2 * t], e = ranges[2 * t + 1];
    const int n = (int)(e - b);
    u64* key = keys + b;
    if (n <= 4096) {
        // m / 256 warps, 8 keys per thread in registers: each warp sorts a
        // run of 256, then the group merges the runs (half the serial merge
        // steps per round of 16 keys per thread)
        int m = 1024;
        while (m < n) m <<= 1;
        const int W = m / 256;
        if ((int)(threadIdx.x >> 5) >= W) return;
        u64 v[8];
        load_blocked<8>(key, n, v, s, (int)threadIdx.x, W * 32);
        sort_regs<8>(v);
        merge_rounds<8>(v, s + pad16((threadIdx.x >> 5) * 256), (int)(threadIdx.x & 31), 32, 8);
        merge_rounds<8>(v, s, (int)threadIdx.x, W * 32, 256);
        store_sorted<8>(key, vals + b, n, (u64)(uint32_t)t << 32, v, s, (int)threadIdx.x, W * 32);
        return;
    }
    if (n <= TS_SMEM_KEYS) {
        // m / 512 warps, 16 keys per thread in registers: each warp sorts a
        // run of 512, then the group merges the runs
        int m = 2 * SW_MAX;
        while (m < n) m <<= 1;
        const int W = m / SW_MAX;
        if ((int)(threadIdx.x >> 5) >= W) return;
        u64 v[16];
        load_blocked<16>(key, n, v, s, (int)threadIdx.x, W * 32);
        sort_regs<16>(v);
        merge_rounds<16>(v, s + pad16((threadIdx.x >> 5) * SW_MAX), (int)(threadIdx.x & 31), 32, 16);
        merge_rounds<16>(v, s, (int)threadIdx.x, W * 32, SW_MAX);
        store_sorted<16>(key, vals + b, n, (u64)(uint32_t)t << 32, v, s, (int)threadIdx.x, W * 32);
        return;
    }
    // long bucket: sorted runs of TS_SMEM_KEYS, then merge by rank
    for (int c = 0; c < n; c += TS_SMEM_KEYS) {
        const int len = min(TS_SMEM_KEYS, n - c);
        for (int i = threadIdx.x; i < TS_SMEM_KEYS; i += blockDim.x) s[i] = i < len ? key[c + i] : ~0ull;
        __syncthreads();
        bitonic_smem(s, TS_SMEM_KEYS);
        for (int i = threadIdx.x; i < len; i += blockDim.x) key[c + i] = s[i];
        __syncthreads();
    }
    __threadfence_block();
    u64* src = key;
    u64* dst = tmp + b;
    for (int run = TS_SMEM_KEYS; run < n; run <<= 1) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int pair = i & ~(2 * run - 1);  // run: a power of two
            const int a0 = pair, a1 = min(pair + run, n), b1 = min(pair + 2 * run, n);
            const u64 x = __ldcg(src + i);
            int out;
            if (i < a1) out = pair + (i - a0) + rank_in(src + a1, b1 - a1, x);
            else out = pair + (i - a1) + rank_in(src + a0, a1 - a0, x);
            dst[out] = x;
        }
        __threadfence_block();
        __syncthreads();
        u64* w = src;
        src = dst;
        dst = w;
    }
    const u64 hi = (u64)(uint32_t)t << 32;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const u64 v = __ldcg(src + i);
        vals[b + i] = (uint32_t)v;
        if (src != key) key[i] = hi | (v >> 32);
    }
    __syncthreads();
    if (src == key)
        for (int i = threadIdx.x; i < n; i += blockDim.x) key[i] = hi | (key[i] >> 32);
}

__global__ void __launch_bounds__(TS_THREADS) k_tile_sort(const uint32_t* __restrict__ ranges,
                                                          const uint32_t* __restrict__ order,
                                                          const uint32_t* __restrict__ n_big_p, int ntiles,
                                                          u64* __restrict__ keys, uint32_t* __restrict__ vals,
                                                          u64* __restrict__ tmp) {
    tile_sort_body(ranges, order, n_big_p, ntiles, keys, vals, tmp, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------
// Multi-session waves: column scan (+ tile scan and order), scatter and sort
// over every job of a wave (gs_track_wave)
// ---------------------------------------------------------------------------
struct WaveScanJob {
    uint32_t* hist;
    int nrows, ntiles;
    uint32_t* total;
    ScanTail tail;
};

__global__ void __launch_bounds__(1024) k_wave_col_scan_tail(const __grid_constant__ Wave<WaveScanJob> W) {
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveScanJob& J = W.job[j];
    col_scan_tail_body(J.hist, J.nrows, J.ntiles, J.total, J.tail, (int)blockIdx.x - W.start[j],
                       W.start[j + 1] - W.start[j]);
}

struct WaveScatterJob {
    int TX;
    const void* splats;
    int64_t n, per;
    int ntiles;
    const uint32_t* start;
    const uint32_t* hist;
    const uint2* rects;
    int64_t cap;
    u64* keys;
    const uint32_t* ranges;
    uint32_t* order;
    uint32_t* n_big;
};

__global__ void __launch_bounds__(BIN_THREADS) k_wave_scatter_rects(const __grid_constant__ Wave<WaveScatterJob> W) {
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveScatterJob& J = W.job[j];
    scatter_rects_body<GS_F32>(J.TX, J.splats, J.n, J.per, J.ntiles, J.start, J.hist, J.rects, J.cap, J.keys,
                               J.ranges, J.order, J.n_big, (int)blockIdx.x - W.start[j],
                               W.start[j + 1] - W.start[j]);
}

struct WaveSortJob {
    const uint32_t* ranges;
    const uint32_t* order;
    const uint32_t* n_big;
    int ntiles;
    u64* keys;
    uint32_t* vals;
    u64* tmp;
};

__global__ void __launch_bounds__(TS_THREADS) k_wave_tile_sort(const __grid_constant__ Wave<WaveSortJob> W) {
    const int j = wave_find(W.start, W.n, (int)blockIdx.x);
    const WaveSortJob& J = W.job[j];
    tile_sort_body(J.ranges, J.order, J.n_big, J.ntiles, J.keys, J.vals, J.tmp, (int)blockIdx.x - W.start[j]);
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
struct BinLayout {
    size_t off_count, off_fill, off_ticket, off_start, off_order, off_nbig, off_hist, off_tmp, zero_bytes, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Gaussians per CTA of the aggregated passes: two per thread (half the
// rows of one per thread for the column scan, and 782 -> 391 CTAs fit one
// wave: projection + binning + sort 63.6-64.6 -> 61.6-62.5 us on the
// tracking frame; four per thread 72.8-74.8), or more when the per-CTA rows
// would pass 2^24 entries (64 MB).
static int64_t agg_per_cta(int64_t n, int ntiles) {
    const int64_t lim = (int64_t)1 << 24;
    const int64_t want = (n * (int64_t)ntiles + lim - 1) / lim;
    return want > 2 * BIN_THREADS ? want : 2 * BIN_THREADS;
}

static BinLayout bin_layout(int64_t n, int64_t cap, int ntiles) {
    BinLayout L;
    size_t o = 0;
    const int64_t per = agg_per_cta(n, ntiles);
    const int64_t rows = n > 0 ? (n + per - 1) / per : 1;
    L.off_count = o; o = align256(o + sizeof(uint32_t) * (size_t)ntiles);
    L.off_fill = o; o = align256(o + sizeof(uint32_t) * (size_t)ntiles);
    L.off_ticket = o; o = align256(o + sizeof(unsigned int));
    L.zero_bytes = o;
    L.off_start = o; o = align256(o + sizeof(uint32_t) * (size_t)ntiles);
    L.off_order = o; o = align256(o + sizeof(uint32_t) * (size_t)ntiles);
    L.off_nbig = o; o = align256(o + sizeof(uint32_t));
    L.off_hist = o;
    if (ntiles <= AGG_MAX_TILES) o = align256(o + sizeof(uint32_t) * (size_t)ntiles * (size_t)rows);
    L.off_tmp = o; o = align256(o + sizeof(u64) * (size_t)(cap > 0 ? cap : 1));
    L.total = o;
    return L;
}

}  // namespace gs

using namespace gs;

static gs_status bin_common_checks(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats,
                                   int64_t n, bool size_query) {
    if (!cfg) return set_error(GS_ERR_INVALID_ARG, "config is NULL");
    if (!cam) return set_error(GS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->sx < 1 || cam->sy < 1 || cam->width > (1 << 20) ||
        cam->height > (1 << 20))
        return set_error(GS_ERR_INVALID_ARG, "bad camera size or stride");
    if (rec_dtype != GS_F32 && rec_dtype != GS_BF16 && rec_dtype != GS_F16)
        return set_error(GS_ERR_INVALID_ARG, "bad record dtype %d", rec_dtype);
    if (n < 0 || n > (int64_t)0xFFFFFFF0LL) return set_error(GS_ERR_INVALID_ARG, "bad Gaussian count");
    if (!size_query && n > 0 && (!splats || ((uintptr_t)splats & 15)))
        return set_error(GS_ERR_INVALID_ARG, "splats NULL or not 16-byte aligned");
    const Grid g = make_grid(*cam);
    if ((int64_t)g.TX * g.TY > (1 << 26)) return set_error(GS_ERR_INVALID_ARG, "too many tiles");
    return GS_OK;
}

static gs_status set_agg_smem_attrs() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && done[dev]) return GS_OK;
    const int bytes = (int)(2 * AGG_MAX_TILES * sizeof(uint32_t));
    bool ok = cudaFuncSetAttribute(k_tile_scatter_rows<GS_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
              cudaFuncSetAttribute(k_tile_scatter_rows<GS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
              cudaFuncSetAttribute(k_tile_scatter_rows<GS_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
              cudaFuncSetAttribute(k_tile_scatter_rects<GS_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
              cudaFuncSetAttribute(k_tile_scatter_rects<GS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
              cudaFuncSetAttribute(k_tile_scatter_rects<GS_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    if (!ok) return set_error(GS_ERR_CUDA, "cudaFuncSetAttribute(k_tile_scatter_rows)");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return GS_OK;
}

// The bucket sort of the scattered keys, heavy tiles first.
static gs_status launch_tile_sort(int ntiles, const uint32_t* tile_ranges, const uint32_t* order,
                                  const uint32_t* n_big, uint64_t* keys_out, uint32_t* vals_out, u64* tmp,
                                  cudaStream_t st) {
    // once per device (not repeated while a graph is being captured)
    static bool attr_done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        if (cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((TS_SMEM_KEYS + TS_SMEM_KEYS / 16) * sizeof(u64))) != cudaSuccess)
            return set_error(GS_ERR_CUDA, "cudaFuncSetAttribute(k_tile_sort)");
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    k_tile_sort<<<(unsigned)ntiles, TS_THREADS, (TS_SMEM_KEYS + TS_SMEM_KEYS / 16) * sizeof(u64), st>>>(
        tile_ranges, order, n_big, ntiles, (u64*)keys_out, vals_out, tmp);
    return check_launch("k_tile_sort");
}

// Tile counts into `count`: per-CTA rows + column scan (rows kept in `hist`
// for the scatter) when the grid is small enough, else direct atomics.
static gs_status launch_count(const gs_camera* cam, float alpha_min, int rec_dtype, const void* splats, int64_t n,
                              uint32_t* count, uint32_t* hist, cudaStream_t st, const ScanTail* tail = nullptr,
                              bool* fused = nullptr) {
    if (fused) *fused = false;
    if (n == 0) return GS_OK;
    const Grid g = make_grid(*cam);
    const int ntiles = g.TX * g.TY;
    if (ntiles <= AGG_MAX_TILES && hist) {
        const int64_t per = agg_per_cta(n, ntiles);
        const unsigned nb = (unsigned)((n + per - 1) / per);
        const size_t sm = sizeof(uint32_t) * (size_t)ntiles;
        if (rec_dtype == GS_F32) k_tile_hist<GS_F32><<<nb, BIN_THREADS, sm, st>>>(*cam, alpha_min, splats, n, per, ntiles, hist);
        else if (rec_dtype == GS_BF16) k_tile_hist<GS_BF16><<<nb, BIN_THREADS, sm, st>>>(*cam, alpha_min, splats, n, per, ntiles, hist);
        else k_tile_hist<GS_F16><<<nb, BIN_THREADS, sm, st>>>(*cam, alpha_min, splats, n, per, ntiles, hist);
        gs_status s;
        if ((s = check_launch("k_tile_hist")) != GS_OK) return s;
        if (tail) {
            k_col_scan_tail<<<(unsigned)((ntiles + 7) / 8), 1024, 0, st>>>(hist, (int)nb, ntiles, count, *tail);
            if (fused) *fused = true;
            return check_launch("k_col_scan_tail");
        }
        k_col_scan<<<(unsigned)((ntiles + 7) / 8), 1024, 0, st>>>(hist, (int)nb, ntiles, count);
        return check_launch("k_col_scan");
    }
    const unsigned nb = (unsigned)((n + BIN_THREADS - 1) / BIN_THREADS);
    if (rec_dtype == GS_F32) k_tile_count<GS_F32><<<nb, BIN_THREADS, 0, st>>>(*cam, alpha_min, splats, n, count);
    else if (rec_dtype == GS_BF16) k_tile_count<GS_BF16><<<nb, BIN_THREADS, 0, st>>>(*cam, alpha_min, splats, n, count);
    else k_tile_count<GS_F16><<<nb, BIN_THREADS, 0, st>>>(*cam, alpha_min, splats, n, count);
    return check_launch("k_tile_count");
}

extern "C" gs_status gs_bin_count(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats,
                                  int64_t n,
                                  void* workspace, size_t* workspace_bytes, int64_t* n_keys_out,
                                  gs_stream stream) {
    gs_status s;
    if ((s = bin_common_checks(cfg, cam, rec_dtype, splats, n, workspace == nullptr)) != GS_OK) return s;
    if (!workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    const Grid g = make_grid(*cam);
    const int ntiles = g.TX * g.TY;
    const BinLayout L = bin_layout(n, 0, ntiles);
    const size_t need = L.off_tmp;
    if (!workspace) { *workspace_bytes = need; return GS_OK; }
    if (*workspace_bytes < need) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, need);
    if (!n_keys_out) return set_error(GS_ERR_INVALID_ARG, "n_keys_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* count = (uint32_t*)((char*)workspace + L.off_count);
    uint32_t* hist = ntiles <= AGG_MAX_TILES ? (uint32_t*)((char*)workspace + L.off_hist) : nullptr;
    if (cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)ntiles, st) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "memset counts");
    if ((s = launch_count(cam, cfg->alpha_min, rec_dtype, splats, n, count, hist, st)) != GS_OK) return s;
    unsigned int* err = status_ptr();
    if (!err) return set_error(GS_ERR_CUDA, "status word address");
    k_tile_scan<<<1, 1024, 0, st>>>(count, ntiles, (int64_t)1 << 62, nullptr, nullptr, n_keys_out, err);
    return check_launch("k_tile_scan");
}

extern "C" gs_status gs_bin_sort(const gs_config* cfg, const gs_camera* cam, int rec_dtype, const void* splats,
                                 int64_t n,
                                 int64_t keys_capacity, void* workspace, size_t* workspace_bytes,
                                 uint64_t* keys_out, uint32_t* vals_out, int64_t* n_keys_out,
                                 uint32_t* tile_ranges, uint32_t* tile_order, gs_stream stream) {
    gs_status s;
    if ((s = bin_common_checks(cfg, cam, rec_dtype, splats, n, workspace == nullptr)) != GS_OK) return s;
    if (!workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    if (keys_capacity < 0 || keys_capacity >= ((int64_t)1 << 30))
        return set_error(GS_ERR_INVALID_ARG, "keys_capacity must be in [0, 2^30)");
    const Grid grid = make_grid(*cam);
    const int ntiles = grid.TX * grid.TY;
    const BinLayout L = bin_layout(n, keys_capacity, ntiles);
    if (!workspace) { *workspace_bytes = L.total; return GS_OK; }
    if (*workspace_bytes < L.total) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, L.total);
    if (((uintptr_t)workspace & 255) != 0) return set_error(GS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (!n_keys_out || !tile_ranges || (keys_capacity > 0 && (!keys_out || !vals_out)))
        return set_error(GS_ERR_INVALID_ARG, "an output pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    uint32_t* count = (uint32_t*)(ws + L.off_count);
    uint32_t* fill = (uint32_t*)(ws + L.off_fill);
    uint32_t* start = (uint32_t*)(ws + L.off_start);
    u64* tmp = (u64*)(ws + L.off_tmp);
    uint32_t* hist = ntiles <= AGG_MAX_TILES ? (uint32_t*)(ws + L.off_hist) : nullptr;
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset bin state");
    unsigned int* err = status_ptr();
    if (!err) return set_error(GS_ERR_CUDA, "status word address");
    // the heavy-first order drives the sort; it is returned when asked for
    uint32_t* order = tile_order ? tile_order : (uint32_t*)(ws + L.off_order);
    uint32_t* n_big = (uint32_t*)(ws + L.off_nbig);
    // with per-CTA rows and keys to scatter, the scatter's extra CTA computes
    // the order; otherwise the column scan's last CTA does
    const bool order_beside = ntiles <= AGG_MAX_TILES && n > 0 && keys_capacity > 0;
    const ScanTail tail = {(unsigned int*)(ws + L.off_ticket), keys_capacity, start, tile_ranges, n_keys_out, err,
                           order_beside ? nullptr : order, n_big};
    bool fused = false;
    if ((s = launch_count(cam, cfg->alpha_min, rec_dtype, splats, n, count, hist, st, &tail, &fused)) != GS_OK) return s;
    if (!fused) {
        k_tile_scan<<<1, 1024, 0, st>>>(count, ntiles, keys_capacity, start, tile_ranges, n_keys_out, err);
        if ((s = check_launch("k_tile_scan")) != GS_OK) return s;
        k_tile_order<<<1, 1024, 0, st>>>(tile_ranges, ntiles, order, n_big);
        if ((s = check_launch("k_tile_order")) != GS_OK) return s;
    }
    if (n == 0 || keys_capacity == 0) return GS_OK;
    const float alpha_min = cfg->alpha_min;
    if (ntiles <= AGG_MAX_TILES) {
        if ((s = set_agg_smem_attrs()) != GS_OK) return s;
        const int64_t per = agg_per_cta(n, ntiles);
        const unsigned nb = (unsigned)((n + per - 1) / per);
        const size_t sm = 2 * sizeof(uint32_t) * (size_t)ntiles;
        if (rec_dtype == GS_F32)
            k_tile_scatter_rows<GS_F32><<<nb + 1, BIN_THREADS, sm, st>>>(*cam, alpha_min, splats, n, per, ntiles, start,
                                                                        hist, keys_capacity, (u64*)keys_out,
                                                                        tile_ranges, order, n_big);
        else if (rec_dtype == GS_BF16)
            k_tile_scatter_rows<GS_BF16><<<nb + 1, BIN_THREADS, sm, st>>>(*cam, alpha_min, splats, n, per, ntiles, start,
                                                                         hist, keys_capacity, (u64*)keys_out,
                                                                         tile_ranges, order, n_big);
        else
            k_tile_scatter_rows<GS_F16><<<nb + 1, BIN_THREADS, sm, st>>>(*cam, alpha_min, splats, n, per, ntiles, start,
                                                                        hist, keys_capacity, (u64*)keys_out,
                                                                        tile_ranges, order, n_big);
        if ((s = check_launch("k_tile_scatter_rows")) != GS_OK) return s;
    } else {
        const unsigned nb = (unsigned)((n + BIN_THREADS - 1) / BIN_THREADS);
        if (rec_dtype == GS_F32)
            k_tile_scatter<GS_F32><<<nb, BIN_THREADS, 0, st>>>(*cam, alpha_min, splats, n, start, fill, keys_capacity, (u64*)keys_out);
        else if (rec_dtype == GS_BF16)
            k_tile_scatter<GS_BF16><<<nb, BIN_THREADS, 0, st>>>(*cam, alpha_min, splats, n, start, fill, keys_capacity, (u64*)keys_out);
        else
            k_tile_scatter<GS_F16><<<nb, BIN_THREADS, 0, st>>>(*cam, alpha_min, splats, n, start, fill, keys_capacity, (u64*)keys_out);
        if ((s = check_launch("k_tile_scatter")) != GS_OK) return s;
    }
    return launch_tile_sort(ntiles, tile_ranges, order, n_big, keys_out, vals_out, tmp, st);
}

// Projection and binning in one call: gs_project, then gs_bin_sort with
// the first binning pass (per-CTA tile rows) done by the projection kernel
// itself and the scatter reading the rects it kept.  Same outputs as the two
// calls.  Workspace: gs_bin_sort's plus 8 bytes per Gaussian.
extern "C" gs_status gs_project_bin_sort(const gs_config* cfg, const gs_camera* cam, const gs_gaussians* g,
                                         int rec_dtype, void* splats, int64_t keys_capacity, void* workspace,
                                         size_t* workspace_bytes, uint64_t* keys_out, uint32_t* vals_out,
                                         int64_t* n_keys_out, uint32_t* tile_ranges, uint32_t* tile_order,
                                         gs_stream stream) {
    gs_status s;
    if ((s = project_checks(cfg, cam, g, rec_dtype)) != GS_OK) return s;
    const int64_t n = g->n;
    if ((s = bin_common_checks(cfg, cam, rec_dtype, splats, n, workspace == nullptr)) != GS_OK) return s;
    if (!workspace_bytes) return set_error(GS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    if (keys_capacity < 0 || keys_capacity >= ((int64_t)1 << 30))
        return set_error(GS_ERR_INVALID_ARG, "keys_capacity must be in [0, 2^30)");
    const Grid grid = make_grid(*cam);
    const int ntiles = grid.TX * grid.TY;
    const BinLayout L = bin_layout(n, keys_capacity, ntiles);
    const size_t off_rects = L.total, total = align256(L.total + sizeof(uint2) * (size_t)(n > 0 ? n : 1));
    if (!workspace) { *workspace_bytes = total; return GS_OK; }
    if (*workspace_bytes < total) return set_error(GS_ERR_WORKSPACE, "workspace %zu < %zu", *workspace_bytes, total);
    if (((uintptr_t)workspace & 255) != 0) return set_error(GS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (!n_keys_out || !tile_ranges || (keys_capacity > 0 && (!keys_out || !vals_out)))
        return set_error(GS_ERR_INVALID_ARG, "an output pointer is NULL");
    if (ntiles > AGG_MAX_TILES || n == 0) {  // no per-CTA rows: the two calls
        if ((s = gs_project(cfg, cam, g, rec_dtype, splats, stream)) != GS_OK) return s;
        size_t wb = *workspace_bytes;
        return gs_bin_sort(cfg, cam, rec_dtype, splats, n, keys_capacity, workspace, &wb, keys_out, vals_out,
                           n_keys_out, tile_ranges, tile_order, stream);
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    uint32_t* count = (uint32_t*)(ws + L.off_count);
    uint32_t* start = (uint32_t*)(ws + L.off_start);
    u64* tmp = (u64*)(ws + L.off_tmp);
    uint32_t* hist = (uint32_t*)(ws + L.off_hist);
    void* rects = ws + off_rects;
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, st) != cudaSuccess) return set_error(GS_ERR_CUDA, "memset bin state");
    unsigned int* err = status_ptr();
    if (!err) return set_error(GS_ERR_CUDA, "status word address");
    uint32_t* order = tile_order ? tile_order : (uint32_t*)(ws + L.off_order);
    uint32_t* n_big = (uint32_t*)(ws + L.off_nbig);
    // the order is computed beside the scatter unless there is none
    const ScanTail tail = {(unsigned int*)(ws + L.off_ticket), keys_capacity, start, tile_ranges, n_keys_out, err,
                           keys_capacity == 0 ? order : nullptr, n_big};
    const int64_t per = agg_per_cta(n, ntiles);
    const unsigned nb = (unsigned)((n + per - 1) / per);
    if ((s = launch_project_hist(cfg, cam, g, rec_dtype, splats, per, nb, ntiles, hist, rects, st)) != GS_OK) return s;
    k_col_scan_tail<<<(unsigned)((ntiles + 7) / 8), 1024, 0, st>>>(hist, (int)nb, ntiles, count, tail);
    if ((s = check_launch("k_col_scan_tail")) != GS_OK) return s;
    if (keys_capacity == 0) return GS_OK;
    if ((s = set_agg_smem_attrs()) != GS_OK) return s;
    const size_t sm = 2 * sizeof(uint32_t) * (size_t)ntiles;
    const uint2* r = (const uint2*)rects;
    if (rec_dtype == GS_F32)
        k_tile_scatter_rects<GS_F32><<<nb + 1, BIN_THREADS, sm, st>>>(grid.TX, splats, n, per, ntiles, start, hist, r,
                                                                     keys_capacity, (u64*)keys_out, tile_ranges,
                                                                     order, n_big);
    else if (rec_dtype == GS_BF16)
        k_tile_scatter_rects<GS_BF16><<<nb + 1, BIN_THREADS, sm, st>>>(grid.TX, splats, n, per, ntiles, start, hist, r,
                                                                      keys_capacity, (u64*)keys_out, tile_ranges,
                                                                      order, n_big);
    else
        k_tile_scatter_rects<GS_F16><<<nb + 1, BIN_THREADS, sm, st>>>(grid.TX, splats, n, per, ntiles, start, hist, r,
                                                                     keys_capacity, (u64*)keys_out, tile_ranges,
                                                                     order, n_big);
    if ((s = check_launch("k_tile_scatter_rects")) != GS_OK) return s;
    return launch_tile_sort(ntiles, tile_ranges, order, n_big, keys_out, vals_out, tmp, st);
}

// ---------------------------------------------------------------------------
// Wave launchers (gs_track_wave)
// ---------------------------------------------------------------------------
namespace gs {

// The job's binning state inside its gs_project_bin_sort workspace (the same
// layout as the single-session call), after checking the workspace size.
gs_status wave_bin_layout(const gs_track_job& j, WaveBin* out) {
    const Grid grid = make_grid(j.cam);
    const int ntiles = grid.TX * grid.TY;
    const int64_t n = j.g.n;
    if (ntiles > AGG_MAX_TILES) return set_error(GS_ERR_INVALID_ARG, "more than %d tiles", AGG_MAX_TILES);
    const BinLayout L = bin_layout(n, j.keys_capacity, ntiles);
    const size_t total = align256(L.total + sizeof(uint2) * (size_t)n);
    if (!j.bin_workspace || j.bin_workspace_bytes < total)
        return set_error(GS_ERR_WORKSPACE, "bin workspace %zu < %zu bytes", j.bin_workspace_bytes, total);
    if (((uintptr_t)j.bin_workspace & 255) != 0) return set_error(GS_ERR_INVALID_ARG, "bin workspace not 256-byte aligned");
    char* ws = (char*)j.bin_workspace;
    out->per = agg_per_cta(n, ntiles);
    out->nb = (unsigned)((n + out->per - 1) / out->per);
    out->ntiles = ntiles;
    out->count = (uint32_t*)(ws + L.off_count);
    out->start = (uint32_t*)(ws + L.off_start);
    out->hist = (uint32_t*)(ws + L.off_hist);
    out->ticket = (unsigned int*)(ws + L.off_ticket);
    out->n_big = (uint32_t*)(ws + L.off_nbig);
    out->tmp = ws + L.off_tmp;
    out->rects = ws + L.total;
    return GS_OK;
}

gs_status wave_bin_sort(const gs_track_job* jobs, const WaveBin* bins, int n, cudaStream_t st) {
    unsigned int* err = status_ptr();
    if (!err) return set_error(GS_ERR_CUDA, "status word address");
    gs_status s;
    {
        Wave<WaveScanJob> W;
        W.n = n;
        int blocks = 0;
        for (int j = 0; j < n; ++j) {
            const gs_track_job& t = jobs[j];
            const WaveBin& b = bins[j];
            W.start[j] = blocks;
            blocks += (b.ntiles + 7) / 8;
            const ScanTail tail = {b.ticket, t.keys_capacity, b.start, t.tile_ranges, t.n_keys, err, nullptr, b.n_big};
            W.job[j] = WaveScanJob{b.hist, (int)b.nb, b.ntiles, b.count, tail};
        }
        W.start[n] = blocks;
        k_wave_col_scan_tail<<<(unsigned)blocks, 1024, 0, st>>>(W);
        if ((s = check_launch("k_wave_col_scan_tail")) != GS_OK) return s;
    }
    {
        static bool attr_done[64] = {false};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !attr_done[dev]) {
            if (cudaFuncSetAttribute(k_wave_scatter_rects, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * AGG_MAX_TILES * sizeof(uint32_t))) != cudaSuccess)
                return set_error(GS_ERR_CUDA, "cudaFuncSetAttribute(k_wave_scatter_rects)");
            if (dev >= 0 && dev < 64) attr_done[dev] = true;
        }
        Wave<WaveScatterJob> W;
        W.n = n;
        int blocks = 0, smax = 1;
        for (int j = 0; j < n; ++j) {
            const gs_track_job& t = jobs[j];
            const WaveBin& b = bins[j];
            W.start[j] = blocks;
            blocks += (int)b.nb + 1;  // + the CTA that computes the heavy-first order
            smax = std::max(smax, b.ntiles);
            W.job[j] = WaveScatterJob{make_grid(t.cam).TX, t.splats, t.g.n, b.per, b.ntiles, b.start, b.hist,
                                      (const uint2*)b.rects, t.keys_capacity, (u64*)t.keys, t.tile_ranges,
                                      t.tile_order, b.n_big};
        }
        W.start[n] = blocks;
        k_wave_scatter_rects<<<(unsigned)blocks, BIN_THREADS, 2 * sizeof(uint32_t) * (size_t)smax, st>>>(W);
        if ((s = check_launch("k_wave_scatter_rects")) != GS_OK) return s;
    }
    {
        static bool attr_done[64] = {false};
        int dev = 0;
        cudaGetDevice(&dev);
        const int sm = (int)((TS_SMEM_KEYS + TS_SMEM_KEYS / 16) * sizeof(u64));
        if (dev < 0 || dev >= 64 || !attr_done[dev]) {
            if (cudaFuncSetAttribute(k_wave_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
                return set_error(GS_ERR_CUDA, "cudaFuncSetAttribute(k_wave_tile_sort)");
            if (dev >= 0 && dev < 64) attr_done[dev] = true;
        }
        Wave<WaveSortJob> W;
        W.n = n;
        int blocks = 0;
        for (int j = 0; j < n; ++j) {
            const gs_track_job& t = jobs[j];
            const WaveBin& b = bins[j];
            W.start[j] = blocks;
            blocks += b.ntiles;
            W.job[j] = WaveSortJob{t.tile_ranges, t.tile_order, b.n_big, b.ntiles, (u64*)t.keys, t.vals, (u64*)b.tmp};
        }
        W.start[n] = blocks;
        k_wave_tile_sort<<<(unsigned)blocks, TS_THREADS, (size_t)sm, st>>>(W);
        if ((s = check_launch("k_wave_tile_sort")) != GS_OK) return s;
    }
    return GS_OK;
}

}  // namespace gs
