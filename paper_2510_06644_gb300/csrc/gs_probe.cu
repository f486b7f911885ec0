// Measurement probes (not steps of the method).
//
// Throughput probe of global float32 reductions (red.global.add.f32), the
// operation that merges per-(Gaussian, tile) gradients into the per-Gaussian
// arrays in the backward (Sec. 2.2 Step 4).  The probe gives the measured
// denominator of the backward's atomic-throughput fraction: thread t of
// `n_threads` adds 1.0 to dst[t % n_dst] `per_thread` times, so n_dst >=
// n_threads measures distinct addresses (each warp's 32 lanes on one 128-byte
// line) and a small n_dst measures contended ones.
#include "gs_internal.cuh"

namespace gs {

__global__ void __launch_bounds__(256) k_probe_red_f32(float* __restrict__ dst, int64_t n_dst, int64_t n_threads,
                                                     int per_thread) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_threads) return;
    float* p = dst + t % n_dst;
#pragma unroll 4
    for (int k = 0; k < per_thread; ++k)
        asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(1.0f) : "memory");
}

// FP32 FMA throughput, the denominator of the compositing kernels' ALU
// fraction: each thread runs 8 independent chains a <- a m + c for `iters`
// steps (16 FLOP per step) and writes the sum of its chains.  With m = c = 1
// and chain k starting at k, every thread writes 28 + 8 iters exactly (for
// iters < 2^21), which is what the test checks.
__global__ void __launch_bounds__(256) k_probe_fma_f32(float* __restrict__ out, int64_t n_threads, int iters,
                                                     float m, float c) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_threads) return;
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)k;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[t] = s;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_probe_red_f32(float* dst, int64_t n_dst, int64_t n_threads, int32_t per_thread,
                                      gs_stream stream) {
    if (!dst) return set_error(GS_ERR_INVALID_ARG, "dst is NULL");
    if (n_dst < 1 || n_threads < 1 || per_thread < 1)
        return set_error(GS_ERR_INVALID_ARG, "n_dst, n_threads and per_thread must be positive");
    if (n_threads > (int64_t)0x7fffffff * 256) return set_error(GS_ERR_INVALID_ARG, "n_threads too large");
    const unsigned nb = (unsigned)((n_threads + 255) / 256);
    k_probe_red_f32<<<nb, 256, 0, (cudaStream_t)stream>>>(dst, n_dst, n_threads, per_thread);
    return check_launch("k_probe_red_f32");
}

extern "C" gs_status gs_probe_fma_f32(float* out, int64_t n_threads, int32_t iters, gs_stream stream) {
    if (!out) return set_error(GS_ERR_INVALID_ARG, "out is NULL");
    if (n_threads < 1 || iters < 1) return set_error(GS_ERR_INVALID_ARG, "n_threads and iters must be positive");
    if (n_threads > (int64_t)0x7fffffff * 256) return set_error(GS_ERR_INVALID_ARG, "n_threads too large");
    const unsigned nb = (unsigned)((n_threads + 255) / 256);
    k_probe_fma_f32<<<nb, 256, 0, (cudaStream_t)stream>>>(out, n_threads, iters, 1.0f, 1.0f);
    return check_launch("k_probe_fma_f32");
}
