// Host-side plumbing of the C ABI: thread-local error messages, the device
// status word, defaults and version.
#include <stdarg.h>
#include <atomic>
#include <stdio.h>

#include "gs_internal.cuh"

namespace gs {

__device__ unsigned int g_status = 0u;

// Cached per device, so that no runtime query happens while a stream is
// being captured into a CUDA graph after the first call on a device.
unsigned int* status_ptr() {
    // threads that race on an entry store the same address
    static std::atomic<unsigned int*> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    unsigned int* q = cache[dev].load(std::memory_order_relaxed);
    if (!q) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
        q = (unsigned int*)p;
        cache[dev].store(q, std::memory_order_relaxed);
    }
    return q;
}

static thread_local char t_msg[512] = "";

gs_status set_error(gs_status code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_msg, sizeof(t_msg), fmt, ap);
    va_end(ap);
    return code;
}

gs_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return GS_OK;
}

int num_sms() {
    static int cache[64] = {0};
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    if (dev >= 0 && dev < 64) cache[dev] = sms;
    return sms;
}

}  // namespace gs

using namespace gs;

extern "C" void gs_default_config(gs_config* c) {
    if (!c) return;
    c->near_z = 0.2f;
    c->dilation = 0.3f;
    c->alpha_min = 1.0f / 255.0f;
    c->alpha_max = 0.99f;
    c->t_eps = 1e-4f;
    c->bg[0] = c->bg[1] = c->bg[2] = 0.f;
    c->lambda_score = 0.8f;
    c->prune_frac = 0.1f;
    c->prune_cap = 0.5f;
    c->change_thr = 0.05f;
    c->k0 = 5;
    c->k_max = 64;
    c->w_rgb = 1.0f;
    c->w_depth = 0.5f;
    c->balance = 1;
}

extern "C" const char* gs_version(void) { return "gs-gb300 0.1 (sm_103a)"; }

extern "C" const char* gs_last_error(void) { return t_msg; }

extern "C" gs_status gs_status_poll(gs_stream stream, int blocking, int* state) {
    cudaStream_t st = (cudaStream_t)stream;
    if (blocking) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "stream sync: %s", cudaGetErrorString(e));
        if (state) *state = GS_IDLE;
    } else if (state) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaErrorNotReady) *state = GS_EXECUTING;
        else if (e == cudaSuccess) *state = GS_IDLE;
        else return set_error(GS_ERR_CUDA, "stream query: %s", cudaGetErrorString(e));
    }
    unsigned int v = 0;
    const cudaError_t e = cudaMemcpyFromSymbol(&v, g_status, sizeof(v));
    if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "read status: %s", cudaGetErrorString(e));
    if (v != 0u) set_error((gs_status)v, "device status %u", v);
    return (gs_status)v;
}

extern "C" gs_status gs_status_reset(gs_stream stream) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return set_error(GS_ERR_CUDA, "status symbol");
    if (cudaMemsetAsync(p, 0, sizeof(unsigned int), (cudaStream_t)stream) != cudaSuccess)
        return set_error(GS_ERR_CUDA, "memset status");
    return GS_OK;
}
