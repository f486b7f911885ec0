// Mapping-iteration optimizer step on the device (the map update that the
// paper's Preprocessing Engines feed, Sec. 5.4): Adam over up to
// GS_ADAM_MAX_TENSORS parameter arrays in one launch.  The step count lives in
// device memory (state[0]) so that a CUDA graph replaying the step keeps the
// bias correction right; the last CTA to finish advances it (ticket in
// state[1], no spin).
#include "gs_internal.cuh"

namespace gs {

struct AdamArgs {
    float* p[GS_ADAM_MAX_TENSORS];
    const float* g[GS_ADAM_MAX_TENSORS];
    float* m[GS_ADAM_MAX_TENSORS];
    float* v[GS_ADAM_MAX_TENSORS];
    int64_t end[GS_ADAM_MAX_TENSORS];  // cumulative element counts
    int nt;
};

__global__ void __launch_bounds__(256) k_adam(AdamArgs a, int64_t total, float lr, float b1, float b2, float eps,
                                              float* __restrict__ state) {
    const float step = state[0] + 1.f;
    const float c1 = 1.f - powf(b1, step), c2 = 1.f - powf(b2, step);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int t = 0;
        while (t < a.nt - 1 && q >= a.end[t]) ++t;
        const int64_t i = q - (t > 0 ? a.end[t - 1] : 0);
        float p = a.p[t][i], m = a.m[t][i], v = a.v[t][i];
        adam_elem(p, m, v, a.g[t][i], lr, b1, b2, c1, c2, eps);
        a.p[t][i] = p;
        a.m[t][i] = m;
        a.v[t][i] = v;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int* ticket = reinterpret_cast<unsigned int*>(state + 1);
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        state[0] = step;
        *reinterpret_cast<unsigned int*>(state + 1) = 0u;
    }
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_adam(int n_tensors, float* const* params, const float* const* grads, float* const* m,
                             float* const* v, const int64_t* counts, float lr, float beta1, float beta2, float eps,
                             float* state, gs_stream stream) {
    if (n_tensors < 1 || n_tensors > GS_ADAM_MAX_TENSORS) return set_error(GS_ERR_INVALID_ARG, "1..%d tensors", GS_ADAM_MAX_TENSORS);
    if (!params || !grads || !m || !v || !counts || !state) return set_error(GS_ERR_INVALID_ARG, "NULL pointer");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return set_error(GS_ERR_INVALID_ARG, "bad Adam constants");
    AdamArgs a;
    int64_t total = 0;
    a.nt = n_tensors;
    for (int t = 0; t < GS_ADAM_MAX_TENSORS; ++t) {
        if (t < n_tensors) {
            if (counts[t] < 0 || (counts[t] > 0 && (!params[t] || !grads[t] || !m[t] || !v[t])))
                return set_error(GS_ERR_INVALID_ARG, "tensor %d", t);
            a.p[t] = params[t];
            a.g[t] = grads[t];
            a.m[t] = m[t];
            a.v[t] = v[t];
            total += counts[t];
        } else {
            a.p[t] = nullptr; a.g[t] = nullptr; a.m[t] = nullptr; a.v[t] = nullptr;
        }
        a.end[t] = total;
    }
    const int sms = num_sms();
    const int64_t want = (total + 255) / 256;
    const unsigned nb = (unsigned)(want < 8 * sms ? (want > 0 ? want : 1) : 8 * sms);
    k_adam<<<nb, 256, 0, (cudaStream_t)stream>>>(a, total, lr, beta1, beta2, eps, state);
    return check_launch("k_adam");
}
