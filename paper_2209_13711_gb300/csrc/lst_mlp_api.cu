// C ABI of the T5 scoring network: parameters, inference, gradient, Adam.
#include <cuda_runtime.h>

#include <cmath>
#include <new>

#include "../../include/lst.h"
#include "lst_mlp.cuh"

using namespace lst;

struct lst_mlp {
    int device = 0;
    int max_batch = 0;
    long step = 0;
    void* mem = nullptr;
    float* theta = nullptr;       // FP32 master parameters
    float* m = nullptr;           // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;        // one float
    float* scores = nullptr;      // [max_batch]
    __nv_bfloat16* w1_bf = nullptr;
    __nv_bfloat16* w2_bf = nullptr;
    __nv_bfloat16* w3_bf = nullptr;
    float* w2_r = nullptr;
    float* w3_r = nullptr;
    MlpSaved saved{};
    MlpDeltas deltas{};
};

namespace {

#define CKM(x)                                              \
    do {                                                    \
        if ((x) != cudaSuccess) return LST_ERR_CUDA;        \
    } while (0)

MlpParams params_of(const lst_mlp* m) {
    MlpParams P;
    P.w1_bf = m->w1_bf;
    P.w2_bf = m->w2_bf;
    P.w3_bf = m->w3_bf;
    P.w2_r = m->w2_r;
    P.w3_r = m->w3_r;
    P.b1 = m->theta + kOffB1;
    P.b2 = m->theta + kOffB2;
    P.b3 = m->theta + kOffB3;
    P.w4 = m->theta + kOffW4;
    P.b4 = m->theta + kOffB4;
    return P;
}

void derive(lst_mlp* m, cudaStream_t st) {
    MlpDerived D{m->w1_bf, m->w2_bf, m->w3_bf, m->w2_r, m->w3_r};
    k_mlp_derive<<<(kParams + 255) / 256, 256, 0, st>>>(m->theta, D);
}

int fwd_blocks(int n) {
    int warps = (n + 15) / 16;
    int b = (warps + 3) / 4;
    return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

// forward with saved activations, per-sample deltas, parameter gradient
lst_status gradient_pass(lst_mlp* m, const float* X, const float* y, int n, cudaStream_t st) {
    CKM(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
    k_mlp_forward<<<fwd_blocks(n), 128, 0, st>>>(params_of(m), X, n, nullptr, m->scores, m->saved);
    k_mlp_backward_samples<<<(n + 127) / 128 < 1 ? 1 : ((n + 127) / 128 > 1024 ? 1024 : (n + 127) / 128), 128, 0,
                             st>>>(params_of(m), y, n, m->scores, m->saved, m->deltas, m->loss);
    k_mlp_weight_grad<<<(kParams + 127) / 128, 128, 0, st>>>(X, n, m->saved, m->deltas, m->grad);
    return cudaGetLastError() == cudaSuccess ? LST_OK : LST_ERR_CUDA;
}

}  // namespace

// Used by the chain (lst_api.cu) to run the network on T5 candidates.
MlpParams lst_mlp_device_params(const lst_mlp* m) { return params_of(m); }

extern "C" {

lst_status lst_mlp_create(lst_mlp** out, int32_t device, int32_t max_batch) {
    if (!out || max_batch <= 0) return LST_ERR_ARG;
    *out = nullptr;
    lst_mlp* m = new (std::nothrow) lst_mlp();
    if (!m) return LST_ERR_OOM;
    m->device = device;
    m->max_batch = max_batch;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete m;
        return LST_ERR_CUDA;
    }
    const size_t B = max_batch;
    size_t bytes = 0;
    auto take = [&](size_t n) { size_t o = (bytes + 255) / 256 * 256; bytes = o + n; return o; };
    size_t o_theta = take(4 * kParams), o_m = take(4 * kParams), o_v = take(4 * kParams), o_g = take(4 * kParams);
    size_t o_loss = take(4), o_sc = take(4 * B);
    size_t o_w1 = take(2 * kH1 * kIn), o_w2 = take(2 * kH2 * kH1), o_w3 = take(2 * kH3 * kH2);
    size_t o_w2r = take(4 * kH2 * kH1), o_w3r = take(4 * kH3 * kH2);
    size_t o_x1 = take(4 * B * kH1), o_x2 = take(4 * B * kH2), o_h3 = take(4 * B * kH3), o_z4 = take(4 * B);
    size_t o_d1 = take(4 * B * kH1), o_d2 = take(4 * B * kH2), o_d3 = take(4 * B * kH3), o_d4 = take(4 * B);
    if (cudaMalloc(&m->mem, bytes) != cudaSuccess) {
        delete m;
        return LST_ERR_OOM;
    }
    char* b = static_cast<char*>(m->mem);
    m->theta = reinterpret_cast<float*>(b + o_theta);
    m->m = reinterpret_cast<float*>(b + o_m);
    m->v = reinterpret_cast<float*>(b + o_v);
    m->grad = reinterpret_cast<float*>(b + o_g);
    m->loss = reinterpret_cast<float*>(b + o_loss);
    m->scores = reinterpret_cast<float*>(b + o_sc);
    m->w1_bf = reinterpret_cast<__nv_bfloat16*>(b + o_w1);
    m->w2_bf = reinterpret_cast<__nv_bfloat16*>(b + o_w2);
    m->w3_bf = reinterpret_cast<__nv_bfloat16*>(b + o_w3);
    m->w2_r = reinterpret_cast<float*>(b + o_w2r);
    m->w3_r = reinterpret_cast<float*>(b + o_w3r);
    m->saved = MlpSaved{reinterpret_cast<float*>(b + o_x1), reinterpret_cast<float*>(b + o_x2),
                        reinterpret_cast<float*>(b + o_h3), reinterpret_cast<float*>(b + o_z4)};
    m->deltas = MlpDeltas{reinterpret_cast<float*>(b + o_d1), reinterpret_cast<float*>(b + o_d2),
                          reinterpret_cast<float*>(b + o_d3), reinterpret_cast<float*>(b + o_d4)};
    if (cudaMemset(m->mem, 0, bytes) != cudaSuccess) {
        cudaFree(m->mem);
        delete m;
        return LST_ERR_CUDA;
    }
    *out = m;
    return LST_OK;
}

void lst_mlp_destroy(lst_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    if (m->mem) cudaFree(m->mem);
    delete m;
}

lst_status lst_mlp_set_params(lst_mlp* m, const float* params) {
    if (!m || !params) return LST_ERR_ARG;
    CKM(cudaSetDevice(m->device));
    CKM(cudaMemcpy(m->theta, params, 4 * kParams, cudaMemcpyHostToDevice));
    CKM(cudaMemset(m->m, 0, 4 * kParams));
    CKM(cudaMemset(m->v, 0, 4 * kParams));
    m->step = 0;
    derive(m, nullptr);
    CKM(cudaDeviceSynchronize());
    return LST_OK;
}

lst_status lst_mlp_get_params(lst_mlp* m, float* params) {
    if (!m || !params) return LST_ERR_ARG;
    CKM(cudaSetDevice(m->device));
    CKM(cudaDeviceSynchronize());
    CKM(cudaMemcpy(params, m->theta, 4 * kParams, cudaMemcpyDeviceToHost));
    return LST_OK;
}

lst_status lst_mlp_get_state(lst_mlp* m, float* params, float* adam_m, float* adam_v, int64_t* step) {
    if (!m || !params || !adam_m || !adam_v || !step) return LST_ERR_ARG;
    CKM(cudaSetDevice(m->device));
    CKM(cudaDeviceSynchronize());
    CKM(cudaMemcpy(params, m->theta, 4 * kParams, cudaMemcpyDeviceToHost));
    CKM(cudaMemcpy(adam_m, m->m, 4 * kParams, cudaMemcpyDeviceToHost));
    CKM(cudaMemcpy(adam_v, m->v, 4 * kParams, cudaMemcpyDeviceToHost));
    *step = m->step;
    return LST_OK;
}

lst_status lst_mlp_set_state(lst_mlp* m, const float* params, const float* adam_m, const float* adam_v,
                             int64_t step) {
    if (!m || !params || !adam_m || !adam_v || step < 0) return LST_ERR_ARG;
    CKM(cudaSetDevice(m->device));
    CKM(cudaDeviceSynchronize());
    CKM(cudaMemcpy(m->theta, params, 4 * kParams, cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(m->m, adam_m, 4 * kParams, cudaMemcpyHostToDevice));
    CKM(cudaMemcpy(m->v, adam_v, 4 * kParams, cudaMemcpyHostToDevice));
    m->step = (long)step;
    derive(m, nullptr);
    CKM(cudaDeviceSynchronize());
    return LST_OK;
}

lst_status lst_mlp_forward(lst_mlp* m, const float* X, int32_t n, float* scores, void* stream) {
    if (!m || n < 0 || (n && (!X || !scores))) return LST_ERR_ARG;
    if (n == 0) return LST_OK;
    CKM(cudaSetDevice(m->device));
    k_mlp_forward<<<fwd_blocks(n), 128, 0, static_cast<cudaStream_t>(stream)>>>(params_of(m), X, n, nullptr, scores,
                                                                                 MlpSaved{});
    return cudaGetLastError() == cudaSuccess ? LST_OK : LST_ERR_CUDA;
}

lst_status lst_mlp_gradient(lst_mlp* m, const float* X, const float* y, int32_t n, float* grad, float* loss,
                            void* stream) {
    if (!m || !X || !y || n <= 0) return LST_ERR_ARG;
    if (n > m->max_batch) return LST_ERR_CAPACITY;
    CKM(cudaSetDevice(m->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    lst_status s = gradient_pass(m, X, y, n, st);
    if (s != LST_OK) return s;
    CKM(cudaStreamSynchronize(st));
    if (grad) CKM(cudaMemcpy(grad, m->grad, 4 * kParams, cudaMemcpyDeviceToHost));
    if (loss) {
        float l = 0.f;
        CKM(cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost));
        *loss = l / float(n);
    }
    return LST_OK;
}

lst_status lst_mlp_train_step(lst_mlp* m, const float* X, const float* y, int32_t n, float lr, float* loss,
                              void* stream) {
    if (!m || !X || !y || n <= 0 || !(lr > 0.f)) return LST_ERR_ARG;
    if (n > m->max_batch) return LST_ERR_CAPACITY;
    CKM(cudaSetDevice(m->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    lst_status s = gradient_pass(m, X, y, n, st);
    if (s != LST_OK) return s;
    ++m->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = float(1.0 / (1.0 - std::pow(0.9, double(m->step))));
    const float c2 = float(1.0 / (1.0 - std::pow(0.999, double(m->step))));
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(m->theta, m->m, m->v, m->grad, lr, b1, b2, 1e-8f, c1, c2);
    derive(m, st);
    CKM(cudaGetLastError());
    if (loss) {
        CKM(cudaStreamSynchronize(st));
        float l = 0.f;
        CKM(cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost));
        *loss = l / float(n);
    }
    return LST_OK;
}

}  // extern "C"
