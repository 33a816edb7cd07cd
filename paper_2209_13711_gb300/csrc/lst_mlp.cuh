// Shapes, parameter layout and kernel declarations of the T5 scoring network.
#pragma once

#include <cuda_bf16.h>

#include "lst_pdl.cuh"

namespace lst {

constexpr int kFeatures = 38;        // defined features; the input is zero padded to kIn
constexpr int kIn = 48, kH1 = 64, kH2 = 64, kH3 = 32;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH1 * kIn;
constexpr int kOffW2 = kOffB1 + kH1;
constexpr int kOffB2 = kOffW2 + kH2 * kH1;
constexpr int kOffW3 = kOffB2 + kH2;
constexpr int kOffB3 = kOffW3 + kH3 * kH2;
constexpr int kOffW4 = kOffB3 + kH3;
constexpr int kOffB4 = kOffW4 + kH3;
constexpr int kParams = kOffB4 + 1;  // 9409

struct MlpParams {
    const __nv_bfloat16* w1_bf;      // [64][48]
    const __nv_bfloat16* w2_bf;      // [64][64]
    const __nv_bfloat16* w3_bf;      // [32][64]
    const float* w2_r;               // BF16-rounded W2 as FP32 (backward)
    const float* w3_r;
    const float* b1;
    const float* b2;
    const float* b3;
    const float* w4;
    const float* b4;
};

struct MlpSaved {
    float* x1;                       // [n][64] BF16-rounded layer-2 inputs
    float* x2;                       // [n][64]
    float* h3;                       // [n][32]
    float* z4;                       // [n]
};

struct MlpDeltas {
    float* dz1;
    float* dz2;
    float* dz3;
    float* dz4;
};

struct MlpDerived {                  // writable views of the derived copies
    __nv_bfloat16* w1_bf;
    __nv_bfloat16* w2_bf;
    __nv_bfloat16* w3_bf;
    float* w2_r;
    float* w3_r;
};

__global__ void k_mlp_forward(MlpParams P, const float* X, int n, const int* n_dev, float* scores, MlpSaved save);
__global__ void k_mlp_backward_samples(MlpParams P, const float* y, int n, const float* scores, MlpSaved sv,
                                       MlpDeltas D, float* loss_sum);
__global__ void k_mlp_weight_grad(const float* X, int n, MlpSaved sv, MlpDeltas D, float* grad);
__global__ void k_mlp_adam(float* theta, float* m, float* v, const float* grad, float lr, float b1, float b2,
                           float eps, float c1, float c2);
__global__ void k_mlp_derive(const float* theta, MlpDerived P);

}  // namespace lst
