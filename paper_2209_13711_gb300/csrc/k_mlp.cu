// T5 scoring network: BF16 tensor-core inference and FP32 training kernels.
//
// Network: 48 inputs (38 features zero padded) -> 64 -> 64 -> 32 -> 1, ReLU
// on hidden layers, sigmoid output. Parameters (FP32 master, 9409 values):
// W1[64][48], b1[64], W2[64][64], b2[64], W3[32][64], b3[32], W4[32], b4.
//
// Forward: one warp scores 16 samples per step with mma.sync m16n8k16
// (BF16 A and B, FP32 accumulate). The accumulator fragment of one layer is
// the A fragment of the next (the m16n8 C layout of two adjacent n-tiles is
// the m16k16 A layout), so activations never leave registers; weights are
// read from shared memory. Layer inputs and W1..W3 are BF16 (round to nearest
// even); W4 and the last dot product are FP32.
// Backward: the chain rule through the BF16 weights, FP32 on CUDA cores:
// per-sample deltas, then per-parameter sums over the batch; Adam update.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lst.h"
#include "lst_kernels.cuh"
#include "lst_mlp.cuh"

namespace lst {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct MlpSmem {
    __nv_bfloat16 w1[kH1 * kIn];
    __nv_bfloat16 w2[kH2 * kH1];
    __nv_bfloat16 w3[kH3 * kH2];
    float b1[kH1], b2[kH2], b3[kH3], w4[kH3], b4;
};

// B fragment (k rows 16s + 2t + {0,1} (+8), n column 8j + g) of W[o][i] (row o contiguous in i)
__device__ __forceinline__ void bfrag(const __nv_bfloat16* W, int n_in, int s, int j, int g, int t, uint32_t& b0,
                                      uint32_t& b1) {
    const __nv_bfloat16* row = W + (8 * j + g) * n_in + 16 * s + 2 * t;
    b0 = *reinterpret_cast<const uint32_t*>(row);
    b1 = *reinterpret_cast<const uint32_t*>(row + 8);
}

// One warp's 16 rows base .. base + 15 (rows >= n skipped) through every
// layer: row r's features come from load(r, c) (two adjacent inputs c, c + 1
// as a float2). scores[r] = sigmoid(z4); keep (optional) receives
// scores[r] >= thr; save (optional) keeps the BF16-rounded layer inputs, h3 and
// z4 for the backward pass. All 32 lanes must call.
template <typename Load>
__device__ __forceinline__ void mlp_rows16(const MlpSmem& S, Load load, int n, int base, float* __restrict__ scores,
                                           MlpSaved save, uint8_t* keep, float thr) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = base + g, r1 = base + g + 8;
    // layer 1: A fragments straight from the FP32 features
    uint32_t a[3][4];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int c = 16 * s + 2 * t;
        float2 v00 = r0 < n ? load(r0, c) : make_float2(0.f, 0.f);
        float2 v10 = r1 < n ? load(r1, c) : make_float2(0.f, 0.f);
        float2 v01 = r0 < n ? load(r0, c + 8) : make_float2(0.f, 0.f);
        float2 v11 = r1 < n ? load(r1, c + 8) : make_float2(0.f, 0.f);
        a[s][0] = pack_bf16(v00.x, v00.y);
        a[s][1] = pack_bf16(v10.x, v10.y);
        a[s][2] = pack_bf16(v01.x, v01.y);
        a[s][3] = pack_bf16(v11.x, v11.y);
    }
    float h1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float bb0 = S.b1[8 * j + 2 * t], bb1 = S.b1[8 * j + 2 * t + 1];
        h1[j][0] = bb0; h1[j][1] = bb1; h1[j][2] = bb0; h1[j][3] = bb1;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            uint32_t b0, b1;
            bfrag(S.w1, kIn, s, j, g, t, b0, b1);
            mma_bf16(h1[j], a[s], b0, b1);
        }
    }
    // ReLU, BF16, and the layer-2 A fragments from the layer-1 accumulators
    uint32_t a2[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a2[s][0] = pack_bf16(fmaxf(h1[2 * s][0], 0.f), fmaxf(h1[2 * s][1], 0.f));
        a2[s][1] = pack_bf16(fmaxf(h1[2 * s][2], 0.f), fmaxf(h1[2 * s][3], 0.f));
        a2[s][2] = pack_bf16(fmaxf(h1[2 * s + 1][0], 0.f), fmaxf(h1[2 * s + 1][1], 0.f));
        a2[s][3] = pack_bf16(fmaxf(h1[2 * s + 1][2], 0.f), fmaxf(h1[2 * s + 1][3], 0.f));
    }
    if (save.x1) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&a2[s][q]);
                const int row = (q & 1) ? r1 : r0;
                const int col = 16 * s + 8 * (q >> 1) + 2 * t;
                if (row < n)
                    *reinterpret_cast<float2*>(save.x1 + (size_t)row * kH1 + col) =
                        make_float2(__bfloat162float(v.x), __bfloat162float(v.y));
            }
        }
    }
    float h2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float bb0 = S.b2[8 * j + 2 * t], bb1 = S.b2[8 * j + 2 * t + 1];
        h2[j][0] = bb0; h2[j][1] = bb1; h2[j][2] = bb0; h2[j][3] = bb1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            uint32_t b0, b1;
            bfrag(S.w2, kH1, s, j, g, t, b0, b1);
            mma_bf16(h2[j], a2[s], b0, b1);
        }
    }
    uint32_t a3[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a3[s][0] = pack_bf16(fmaxf(h2[2 * s][0], 0.f), fmaxf(h2[2 * s][1], 0.f));
        a3[s][1] = pack_bf16(fmaxf(h2[2 * s][2], 0.f), fmaxf(h2[2 * s][3], 0.f));
        a3[s][2] = pack_bf16(fmaxf(h2[2 * s + 1][0], 0.f), fmaxf(h2[2 * s + 1][1], 0.f));
        a3[s][3] = pack_bf16(fmaxf(h2[2 * s + 1][2], 0.f), fmaxf(h2[2 * s + 1][3], 0.f));
    }
    if (save.x2) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&a3[s][q]);
                const int row = (q & 1) ? r1 : r0;
                const int col = 16 * s + 8 * (q >> 1) + 2 * t;
                if (row < n)
                    *reinterpret_cast<float2*>(save.x2 + (size_t)row * kH2 + col) =
                        make_float2(__bfloat162float(v.x), __bfloat162float(v.y));
            }
        }
    }
    float h3[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float bb0 = S.b3[8 * j + 2 * t], bb1 = S.b3[8 * j + 2 * t + 1];
        h3[j][0] = bb0; h3[j][1] = bb1; h3[j][2] = bb0; h3[j][3] = bb1;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            uint32_t b0, b1;
            bfrag(S.w3, kH2, s, j, g, t, b0, b1);
            mma_bf16(h3[j], a3[s], b0, b1);
        }
    }
    // layer 4 (FP32): rows g and g+8, reduced over the 4 lanes of the group
    float z0 = 0.f, z1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = 8 * j + 2 * t;
        const float p0 = fmaxf(h3[j][0], 0.f), p1 = fmaxf(h3[j][1], 0.f);
        const float q0 = fmaxf(h3[j][2], 0.f), q1 = fmaxf(h3[j][3], 0.f);
        z0 += p0 * S.w4[c] + p1 * S.w4[c + 1];
        z1 += q0 * S.w4[c] + q1 * S.w4[c + 1];
        if (save.h3) {
            if (r0 < n) *reinterpret_cast<float2*>(save.h3 + (size_t)r0 * kH3 + c) = make_float2(p0, p1);
            if (r1 < n) *reinterpret_cast<float2*>(save.h3 + (size_t)r1 * kH3 + c) = make_float2(q0, q1);
        }
    }
    z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
    z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
    z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
    z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
    if (t == 0) {
        const float s0 = 1.f / (1.f + expf(-(z0 + S.b4))), s1 = 1.f / (1.f + expf(-(z1 + S.b4)));
        if (r0 < n) scores[r0] = s0;
        if (r1 < n) scores[r1] = s1;
        if (keep) {
            if (r0 < n) keep[r0] = s0 >= thr;
            if (r1 < n) keep[r1] = s1 >= thr;
        }
        if (save.z4) {
            if (r0 < n) save.z4[r0] = z0 + S.b4;
            if (r1 < n) save.z4[r1] = z1 + S.b4;
        }
    }
}

__device__ __forceinline__ void mlp_load_weights(MlpSmem& S, const MlpParams& P) {
    for (int i = threadIdx.x; i < kH1 * kIn; i += blockDim.x) S.w1[i] = P.w1_bf[i];
    for (int i = threadIdx.x; i < kH2 * kH1; i += blockDim.x) S.w2[i] = P.w2_bf[i];
    for (int i = threadIdx.x; i < kH3 * kH2; i += blockDim.x) S.w3[i] = P.w3_bf[i];
    for (int i = threadIdx.x; i < kH1; i += blockDim.x) { S.b1[i] = P.b1[i]; S.b2[i] = P.b2[i]; }
    for (int i = threadIdx.x; i < kH3; i += blockDim.x) { S.b3[i] = P.b3[i]; S.w4[i] = P.w4[i]; }
    if (threadIdx.x == 0) S.b4 = P.b4[0];
    __syncthreads();
}

// Forward pass over n samples X [n][48]. scores[i] = sigmoid(z4); when save
// != nullptr the BF16-rounded layer inputs x1, x2 (as float), h3 and the
// score are kept for the backward pass.
__global__ void __launch_bounds__(128) k_mlp_forward(MlpParams P, const float* __restrict__ X, int n,
                                                     const int* n_dev, float* __restrict__ scores, MlpSaved save) {
    pdl_begin();
    __shared__ MlpSmem S;
    if (n_dev) n = min(*n_dev, n);      // in the chain the candidate count lives on the device
    mlp_load_weights(S, P);
    const int warps = gridDim.x * (blockDim.x >> 5);
    auto load = [&](int r, int c) { return *reinterpret_cast<const float2*>(X + (size_t)r * kIn + c); };
    for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16; base < n; base += warps * 16)
        mlp_rows16(S, load, n, base, scores, save, nullptr, 0.f);
}

// Learned triplet selection, fused: each warp computes the scoring features
// of 32 T3s (one per lane) into a BF16 shared-memory tile, runs the network
// over its two 16-row halves and writes the score and the keep flag (score >=
// threshold) of each T3. The features never go to global memory. The tile
// holds the BF16 values the first layer's fragments take anyway, so the scores
// equal those of an FP32 tile; at half its shared memory, four blocks of eight
// warps fit on an SM.
constexpr int kScoreWarps = 8;
constexpr int kTileStride = 56;       // BF16 per tile row: 112-byte rows, conflict-free fragment loads
__global__ void __launch_bounds__(kScoreWarps * 32, 4) k_t3_score(Arena A, DevCfg c, MlpParams P) {
    pdl_begin();
    __shared__ MlpSmem S;
    __shared__ __align__(16) __nv_bfloat16 F[kScoreWarps][32][kTileStride];
    mlp_load_weights(S, P);
    const int n = min(A.counters[2], A.t3_cap);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int base = (blockIdx.x * (blockDim.x >> 5) + w) * 32; base < n; base += warps * 32) {
        const int i = base + lane;
        if (i < n) {
            Pt<float> Pp[3], H[6];
            int code[3];
            t3_feature_inputs(A, i, Pp, H, code);
            float v[48];
            t3_features(c, Pp, H, code, v);
            uint4* f = reinterpret_cast<uint4*>(&F[w][lane][0]);
#pragma unroll
            for (int j = 0; j < 6; ++j)
                f[j] = make_uint4(pack_bf16(v[8 * j], v[8 * j + 1]), pack_bf16(v[8 * j + 2], v[8 * j + 3]),
                                  pack_bf16(v[8 * j + 4], v[8 * j + 5]), pack_bf16(v[8 * j + 6], v[8 * j + 7]));
        }
        __syncwarp();
        const __nv_bfloat16* tile = &F[w][0][0];
        auto load = [&](int r, int col) {
            return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(tile + (r - base) * kTileStride + col));
        };
        mlp_rows16(S, load, n, base, A.t3_mlp, MlpSaved{}, A.t3_ok, c.t3_threshold);
        mlp_rows16(S, load, n, base + 16, A.t3_mlp, MlpSaved{}, A.t3_ok, c.t3_threshold);
        __syncwarp();
    }
}

// Per-sample deltas of the mean BCE: dz4, dz3 (32), dz2 (64), dz1 (64), and
// the loss sum. Weights: the BF16-rounded values as FP32.
__global__ void __launch_bounds__(128) k_mlp_backward_samples(MlpParams P, const float* __restrict__ y, int n,
                                                              const float* __restrict__ scores, MlpSaved sv,
                                                              MlpDeltas D, float* loss_sum) {
    __shared__ float w2[kH2 * kH1];
    __shared__ float w3[kH3 * kH2];
    __shared__ float w4[kH3];
    for (int i = threadIdx.x; i < kH2 * kH1; i += blockDim.x) w2[i] = P.w2_r[i];
    for (int i = threadIdx.x; i < kH3 * kH2; i += blockDim.x) w3[i] = P.w3_r[i];
    for (int i = threadIdx.x; i < kH3; i += blockDim.x) w4[i] = P.w4[i];
    __syncthreads();
    float lsum = 0.f;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const float z4 = sv.z4[b];
        const float yb = y[b];
        lsum += fmaxf(z4, 0.f) - yb * z4 + log1pf(expf(-fabsf(z4)));
        const float d4 = (scores[b] - yb) / float(n);
        D.dz4[b] = d4;
        float d3[kH3];
#pragma unroll
        for (int k = 0; k < kH3; ++k) {
            d3[k] = sv.h3[(size_t)b * kH3 + k] > 0.f ? d4 * w4[k] : 0.f;
            D.dz3[(size_t)b * kH3 + k] = d3[k];
        }
        float d2[kH2];
        for (int j = 0; j < kH2; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < kH3; ++k) acc += d3[k] * w3[k * kH2 + j];
            d2[j] = sv.x2[(size_t)b * kH2 + j] > 0.f ? acc : 0.f;
            D.dz2[(size_t)b * kH2 + j] = d2[j];
        }
        for (int i = 0; i < kH1; ++i) {
            float acc = 0.f;
            for (int j = 0; j < kH2; ++j) acc += d2[j] * w2[j * kH1 + i];
            D.dz1[(size_t)b * kH1 + i] = sv.x1[(size_t)b * kH1 + i] > 0.f ? acc : 0.f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, lsum);
}

// Parameter gradient: one thread per parameter, summed over the batch.
__global__ void k_mlp_weight_grad(const float* __restrict__ X, int n, MlpSaved sv, MlpDeltas D,
                                  float* __restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    float acc = 0.f;
    if (p < kOffB1) {                       // W1[o][i]: sum_b dz1[b][o] x0[b][i]
        const int o = p / kIn, i = p % kIn;
        for (int b = 0; b < n; ++b)
            acc += D.dz1[(size_t)b * kH1 + o] * __bfloat162float(__float2bfloat16_rn(X[(size_t)b * kIn + i]));
    } else if (p < kOffW2) {
        const int o = p - kOffB1;
        for (int b = 0; b < n; ++b) acc += D.dz1[(size_t)b * kH1 + o];
    } else if (p < kOffB2) {
        const int q = p - kOffW2, o = q / kH1, i = q % kH1;
        for (int b = 0; b < n; ++b) acc += D.dz2[(size_t)b * kH2 + o] * sv.x1[(size_t)b * kH1 + i];
    } else if (p < kOffW3) {
        const int o = p - kOffB2;
        for (int b = 0; b < n; ++b) acc += D.dz2[(size_t)b * kH2 + o];
    } else if (p < kOffB3) {
        const int q = p - kOffW3, o = q / kH2, i = q % kH2;
        for (int b = 0; b < n; ++b) acc += D.dz3[(size_t)b * kH3 + o] * sv.x2[(size_t)b * kH2 + i];
    } else if (p < kOffW4) {
        const int o = p - kOffB3;
        for (int b = 0; b < n; ++b) acc += D.dz3[(size_t)b * kH3 + o];
    } else if (p < kOffB4) {
        const int k = p - kOffW4;
        for (int b = 0; b < n; ++b) acc += D.dz4[b] * sv.h3[(size_t)b * kH3 + k];
    } else {
        for (int b = 0; b < n; ++b) acc += D.dz4[b];
    }
    grad[p] = acc;
}

// Adam on the FP32 master parameters; c1, c2 = 1 / (1 - beta^step).
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float gr = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * gr;
    const float vv = b2 * v[p] + (1.f - b2) * gr * gr;
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// Derived copies of the master parameters: BF16 weights for the forward and
// their FP32 values for the backward.
__global__ void k_mlp_derive(const float* __restrict__ theta, MlpDerived P) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
        const float w = theta[p];
        const __nv_bfloat16 b = __float2bfloat16_rn(w);
        if (p < kOffB1) { P.w1_bf[p] = b; }
        else if (p >= kOffW2 && p < kOffB2) { P.w2_bf[p - kOffW2] = b; P.w2_r[p - kOffW2] = __bfloat162float(b); }
        else if (p >= kOffW3 && p < kOffB3) { P.w3_bf[p - kOffW3] = b; P.w3_r[p - kOffW3] = __bfloat162float(b); }
    }
}

}  // namespace lst
