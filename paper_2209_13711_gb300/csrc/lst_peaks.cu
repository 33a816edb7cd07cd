// Calibration kernels: the device's FP32 and FP64 FMA rates and its global
// atomic rates, measured with the library's own kernels. They are the
// denominators of the per-kernel ALU and atomic fractions reported beside
// the HBM fraction; none of them is on the track-finding path.
//
// Every kernel runs a fixed number of iterations and indexes its buffer
// through a power-of-two mask, so every access stays inside the buffer.
#include <cuda_runtime.h>

#include "../../include/lst.h"

namespace {

constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kFmaIters = 16384;      // x 8 chains x 2 flop per thread
constexpr int kDfmaIters = 512;       // x 4 chains x 2 flop per thread
constexpr int kAtomIters = 512;       // per warp (distinct lines)
constexpr int kSameIters = 32;        // per warp (one shared address)
constexpr int kRedIters = 256;        // per lane
constexpr unsigned kLines = 1u << 16;  // 128-byte lines of the warp-atomic buffer (8 MB)
constexpr unsigned kWords = 1u << 22;  // words of the lane-atomic buffer (16 MB)

// Eight independent FFMA chains per thread (enough to cover the pipe latency).
__global__ void __launch_bounds__(kBlock) k_peak_ffma(float* out, int iters, float b, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) k_peak_dfma(double* out, int iters, double b, double c) {
    double a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = fma(a[k], b, c);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a[0] + a[1] + a[2] + a[3];
}

// One single-lane atomicAdd with a used return per warp and iteration (the
// form of the chain's warp-aggregated counters), each on its own 128-byte
// line, the lines spread over the buffer.
__global__ void __launch_bounds__(kBlock) k_peak_atom_warp(unsigned* buf, int iters) {
    const unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned s = 0;
    if ((threadIdx.x & 31) == 0) {
        for (int i = 0; i < iters; ++i) s += atomicAdd(&buf[((w + 9973u * i) & (kLines - 1)) * 32], 1u);
    }
    if (s == 0xffffffffu) buf[(w & (kLines - 1)) * 32 + 1] = s;   // keeps the returns live
}

// The same on one address shared by every warp: the contended rate.
__global__ void __launch_bounds__(kBlock) k_peak_atom_same(unsigned* buf, int iters) {
    unsigned s = 0;
    if ((threadIdx.x & 31) == 0) {
        for (int i = 0; i < iters; ++i) s += atomicAdd(&buf[0], 1u);
    }
    if (s == 0xffffffffu) buf[1] = s;
}

// Every lane adds to its own word without using the result (reductions),
// consecutive lanes on consecutive words.
__global__ void __launch_bounds__(kBlock) k_peak_red_lane(unsigned* buf, int iters) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < iters; ++i) atomicAdd(&buf[(t + 1048573u * i) & (kWords - 1)], 1u);
}

struct Timer {
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (st) cudaStreamDestroy(st);
    }
};

// Best of three timed launches (after one untimed), in milliseconds; < 0 on a CUDA error.
template <typename Launch>
float best_ms(Timer& t, Launch launch) {
    launch();
    float best = -1.f;
    for (int r = 0; r < 3; ++r) {
        if (cudaEventRecord(t.a, t.st) != cudaSuccess) return -1.f;
        launch();
        if (cudaEventRecord(t.b, t.st) != cudaSuccess || cudaEventSynchronize(t.b) != cudaSuccess) return -1.f;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) return -1.f;
        if (best < 0.f || ms < best) best = ms;
    }
    return cudaGetLastError() == cudaSuccess ? best : -1.f;
}

}  // namespace

extern "C" lst_status lst_measure_peaks(int32_t device, lst_peaks* out) {
    if (!out || device < 0) return LST_ERR_ARG;
    int n_sm = 0, clk = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return LST_ERR_CUDA;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);   // kHz; informational
    const int blocks = n_sm * kBlocksPerSm;
    const size_t threads = (size_t)blocks * kBlock;
    Timer t;
    if (cudaStreamCreateWithFlags(&t.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess)
        return LST_ERR_CUDA;
    void* buf = nullptr;
    const size_t bytes = sizeof(unsigned) * (size_t)kWords;   // >= kLines * 128 B and >= threads * 8 B
    if (bytes < (size_t)kLines * 128 || bytes < threads * sizeof(double)) return LST_ERR_ARG;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return LST_ERR_OOM;
    lst_status s = LST_OK;
    if (cudaMemsetAsync(buf, 0, bytes, t.st) != cudaSuccess) s = LST_ERR_CUDA;
    float ms[5] = {-1.f, -1.f, -1.f, -1.f, -1.f};
    if (s == LST_OK) {
        ms[0] = best_ms(t, [&] { k_peak_ffma<<<blocks, kBlock, 0, t.st>>>((float*)buf, kFmaIters, 0.999f, 1e-3f); });
        ms[1] = best_ms(t, [&] { k_peak_dfma<<<blocks, kBlock, 0, t.st>>>((double*)buf, kDfmaIters, 0.999, 1e-3); });
        ms[2] = best_ms(t, [&] { k_peak_atom_warp<<<blocks, kBlock, 0, t.st>>>((unsigned*)buf, kAtomIters); });
        ms[3] = best_ms(t, [&] { k_peak_atom_same<<<blocks, kBlock, 0, t.st>>>((unsigned*)buf, kSameIters); });
        ms[4] = best_ms(t, [&] { k_peak_red_lane<<<blocks, kBlock, 0, t.st>>>((unsigned*)buf, kRedIters); });
        for (float m : ms)
            if (!(m > 0.f)) s = LST_ERR_CUDA;
    }
    cudaFree(buf);
    if (s != LST_OK) return s;
    const double warps = threads / 32.0;
    out->fp32_tflops = threads * kFmaIters * 8.0 * 2.0 / (ms[0] * 1e-3) / 1e12;
    out->fp64_tflops = threads * kDfmaIters * 4.0 * 2.0 / (ms[1] * 1e-3) / 1e12;
    out->atom_warp_gops = warps * kAtomIters / (ms[2] * 1e-3) / 1e9;
    out->atom_same_gops = warps * kSameIters / (ms[3] * 1e-3) / 1e9;
    out->red_lane_gops = threads * kRedIters / (ms[4] * 1e-3) / 1e9;
    for (int k = 0; k < 5; ++k) out->ms[k] = ms[k];
    out->sm_count = n_sm;
    out->clock_khz = clk;
    return LST_OK;
}
