// Allocation-free mini-doublet builder.
//
// Some callers cannot allocate device memory: a host framework that owns the
// whole device budget through its own pool and forbids plugins from calling
// cudaMalloc, or a latency-critical loop that must not pay for an allocation
// (cudaMalloc / cudaFree can synchronize the device). For them this file
// offers lst_build_mini_doublets_static: the hit binning of the chain
// (count, scan, scatter and the per-sensor sort by input index, so the same
// hits are kept when a sensor holds more than 256) and a one-warp-per-module
// mini-doublet kernel with the chain's predicates, with every scratch buffer
// (bucket counters and
// offsets, sorted hits, module table in device layout, per-module segments,
// MD anchors) placed in one file-scope __device__ array of fixed size. The
// caller passes device inputs and device outputs; nothing is allocated.
//
// Limits: 262144 hits, 16384 modules, 131072 mini-doublets per call; the
// array holds about 9 MB on every device that loads the library, until the
// process exits. Every call reuses the same array: calls that overlap on the
// GPU (two streams, two host threads) race on it and must be serialized by
// the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lst.h"
#include "lst_kernels.cuh"

using namespace lst;

namespace {

constexpr int kStaticMaxHits = 262144;
constexpr int kStaticMaxModules = 16384;
constexpr int kStaticMaxMd = 131072;
constexpr int kMaxDevices = 64;

struct alignas(256) MdScratch {
    BatchDesc bd;
    int hit_off[64];
    int counters[32];
    int ev_counts[32];
    int ev_drop[32];
    float4 mod[kStaticMaxModules];
    int bcnt[2 * kStaticMaxModules];
    int boff[2 * kStaticMaxModules + 64];
    float sx[kStaticMaxHits];
    float sy[kStaticMaxHits];
    float sz[kStaticMaxHits];
    int sidx[kStaticMaxHits];
    int md_moff[kStaticMaxModules];
    int md_mcnt[kStaticMaxModules];
    float4 md_p4[kStaticMaxMd];
    float2 md_sr[kStaticMaxMd];
    float md_dx[kStaticMaxMd];
    float md_dy[kStaticMaxMd];
};

}  // namespace

// The scratch array. In host code its name is only a stand-in for the symbol;
// its device address is obtained once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_md_scratch[sizeof(MdScratch)];

namespace {

std::mutex g_setup_mutex;
MdScratch* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_static_prepare(MdScratch* S, const lst_module* mods, int n_mod, int n_hits, const float* x,
                                 const float* y, const float* z, const int32_t* module, const uint8_t* side) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        S->hit_off[0] = 0;
        S->hit_off[1] = n_hits;
        S->bd.n_ev = 1;
        S->bd.n_hits = n_hits;
        S->bd.n_seeds = 0;
        S->bd.hx = x;
        S->bd.hy = y;
        S->bd.hz = z;
        S->bd.hmod = module;
        S->bd.hside = side;
        S->bd.seeds = nullptr;
    }
    for (; i < n_mod; i += gridDim.x * blockDim.x)
        S->mod[i] = make_float4(mods[i].dsep, mods[i].sig_rphi, mods[i].sig_long, float(mods[i].subdet));
}

// Rows written, and everything lost: MDs over the per-module bounds or over
// the capacity, plus hits ignored for an invalid module id or side
// (counters[16], counted by the binning).
__global__ void k_static_finish(const MdScratch* S, int cap, int* count, int* dropped) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *count = min(S->counters[0], cap);
        if (dropped) *dropped = S->ev_drop[0] + S->counters[16];
    }
}

DevCfg static_devcfg(const lst_config& c) {
    DevCfg d{};
    d.a = c.k_field * c.b_field / (200.0 * c.pt_min);
    d.z_lumi = c.z_lumi;
    d.n_md = c.n_md;
    d.k_field = c.k_field;
    d.b_field = c.b_field;
    d.f.a = float(d.a);
    d.f.z_lumi = float(d.z_lumi);
    d.f.n_md = float(d.n_md);
    return d;
}

// Per-device set-up on the first call: the array's device address and the
// MD kernel's shared-memory limit.
lst_status scratch_for_current_device(MdScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LST_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LST_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_md_scratch) != cudaSuccess || !p) return LST_ERR_CUDA;
        if (cudaFuncSetAttribute(k_md, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)md_smem_bytes()) !=
            cudaSuccess)
            return LST_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<MdScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LST_OK;
}

}  // namespace

extern "C" lst_status lst_build_mini_doublets_static(const lst_config* cfg, const lst_module* modules, int32_t n_mod,
                                                     const float* x, const float* y, const float* z,
                                                     const int32_t* module, const uint8_t* side, int32_t n_hits,
                                                     int32_t md_capacity, int32_t* md_lower, int32_t* md_upper,
                                                     int32_t* md_module, float* md_dphi, float* md_dlong,
                                                     int32_t* md_count, int32_t* md_dropped, void* cuda_stream) {
    if (!cfg || !modules || !md_lower || !md_upper || !md_module || !md_dphi || !md_dlong || !md_count)
        return LST_ERR_ARG;
    if (n_mod <= 0 || n_hits < 0 || md_capacity < 0) return LST_ERR_ARG;
    if (n_hits > 0 && (!x || !y || !z || !module || !side)) return LST_ERR_ARG;
    if (n_mod > kStaticMaxModules || n_hits > kStaticMaxHits || md_capacity > kStaticMaxMd)
        return LST_ERR_CAPACITY;
    MdScratch* S = nullptr;
    lst_status s = scratch_for_current_device(&S);
    if (s != LST_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Arena A{};
    A.n_mod = n_mod;
    A.mod = S->mod;
    A.bd = &S->bd;
    A.max_events = 1;
    A.hit_off = S->hit_off;
    A.bcnt = S->bcnt;
    A.boff = S->boff;
    A.sx = S->sx;
    A.sy = S->sy;
    A.sz = S->sz;
    A.sidx = S->sidx;
    A.counters = S->counters;
    A.ev_counts = S->ev_counts;
    A.ev_drop = S->ev_drop;
    A.md_cap = md_capacity;
    A.md_lo = md_lower;
    A.md_up = md_upper;
    A.md_gmod = md_module;          // one event: the unit index is the module id
    A.md_p4 = S->md_p4;
    A.md_sr = S->md_sr;
    A.md_dx = S->md_dx;
    A.md_dy = S->md_dy;
    A.md_dphi = md_dphi;
    A.md_dlong = md_dlong;
    A.md_moff = S->md_moff;
    A.md_mcnt = S->md_mcnt;
    const DevCfg dc = static_devcfg(*cfg);
    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(S->counters, 0, sizeof(S->counters) + sizeof(S->ev_counts) + sizeof(S->ev_drop), st) !=
            cudaSuccess ||
        cudaMemsetAsync(S->bcnt, 0, sizeof(int) * 2 * (size_t)n_mod, st) != cudaSuccess)
        return LST_ERR_CUDA;
    int n_sm = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LST_ERR_CUDA;
    const int hb = (n_hits + 255) / 256;
    const int hit_blocks = hb < 1 ? 1 : (hb > 8 * n_sm ? 8 * n_sm : hb);
    k_static_prepare<<<(n_mod + 255) / 256, 256, 0, st>>>(S, modules, n_mod, n_hits, x, y, z, module, side);
    k_bin_count<<<hit_blocks, 256, 0, st>>>(A);
    k_bin_scan<<<1, 1024, 0, st>>>(A);
    k_bin_scatter<<<hit_blocks, 256, 0, st>>>(A);
    k_bin_sort<<<4 * n_sm, 128, 0, st>>>(A);
    k_md<<<4 * n_sm, kMdWarps * 32, md_smem_bytes(), st>>>(A, dc);
    k_static_finish<<<1, 32, 0, st>>>(S, md_capacity, md_count, md_dropped);
    return cudaGetLastError() == cudaSuccess ? LST_OK : LST_ERR_CUDA;
}
