// C ABI of the Segment Linking library: context, device memory, launch
// sequence and result readback. See include/lst.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lst.h"
#include "lst_kernels.cuh"
#include "lst_mlp.cuh"

lst::MlpParams lst_mlp_device_params(const lst_mlp* m);

using namespace lst;

namespace {

constexpr size_t kAlign = 256;

struct Buffer {
    void* base = nullptr;
    size_t size = 0, used = 0;
    template <typename T> T* take(size_t n) {
        size_t off = (used + kAlign - 1) / kAlign * kAlign;
        used = off + std::max<size_t>(n, 1) * sizeof(T);
        return base ? reinterpret_cast<T*>(static_cast<char*>(base) + off) : nullptr;
    }
};

// The stages of the chain (Fig. KernelFlow order) with their default launch
// shape. `generic` stages index threads only through blockDim and grid-stride
// loops, so any block size is valid for them; the warp-per-unit stages size
// their shared-memory stages by a compile-time warp count and keep their block.
// `tunable` stages are grid-stride over their units, so any grid is valid.
enum LaunchId {
    L_RESET, L_BIN_COUNT, L_BIN_SCAN, L_BIN_SCATTER, L_BIN_SORT, L_MD_PLAN, L_MD, L_MD_WRITE, L_LS, L_T3,
    L_T3_FEAT, L_T3_SCORE, L_T5_PLAN, L_T5, L_T5_GATHER, L_T5_REFINE,
    L_T5_MLP, L_T5_MLP_SELECT, L_PLS, L_PT_PLAN, L_T3_ORDER, L_PT5, L_PT5_REFINE, L_PT3, L_PT3_REFINE, L_CLEAN_KEYS, L_CLEAN_KEEP,
    L_CLEAN_PT5, L_CLEAN_PT3_CROSS, L_CLEAN_PT3_MARK, L_CLEAN_T5, L_CLEAN_PLS, L_TC_PACK, kNumLaunch
};

struct LaunchInfo {
    const char* name;
    int bpsm;       // default blocks per SM
    int block;      // default threads per block
    bool tunable;   // grid may change
    bool generic;   // block size may change
};

const LaunchInfo kLaunch[kNumLaunch] = {
    {"reset", 8, 256, true, true},
    {"bin_count", 8, 256, true, true},
    {"bin_scan", 0, 1024, false, false},        // one block per event
    {"bin_scatter", 8, 256, true, true},
    {"bin_sort", 4, 128, true, false},
    {"md_plan", 4, 256, true, true},
    {"md", 4, kMdWarps * 32, true, false},
    {"md_write", 4, 128, true, false},
    {"ls", 8, kLsWarps * 32, true, false},
    {"t3", 8, kT3Warps * 32, true, false},
    {"t3_features", 4, 128, true, true},
    {"t3_score", 4, 256, true, false},
    {"t5_plan", 4, 256, true, true},
    {"t5", 6, kT5Warps * 32, true, false},
    {"t5_gather", 4, 128, true, false},
    {"t5_refine", 4, 128, true, true},
    {"t5_mlp", 4, 128, true, false},
    {"t5_mlp_select", 4, 128, true, true},
    {"pls", 4, 128, true, true},
    {"pt_plan", 4, 256, true, true},
    {"t3_order", 8, 256, true, false},
    {"pt5", 8, kPtWarps * 32, true, false},
    {"pt5_refine", 2, 128, true, true},
    {"pt3", 8, kPtWarps * 32, true, false},
    {"pt3_refine", 2, 128, true, true},
    {"clean_keys", 4, 256, true, true},
    {"clean_keep", 4, 256, true, true},
    {"clean_pt5", 2, 256, true, true},
    {"clean_pt3_cross", 2, 256, true, true},
    {"clean_pt3_mark", 2, 256, true, true},
    {"clean_t5", 4, 256, true, true},
    {"clean_pls", 4, 128, true, true},
    {"tc_pack", 1, 256, true, true},
};

struct LaunchCfg {
    int bpsm = 0;    // 0: the default
    int block = 0;
};

}  // namespace

struct lst_ctx {
    int device = 0;
    int n_sm = 0;
    lst_config cfg{};
    lst_capacity cap{};
    DevCfg dc{};
    bool geometry = false;
    void* dev_mem = nullptr;
    size_t dev_bytes = 0;
    Arena A{};              // pointers into dev_mem; batch fields set per run
    // device input staging (host-memory inputs are copied here)
    float* in_x = nullptr;
    float* in_y = nullptr;
    float* in_z = nullptr;
    int* in_mod = nullptr;
    uint8_t* in_side = nullptr;
    float* in_seeds = nullptr;
    int* d_hit_off = nullptr;
    int* d_seed_off = nullptr;
    int* h_offsets = nullptr;   // pinned: [2 (max_events + 1)]
    cudaEvent_t done = nullptr;
    bool ran = false;
    int n_ev = 0;
    // Result slots: the packed track candidates, offsets and per-event
    // statistics of a batch (written by the chain's last stage). A batch run
    // with handles holds its slot until every event is released; a batch run
    // without gives it up to the next run.
    struct Slot {
        TcRec* rec = nullptr;
        int* off = nullptr;
        int* stats = nullptr;
        cudaEvent_t done = nullptr;
        uint32_t gen = 0;              // generation of the batch in the slot (0: none)
        int n_ev = 0;
        int held = 0;                  // events not released (0: the slot is free)
        std::vector<char> released;
    } slot[LST_RESULT_SLOTS];
    uint32_t next_gen = 1;
    int last = -1;                     // slot of the last batch (its intermediate objects are in the arena)
    int launches = 0;
    std::vector<int> hit_off_host, seed_off_host;
    bool profiling = false;
    bool use_graph = true;
    const lst_mlp* mlp = nullptr;     // network deciding T5 validity (NULL: the hand-set cuts)
    const lst_mlp* mlp3 = nullptr;    // network pruning triplets (NULL: every T3 that passes the cuts)
    bool t3_features = false;         // the T3 buffers exist (network attached or features captured)
    bool t3_capture = false;          // write the T3 scoring features out (training)
    void* t3_mem = nullptr;           // features, scores and flags of the learned triplet selection
    BatchDesc* d_bd = nullptr;        // device batch descriptor
    BatchDesc* h_bd = nullptr;        // pinned staging of the descriptor
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;   // second branch of the captured graph (pLS, pT3)
    cudaEvent_t ev_fork = nullptr, ev_t3 = nullptr, ev_plan = nullptr, ev_pt3 = nullptr;
    cudaGraphExec_t graph = nullptr;
    LaunchCfg tune[kNumLaunch];       // per-stage launch shape (autotuner or caller)
    static constexpr int kMaxProf = 64;
    cudaEvent_t prof_ev[2 * kMaxProf] = {};
    const char* prof_name[kMaxProf] = {};
    int prof_id[kMaxProf] = {};
};

#define CK(x)                                      \
    do {                                           \
        cudaError_t err__ = (x);                   \
        if (err__ != cudaSuccess) return LST_ERR_CUDA; \
    } while (0)

// FP32 limits of the fit prefilter: rejected only when a cut fails by far
// more than FP32 rounding can explain: |kappa| above 1.01 kmax + 1e-5, a chi2
// above rel * chi2_max + abs. T5: rel 1.05, abs 0.2 (the FP32 five-point fit's
// chi2 differs from FP64 by at most 1.3e-3 relative over the 2e6 candidates of
// a PU200 event); pT5/pT3 (pixel points, 10 um errors): rel 1.25, abs 2.
static FitLimits prefit_limits(const DevCfg& d, double chi2_max, double chi2z_max, float scale, float rel,
                               float abs_) {
    const float kmax = float((1.0 + d.tol_r) * 2.0 * d.a);
    return FitLimits{kmax * 1.01f + 1e-5f, rel * (float(chi2_max) * scale) + abs_,
                     rel * (float(chi2z_max) * scale) + abs_};
}

static void derive_fp32(DevCfg& d) {
    d.f = CfgF{float(d.a),    float(d.z_lumi), float(d.n_md), float(d.n_ls),
               float(d.n_t3), float(d.n_t5),   float(d.n_pt), float(d.sig_pix)};
    d.lim_t5 = prefit_limits(d, d.chi2_rphi_t5, d.chi2_rz_t5, d.prefit_scale, 1.05f, 0.2f);
    d.lim_pt5 = prefit_limits(d, d.chi2_rphi_pt5, d.chi2_rz_pt5, 1.0f, 1.25f, 2.f);
    d.lim_pt3 = prefit_limits(d, d.chi2_rphi_pt3, d.chi2_rz_pt3, 1.0f, 1.25f, 2.f);
}

static DevCfg make_devcfg(const lst_config& c) {
    DevCfg d{};
    d.a = c.k_field * c.b_field / (200.0 * c.pt_min);
    d.z_lumi = c.z_lumi; d.n_md = c.n_md; d.n_ls = c.n_ls; d.n_t3 = c.n_t3; d.n_t5 = c.n_t5; d.n_pt = c.n_pt;
    d.tol_r = c.tol_r;
    d.chi2_rphi_t5 = c.chi2_rphi_t5; d.chi2_rz_t5 = c.chi2_rz_t5;
    d.chi2_rphi_pt3 = c.chi2_rphi_pt3; d.chi2_rz_pt3 = c.chi2_rz_pt3;
    d.chi2_rphi_pt5 = c.chi2_rphi_pt5; d.chi2_rz_pt5 = c.chi2_rz_pt5;
    d.pls_pt_tol = c.pls_pt_tol; d.sig_pix = c.sig_pix; d.sb_eta_max = c.sb_eta_max;
    d.sb_n_eta = c.sb_n_eta; d.sb_n_phi = c.sb_n_phi;
    d.dr_clean = c.dr_clean; d.k_field = c.k_field; d.b_field = c.b_field;
    d.features_on = 0;
    d.use_mlp = 0;
    d.fp64_fit = 0;
    d.prefit_scale = 1.0f;
    d.mlp_threshold = 0.5f;
    d.t5_stage = kT5Stage;
    d.pt_stage = kPtStage;
    derive_fp32(d);
    return d;
}

template <typename T> static lst_status fetch(std::vector<T>& v, const T* d, size_t n) {
    v.resize(n);
    if (n) CK(cudaMemcpy(v.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost));
    return LST_OK;
}

extern "C" {

const char* lst_status_str(lst_status s) {
    switch (s) {
        case LST_OK: return "ok";
        case LST_WARN_TRUNCATED: return "output truncated by a capacity";
        case LST_ERR_ARG: return "invalid argument";
        case LST_ERR_CUDA: return "CUDA runtime error";
        case LST_ERR_OOM: return "device allocation failed";
        case LST_ERR_NO_GEOMETRY: return "geometry not loaded";
        case LST_ERR_TIMEOUT: return "device wait timed out";
        case LST_ERR_CAPACITY: return "batch exceeds the context capacity";
    }
    return "unknown status";
}

lst_status lst_config_default(lst_config* c) {
    if (!c) return LST_ERR_ARG;
    *c = lst_config{};
    c->pt_min = 0.8; c->k_field = 0.3; c->b_field = 3.8; c->z_lumi = 20.0;
    c->n_md = 3; c->n_ls = 3; c->n_t3 = 3; c->n_t5 = 3; c->n_pt = 3; c->tol_r = 0.05;
    c->chi2_rphi_t5 = 15; c->chi2_rz_t5 = 17; c->chi2_rphi_pt3 = 17; c->chi2_rz_pt3 = 19;
    c->chi2_rphi_pt5 = 21; c->chi2_rz_pt5 = 23;
    c->pls_pt_tol = 0.05; c->sig_pix = 0.001; c->sb_eta_max = 3.0; c->sb_n_eta = 120; c->sb_n_phi = 72;
    c->dr_clean = 0.02;
    return LST_OK;
}

lst_status lst_capacity_default(lst_capacity* c, int32_t max_events) {
    if (!c || max_events <= 0) return LST_ERR_ARG;
    c->max_events = max_events;
    c->max_hits = 140000 * max_events;
    c->max_seeds = 10000 * max_events;
    c->md_per_event = 80000;
    c->ls_per_event = 400000;
    c->t3_per_event = 800000;
    c->t5_per_event = 100000;
    c->pt3_per_event = 40000;
    c->pt5_per_event = 40000;
    c->tc_per_event = 16000;
    return LST_OK;
}

lst_status lst_create(lst_ctx** out, const lst_config* cfg, const lst_capacity* cap, int32_t device) {
    if (!out) return LST_ERR_ARG;
    *out = nullptr;
    if (!cfg || !cap || cap->max_events <= 0 || cap->max_events > 8192 || cap->max_hits < 0 || cap->max_seeds < 0)
        return LST_ERR_ARG;
    lst_ctx* c = new (std::nothrow) lst_ctx();
    if (!c) return LST_ERR_OOM;
    c->device = device;
    c->cfg = *cfg;
    c->cap = *cap;
    c->dc = make_devcfg(*cfg);
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&c->h_offsets, sizeof(int) * 2 * (cap->max_events + 1)) != cudaSuccess ||
        cudaMallocHost(&c->h_bd, sizeof(BatchDesc)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_t3, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_plan, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_pt3, cudaEventDisableTiming) != cudaSuccess) {
        delete c;
        return LST_ERR_CUDA;
    }
    for (auto& sl : c->slot)
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            lst_destroy(c);
            return LST_ERR_CUDA;
        }
    *out = c;
    return LST_OK;
}

void lst_destroy(lst_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->done) {
        cudaEventSynchronize(c->done);
        cudaEventDestroy(c->done);
    }
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    for (cudaEvent_t e : {c->ev_fork, c->ev_t3, c->ev_plan, c->ev_pt3})
        if (e) cudaEventDestroy(e);
    for (auto& sl : c->slot)
        if (sl.done) cudaEventDestroy(sl.done);
    if (c->dev_mem) cudaFree(c->dev_mem);
    if (c->t3_mem) cudaFree(c->t3_mem);
    if (c->h_offsets) cudaFreeHost(c->h_offsets);
    if (c->h_bd) cudaFreeHost(c->h_bd);
    for (cudaEvent_t& e : c->prof_ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

// Carve every device buffer out of one allocation (first pass with a null
// base only measures).
static void layout(lst_ctx* c, Buffer& b, int n_mod, int n_conn, int n_sb, int n_sbt, int max_sbt) {
    const lst_capacity& K = c->cap;
    const size_t E = K.max_events, H = K.max_hits, S = K.max_seeds;
    Arena& A = c->A;
    A.n_mod = n_mod;
    A.n_sb = n_sb;
    A.mod = b.take<float4>(n_mod);
    A.mod_layer = b.take<int>(n_mod);
    A.conn_off = b.take<int>(n_mod + 1);
    A.conn_tgt = b.take<int>(n_conn);
    A.sb_off = b.take<int>(n_sb + 1);
    A.sb_tgt = b.take<int>(n_sbt);
    c->d_hit_off = b.take<int>(E + 1);
    c->d_seed_off = b.take<int>(E + 1);
    c->d_bd = b.take<BatchDesc>(1);
    A.bd = c->d_bd;
    A.max_events = (int)E;
    A.hit_off = c->d_hit_off;
    A.seed_off = c->d_seed_off;
    c->in_x = b.take<float>(H);
    c->in_y = b.take<float>(H);
    c->in_z = b.take<float>(H);
    c->in_mod = b.take<int>(H);
    c->in_side = b.take<uint8_t>(H);
    c->in_seeds = b.take<float>(9 * S);
    A.bcnt = b.take<int>(E * 2 * n_mod);
    A.boff = b.take<int>(E * (2 * n_mod + 1));
    A.sx = b.take<float>(H);
    A.sy = b.take<float>(H);
    A.sz = b.take<float>(H);
    A.sidx = b.take<int>(H);
    A.counters = b.take<int>(32);
    A.ev_counts = b.take<int>(E * 8);
    A.ev_drop = b.take<int>(E * 8);
    const size_t MD = E * K.md_per_event;
    A.md_cap = (int)MD;
    A.md_lo = b.take<int>(MD); A.md_up = b.take<int>(MD); A.md_gmod = b.take<int>(MD);
    A.md_p4 = b.take<float4>(MD); A.md_sr = b.take<float2>(MD); A.md_lsc = b.take<float4>(MD);
    A.md_dx = b.take<float>(MD); A.md_dy = b.take<float>(MD);
    A.md_dphi = b.take<float>(MD); A.md_dlong = b.take<float>(MD);
    A.md_moff = b.take<int>(E * n_mod); A.md_mcnt = b.take<int>(E * n_mod);
    A.md_item_cap = (int)std::max<size_t>(H, 1);
    A.md_items = b.take<int2>(A.md_item_cap);
    A.md_chunk_off = b.take<int>(H); A.md_chunk_cnt = b.take<int>(H);
    A.md_tmp = b.take<int2>(MD);
    const size_t LS = E * K.ls_per_event;
    A.ls_cap = (int)LS;
    A.ls_in = b.take<int>(LS); A.ls_out = b.take<int>(LS); A.ls_dphi = b.take<float>(LS);
    A.ls_off = b.take<int>(MD); A.ls_cnt = b.take<int>(MD);
    const size_t T3 = E * K.t3_per_event;
    A.t3_cap = (int)T3;
    A.t3_lsin = b.take<int>(T3); A.t3_lsout = b.take<int>(T3);
    A.t3_beta = b.take<float>(T3); A.t3_ks = b.take<float2>(T3);
    A.t3_ksh = b.take<__half2>(T3);
    A.two_a = float(2.0 * c->dc.a);
    A.t3_md = b.take<int4>(T3);
    A.t3_off = b.take<int>(MD); A.t3_cnt = b.take<int>(MD);
    A.t3_perm = b.take<int>(T3); A.t3_kord = b.take<float2>(T3); A.t3_smax = b.take<float>(MD);
    const size_t T5 = E * K.t5_per_event;
    A.t5_cap = (int)T5;
    A.t5_in = b.take<int>(T5); A.t5_out = b.take<int>(T5);
    A.t5_kappa = b.take<double>(T5); A.t5_sigk = b.take<double>(T5);
    A.t5_eta = b.take<double>(T5); A.t5_phi = b.take<double>(T5);
    A.t5_chi2 = b.take<float>(T5); A.t5_chi2z = b.take<float>(T5); A.t5_score = b.take<float>(T5);
    A.t5_pt = b.take<float>(T5); A.t5_valid = b.take<uint8_t>(T5); A.t5_cut = b.take<uint8_t>(T5);
    A.t5_feat = b.take<float>(48 * T5); A.t5_mlp = b.take<float>(T5);
    A.t5_off = b.take<int>(MD); A.t5_cnt = b.take<int>(MD);
    A.t5_ks = b.take<float2>(T5);
    A.t5_evf = b.take<int>(E);
    A.t5_evb = b.take<int>(E);
    A.t5_evc = b.take<int>(E);
    A.t5_evbase = b.take<int>(E + 1);
    A.t5_items = b.take<int>(T3); A.t5_chunk_off = b.take<int>(T3); A.t5_chunk_cnt = b.take<int>(T3);
    A.t5_tmp = b.take<int2>(T5);
    A.pls_pass = b.take<int>(S); A.pls_sb = b.take<int>(S);
    A.pls_kappa = b.take<double>(S); A.pls_sigk = b.take<double>(S);
    A.pls_eta = b.take<double>(S); A.pls_phi = b.take<double>(S);
    A.pls_z0 = b.take<float>(S); A.pls_pt = b.take<float>(S);
    A.pt_item_cap = (int)std::min<size_t>(S * (size_t)std::max((max_sbt + kPtChunk - 1) / kPtChunk, 1),
                                          (size_t)INT32_MAX / 2);
    A.pt_items = b.take<int2>(A.pt_item_cap);
    const size_t P5 = E * K.pt5_per_event, P3 = E * K.pt3_per_event;
    A.pt5_cap = (int)P5;
    A.pt5_seed = b.take<int>(P5); A.pt5_obj = b.take<int>(P5); A.pt5_kappa = b.take<float>(P5);
    A.pt5_chi2 = b.take<float>(P5); A.pt5_chi2z = b.take<float>(P5); A.pt5_score = b.take<float>(P5);
    A.pt5_pt = b.take<float>(P5); A.pt5_valid = b.take<uint8_t>(P5);
    A.pt3_cap = (int)P3;
    A.pt3_seed = b.take<int>(P3); A.pt3_obj = b.take<int>(P3); A.pt3_kappa = b.take<float>(P3);
    A.pt3_chi2 = b.take<float>(P3); A.pt3_chi2z = b.take<float>(P3); A.pt3_score = b.take<float>(P3);
    A.pt3_pt = b.take<float>(P3); A.pt3_valid = b.take<uint8_t>(P3);
    const size_t NK = H + 3 * S;
    A.best = b.take<unsigned long long>(3 * NK);
    A.mark = b.take<int>(NK);
    A.obj_key = b.take<unsigned long long>(P5 + P3 + T5);
    A.obj_meta = b.take<int>(P5 + P3 + T5);
    A.obj_slot = b.take<int>(16 * (P5 + P3 + T5));
    A.keep_pt5 = b.take<uint8_t>(P5); A.keep_pt3 = b.take<uint8_t>(P3); A.keep_t5 = b.take<uint8_t>(T5);
    A.seed_link = b.take<int>(S);
    A.list_cap = 32768;
    A.list_cnt = b.take<int>(E * 2);
    A.list_ef = b.take<float2>(E * 2 * A.list_cap);
    A.list_ref = b.take<int>(E * 2 * A.list_cap);
    A.list_q = b.take<unsigned>(E * 2 * A.list_cap);
    {
        const double w = std::max(0.1, 2.0 * (c->dc.dr_clean + 1e-3));
        A.cell_ne = int(std::ceil(2.0 * kCellEta / w));
        A.cell_np = std::max(1, int(std::floor(2.0 * kPi / w)));
        A.cell_we = float(w);
        A.cell_wp = float(2.0 * kPi / A.cell_np);
    }
    const size_t NC = (size_t)A.cell_ne * A.cell_np;
    A.cell_cnt = b.take<int>(E * 2 * NC);
    A.cell_idx = b.take<int>(E * 2 * NC * kCellSlots);
    A.ovf_cnt = b.take<int>(E * 2);
    A.ovf_idx = b.take<int>(E * 2 * A.list_cap);
    A.tc_cap = K.tc_per_event;
    A.tc_cnt = b.take<int>(E);
    const size_t TC = E * K.tc_per_event;
    A.tc_type = b.take<int>(TC); A.tc_seed = b.take<int>(TC); A.tc_obj = b.take<int>(TC);
    A.tc_hits = b.take<int>(10 * TC);
    A.tc_pt = b.take<float>(TC); A.tc_eta = b.take<float>(TC); A.tc_phi = b.take<float>(TC);
    for (auto& sl : c->slot) {
        sl.rec = b.take<TcRec>(TC);
        sl.off = b.take<int>(E + 1);
        sl.stats = b.take<int>(E * kSlotStats);
    }
}

lst_status lst_load_geometry(lst_ctx* c, const lst_module* mods, int32_t n_mod, const int32_t* conn_off,
                             const int32_t* conn_tgt, const int32_t* sb_off, const int32_t* sb_tgt, int32_t n_sb) {
    if (!c || !mods || n_mod <= 0 || !conn_off || !sb_off || n_sb <= 0) return LST_ERR_ARG;
    if (n_sb != c->cfg.sb_n_eta * c->cfg.sb_n_phi * 2) return LST_ERR_ARG;
    const int n_conn = conn_off[n_mod], n_sbt = sb_off[n_sb];
    if (n_conn < 0 || n_sbt < 0 || (n_conn && !conn_tgt) || (n_sbt && !sb_tgt)) return LST_ERR_ARG;
    for (int i = 0; i < n_conn; ++i)
        if (conn_tgt[i] < 0 || conn_tgt[i] >= n_mod) return LST_ERR_ARG;
    for (int i = 0; i < n_sbt; ++i)
        if (sb_tgt[i] < 0 || sb_tgt[i] >= n_mod) return LST_ERR_ARG;
    int max_sbt = 0;
    for (int i = 0; i < n_sb; ++i) {
        if (sb_off[i + 1] < sb_off[i] || sb_off[0] != 0) return LST_ERR_ARG;
        max_sbt = std::max(max_sbt, sb_off[i + 1] - sb_off[i]);
    }
    for (int i = 0; i < n_mod; ++i)
        if (conn_off[i + 1] < conn_off[i] || conn_off[0] != 0) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (c->dev_mem) {
        cudaEventSynchronize(c->done);
        cudaFree(c->dev_mem);
        c->dev_mem = nullptr;
    }
    Buffer probe;
    layout(c, probe, n_mod, n_conn, n_sb, n_sbt, max_sbt);
    if (cudaMalloc(&c->dev_mem, probe.used) != cudaSuccess) {
        c->dev_mem = nullptr;
        c->geometry = false;
        return LST_ERR_OOM;
    }
    c->dev_bytes = probe.used;
    Buffer real;
    real.base = c->dev_mem;
    real.size = probe.used;
    layout(c, real, n_mod, n_conn, n_sb, n_sbt, max_sbt);
    std::vector<float4> m4(n_mod);
    for (int i = 0; i < n_mod; ++i)
        m4[i] = make_float4(mods[i].dsep, mods[i].sig_rphi, mods[i].sig_long, float(mods[i].subdet));
    CK(cudaMemcpy((void*)c->A.mod, m4.data(), sizeof(float4) * n_mod, cudaMemcpyHostToDevice));
    std::vector<int> lay(n_mod);
    for (int i = 0; i < n_mod; ++i) lay[i] = mods[i].layer;
    CK(cudaMemcpy((void*)c->A.mod_layer, lay.data(), sizeof(int) * n_mod, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)c->A.conn_off, conn_off, sizeof(int) * (n_mod + 1), cudaMemcpyHostToDevice));
    if (n_conn) CK(cudaMemcpy((void*)c->A.conn_tgt, conn_tgt, sizeof(int) * n_conn, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)c->A.sb_off, sb_off, sizeof(int) * (n_sb + 1), cudaMemcpyHostToDevice));
    if (n_sbt) CK(cudaMemcpy((void*)c->A.sb_tgt, sb_tgt, sizeof(int) * n_sbt, cudaMemcpyHostToDevice));
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->geometry = true;
    c->ran = false;
    for (auto& sl : c->slot) {      // the results lived in the freed allocation
        sl.gen = 0;
        sl.n_ev = 0;
        sl.held = 0;
        sl.released.clear();
    }
    c->last = -1;
    return LST_OK;
}


// The launch sequence of one batch (Fig. KernelFlow order). Grids are fixed
// per context (grid-stride loops read the batch shape from the descriptor),
// so the sequence can be captured once into a CUDA graph.
static int grid_of(const lst_ctx* c, int id) {
    const LaunchInfo& k = kLaunch[id];
    const int m = c->tune[id].bpsm > 0 ? c->tune[id].bpsm : k.bpsm;
    return c->n_sm * m;
}

static int block_of(const lst_ctx* c, int id) {
    const LaunchInfo& k = kLaunch[id];
    return (k.generic && c->tune[id].block > 0) ? c->tune[id].block : k.block;
}

// One launch of the chain; with pdl, the kernel may be scheduled while its
// predecessor drains (every kernel starts with pdl_begin()).
extern "C++" template <typename... KArgs, typename... Args>
void run_k(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, bool pdl,
                  Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// The launch sequence. With `side` (graph capture), pLS and the pT3 search
// run on a second branch: pLS and the pT plan after the reset, the pT3 search
// and refine once T3 exist; the main branch joins them before pT5 and before
// the cleaning. Without it everything is one stream in the listed order.
static void enqueue_chain(lst_ctx* c, cudaStream_t st, bool profile, cudaStream_t side = nullptr) {
    const Arena& A = c->A;
    const bool pdl = !profile;     // profiling events between launches would serialise them anyway
    const DevCfg& dc = c->dc;
    int L = 0;
#define GB(ID) grid_of(c, ID), block_of(c, ID)
#define LAUNCH(ID, ...)                                                                \
    do {                                                                               \
        if (profile && L < lst_ctx::kMaxProf) {                                        \
            c->prof_name[L] = kLaunch[ID].name;                                        \
            c->prof_id[L] = ID;                                                        \
            cudaEventRecord(c->prof_ev[2 * L], st);                                    \
        }                                                                              \
        __VA_ARGS__;                                                                   \
        if (profile && L < lst_ctx::kMaxProf) cudaEventRecord(c->prof_ev[2 * L + 1], st); \
        ++L;                                                                           \
    } while (0)
    LAUNCH(L_RESET, run_k(k_reset, GB(L_RESET), 0, st, pdl, A));
    if (side) {
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(side, c->ev_fork, 0);
        LAUNCH(L_PLS, run_k(k_pls, GB(L_PLS), 0, side, false, A, dc));
        LAUNCH(L_PT_PLAN, run_k(k_pt_plan, GB(L_PT_PLAN), 0, side, pdl, A));
        cudaEventRecord(c->ev_plan, side);
    }
    LAUNCH(L_BIN_COUNT, run_k(k_bin_count, GB(L_BIN_COUNT), 0, st, pdl, A));
    LAUNCH(L_BIN_SCAN, run_k(k_bin_scan, A.max_events, 1024, 0, st, pdl, A));
    LAUNCH(L_BIN_SCATTER, run_k(k_bin_scatter, GB(L_BIN_SCATTER), 0, st, pdl, A));
    LAUNCH(L_BIN_SORT, run_k(k_bin_sort, GB(L_BIN_SORT), 0, st, pdl, A));
    LAUNCH(L_MD_PLAN, run_k(k_md_plan, GB(L_MD_PLAN), 0, st, pdl, A));
    LAUNCH(L_MD, run_k(k_md_search, GB(L_MD), 0, st, pdl, A, dc));
    LAUNCH(L_MD_WRITE, run_k(k_md_write, GB(L_MD_WRITE), 0, st, pdl, A, dc));
    LAUNCH(L_LS, run_k(k_ls, GB(L_LS), 0, st, pdl, A, dc));
    LAUNCH(L_T3, run_k(k_t3, GB(L_T3), 0, st, pdl, A, dc));
    if (side) {
        cudaEventRecord(c->ev_t3, st);
        cudaStreamWaitEvent(side, c->ev_t3, 0);
        LAUNCH(L_T3_ORDER, run_k(k_t3_order, GB(L_T3_ORDER), 0, side, false, A));
        LAUNCH(L_PT3, run_k(k_pt3, GB(L_PT3), 0, side, pdl, A, dc));
        LAUNCH(L_PT3_REFINE, run_k(k_pt3_refine, GB(L_PT3_REFINE), 0, side, pdl, A, dc));
        cudaEventRecord(c->ev_pt3, side);
    }
    // the learned triplet selection gates the T5 search only, so the pT3 branch starts at once
    if (c->t3_capture) LAUNCH(L_T3_FEAT, run_k(k_t3_features, GB(L_T3_FEAT), 0, st, side ? false : pdl, A, dc));
    if (c->mlp3)
        LAUNCH(L_T3_SCORE, run_k(k_t3_score, GB(L_T3_SCORE), 0, st, side && !c->t3_capture ? false : pdl, A, dc,
                                 lst_mlp_device_params(c->mlp3)));
    LAUNCH(L_T5_PLAN, run_k(k_t5_plan, GB(L_T5_PLAN), t5_plan_smem_bytes(A.max_events), st, pdl, A));
    LAUNCH(L_T5, run_k(k_t5, GB(L_T5), 0, st, pdl, A, dc));
    LAUNCH(L_T5_GATHER, run_k(k_t5_gather, GB(L_T5_GATHER), 0, st, pdl, A));
    LAUNCH(L_T5_REFINE, run_k(k_t5_refine, GB(L_T5_REFINE), 0, st, pdl, A, dc));
    if (c->mlp) {
        LAUNCH(L_T5_MLP, run_k(k_mlp_forward, GB(L_T5_MLP), 0, st, pdl, lst_mlp_device_params(c->mlp), A.t5_feat,
                               A.t5_cap, A.counters + 3, A.t5_mlp, MlpSaved{}));
        LAUNCH(L_T5_MLP_SELECT, run_k(k_t5_mlp_select, GB(L_T5_MLP_SELECT), 0, st, pdl, A, dc));
    }
    if (side) {
        cudaStreamWaitEvent(st, c->ev_plan, 0);
    } else {
        LAUNCH(L_PLS, run_k(k_pls, GB(L_PLS), 0, st, pdl, A, dc));
        LAUNCH(L_PT_PLAN, run_k(k_pt_plan, GB(L_PT_PLAN), 0, st, pdl, A));
    }
    LAUNCH(L_PT5, run_k(k_pt5, GB(L_PT5), 0, st, side ? false : pdl, A, dc));
    LAUNCH(L_PT5_REFINE, run_k(k_pt5_refine, GB(L_PT5_REFINE), 0, st, pdl, A, dc));
    if (side) {
        cudaStreamWaitEvent(st, c->ev_pt3, 0);
    } else {
        LAUNCH(L_T3_ORDER, run_k(k_t3_order, GB(L_T3_ORDER), 0, st, pdl, A));
        LAUNCH(L_PT3, run_k(k_pt3, GB(L_PT3), 0, st, pdl, A, dc));
        LAUNCH(L_PT3_REFINE, run_k(k_pt3_refine, GB(L_PT3_REFINE), 0, st, pdl, A, dc));
    }
    LAUNCH(L_CLEAN_KEYS, run_k(k_clean_keys, GB(L_CLEAN_KEYS), 0, st, side ? false : pdl, A, 0));
    LAUNCH(L_CLEAN_KEEP, run_k(k_clean_keys, GB(L_CLEAN_KEEP), 0, st, pdl, A, 1));
    LAUNCH(L_CLEAN_PT5, run_k(k_clean_pt5, GB(L_CLEAN_PT5), 0, st, pdl, A));
    LAUNCH(L_CLEAN_PT3_CROSS, run_k(k_clean_pt3_cross, GB(L_CLEAN_PT3_CROSS), 0, st, pdl, A, dc));
    LAUNCH(L_CLEAN_PT3_MARK, run_k(k_clean_pt3_mark, GB(L_CLEAN_PT3_MARK), 0, st, pdl, A));
    LAUNCH(L_CLEAN_T5, run_k(k_clean_t5, GB(L_CLEAN_T5), 0, st, pdl, A, dc));
    LAUNCH(L_CLEAN_PLS, run_k(k_clean_pls, GB(L_CLEAN_PLS), 0, st, pdl, A, dc));
    LAUNCH(L_TC_PACK, run_k(k_tc_pack, GB(L_TC_PACK), 0, st, pdl, A));
#undef LAUNCH
#undef GB
    c->launches = L;
}

// Offsets and descriptor are in the pinned staging (h_offsets, h_bd); copy
// them, launch the chain (captured graph, or direct launches when profiling)
// and record the completion event.
// A slot for the next batch: the free one (no held events) that has gone
// longest without a batch; -1 when every slot is held.
static int free_slot(const lst_ctx* c) {
    int best = -1;
    for (int k = 0; k < LST_RESULT_SLOTS; ++k)
        if (c->slot[k].held == 0 && (best < 0 || c->slot[k].gen < c->slot[best].gen)) best = k;
    return best;
}

static lst_event_id make_id(uint32_t gen, int k, int e) {
    return (lst_event_id)(((uint64_t)gen << 32) | ((uint64_t)k << 24) | (uint64_t)e);
}

static lst_status launch_prepared(lst_ctx* c, cudaStream_t st, int n_ev, int k, lst_event_id* ids) {
    lst_ctx::Slot& sl = c->slot[k];
    c->h_bd->out_rec = sl.rec;
    c->h_bd->out_off = sl.off;
    c->h_bd->out_stats = sl.stats;
    CK(cudaMemcpyAsync(c->d_hit_off, c->h_offsets, sizeof(int) * (n_ev + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_seed_off, c->h_offsets + n_ev + 1, sizeof(int) * (n_ev + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_bd, c->h_bd, sizeof(BatchDesc), cudaMemcpyHostToDevice, st));
    if (c->profiling || !c->use_graph) {
        enqueue_chain(c, st, c->profiling);
        CK(cudaGetLastError());
    } else {
        if (!c->graph) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            enqueue_chain(c, c->cap_stream, false, c->side_stream);
            cudaError_t e1 = cudaStreamEndCapture(c->cap_stream, &g);
            if (e1 != cudaSuccess) return LST_ERR_CUDA;
            cudaError_t e2 = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (e2 != cudaSuccess) {
                c->graph = nullptr;
                return LST_ERR_CUDA;
            }
        }
        CK(cudaGraphLaunch(c->graph, st));
    }
    CK(cudaEventRecord(c->done, st));
    CK(cudaEventRecord(sl.done, st));
    c->ran = true;
    sl.gen = c->next_gen++;
    if (c->next_gen == 0) c->next_gen = 1;
    sl.n_ev = n_ev;
    sl.held = ids ? n_ev : 0;
    sl.released.assign(n_ev, 0);
    c->last = k;
    if (ids)
        for (int e = 0; e < n_ev; ++e) ids[e] = make_id(sl.gen, k, e);
    return LST_OK;
}

// Host copies of the batch's offsets (before the staging is overwritten, the
// previous batch must have finished: the pinned staging is reused).
static void set_offsets(lst_ctx* c, const int32_t* hit_off, const int32_t* seed_off, int n_ev) {
    c->n_ev = n_ev;
    c->hit_off_host.assign(hit_off, hit_off + n_ev + 1);
    c->seed_off_host.assign(seed_off, seed_off + n_ev + 1);
    std::memcpy(c->h_offsets, hit_off, sizeof(int) * (n_ev + 1));
    std::memcpy(c->h_offsets + n_ev + 1, seed_off, sizeof(int) * (n_ev + 1));
}

static void use_staging(lst_ctx* c, BatchDesc& d) {
    d.hx = c->in_x; d.hy = c->in_y; d.hz = c->in_z; d.hmod = c->in_mod; d.hside = c->in_side;
    d.seeds = c->in_seeds;
}

lst_status lst_run_batch(lst_ctx* c, const lst_hits* hits, const int32_t* hit_off, const lst_seeds* seeds,
                         const int32_t* seed_off, int32_t n_ev, int32_t mem_is_device, void* stream_,
                         lst_event_id* ids) {
    if (!c) return LST_ERR_ARG;
    if (!c->geometry) return LST_ERR_NO_GEOMETRY;
    if (!hits || !hit_off || !seeds || !seed_off || n_ev <= 0) return LST_ERR_ARG;
    if (n_ev > c->cap.max_events || hits->n > c->cap.max_hits || seeds->n > c->cap.max_seeds) return LST_ERR_CAPACITY;
    if (hits->n < 0 || seeds->n < 0 || hit_off[0] != 0 || seed_off[0] != 0 || hit_off[n_ev] != hits->n ||
        seed_off[n_ev] != seeds->n)
        return LST_ERR_ARG;
    for (int e = 0; e < n_ev; ++e)
        if (hit_off[e + 1] < hit_off[e] || seed_off[e + 1] < seed_off[e]) return LST_ERR_ARG;
    if ((hits->n && (!hits->x || !hits->y || !hits->z || !hits->module || !hits->side)) || (seeds->n && !seeds->xyz))
        return LST_ERR_ARG;
    const int k = free_slot(c);
    if (k < 0) return LST_ERR_CAPACITY;              // every result slot is held: release events first
    CK(cudaSetDevice(c->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream_);
    if (c->ran) CK(cudaEventSynchronize(c->done));   // the pinned staging is reused
    set_offsets(c, hit_off, seed_off, n_ev);
    const size_t H = hits->n, S = seeds->n;
    BatchDesc& d = *c->h_bd;
    d.n_ev = n_ev;
    d.n_hits = (int)H;
    d.n_seeds = (int)S;
    if (mem_is_device) {
        d.hx = hits->x; d.hy = hits->y; d.hz = hits->z; d.hmod = hits->module; d.hside = hits->side;
        d.seeds = seeds->xyz;
    } else {
        if (H) {
            CK(cudaMemcpyAsync(c->in_x, hits->x, 4 * H, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(c->in_y, hits->y, 4 * H, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(c->in_z, hits->z, 4 * H, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(c->in_mod, hits->module, 4 * H, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(c->in_side, hits->side, H, cudaMemcpyHostToDevice, st));
        }
        if (S) CK(cudaMemcpyAsync(c->in_seeds, seeds->xyz, 36 * S, cudaMemcpyHostToDevice, st));
        use_staging(c, d);
    }
    return launch_prepared(c, st, n_ev, k, ids);
}

lst_status lst_run_events(lst_ctx* c, const lst_hits* hits, const lst_seeds* seeds, int32_t n_ev,
                          int32_t mem_is_device, void* stream_, lst_event_id* ids) {
    if (!c) return LST_ERR_ARG;
    if (!c->geometry) return LST_ERR_NO_GEOMETRY;
    if (!hits || !seeds || n_ev <= 0) return LST_ERR_ARG;
    if (n_ev > c->cap.max_events) return LST_ERR_CAPACITY;
    std::vector<int32_t> ho(n_ev + 1, 0), so(n_ev + 1, 0);
    for (int e = 0; e < n_ev; ++e) {
        const lst_hits& h = hits[e];
        const lst_seeds& q = seeds[e];
        if (h.n < 0 || q.n < 0) return LST_ERR_ARG;
        if ((h.n && (!h.x || !h.y || !h.z || !h.module || !h.side)) || (q.n && !q.xyz)) return LST_ERR_ARG;
        ho[e + 1] = ho[e] + h.n;
        so[e + 1] = so[e] + q.n;
        if (ho[e + 1] > c->cap.max_hits || so[e + 1] > c->cap.max_seeds) return LST_ERR_CAPACITY;
    }
    const int k = free_slot(c);
    if (k < 0) return LST_ERR_CAPACITY;
    CK(cudaSetDevice(c->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream_);
    if (c->ran) CK(cudaEventSynchronize(c->done));
    set_offsets(c, ho.data(), so.data(), n_ev);
    const cudaMemcpyKind kind = mem_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int e = 0; e < n_ev; ++e) {
        const lst_hits& h = hits[e];
        const size_t o = ho[e], n = h.n;
        if (n) {
            CK(cudaMemcpyAsync(c->in_x + o, h.x, 4 * n, kind, st));
            CK(cudaMemcpyAsync(c->in_y + o, h.y, 4 * n, kind, st));
            CK(cudaMemcpyAsync(c->in_z + o, h.z, 4 * n, kind, st));
            CK(cudaMemcpyAsync(c->in_mod + o, h.module, 4 * n, kind, st));
            CK(cudaMemcpyAsync(c->in_side + o, h.side, n, kind, st));
        }
        if (seeds[e].n) CK(cudaMemcpyAsync(c->in_seeds + 9 * (size_t)so[e], seeds[e].xyz, 36 * (size_t)seeds[e].n, kind, st));
    }
    BatchDesc& d = *c->h_bd;
    d.n_ev = n_ev;
    d.n_hits = ho[n_ev];
    d.n_seeds = so[n_ev];
    use_staging(c, d);
    return launch_prepared(c, st, n_ev, k, ids);
}

lst_status lst_run_event(lst_ctx* c, const lst_hits* hits, const lst_seeds* seeds, int32_t mem_is_device,
                         void* stream, lst_event_id* id) {
    if (!hits || !seeds) return LST_ERR_ARG;
    int32_t ho[2] = {0, hits->n}, so[2] = {0, seeds->n};
    return lst_run_batch(c, hits, ho, seeds, so, 1, mem_is_device, stream, id);
}

lst_status lst_release_event(lst_ctx* c, lst_event_id id) {
    if (!c || id < 0 || (id >> 32) == 0) return LST_ERR_ARG;
    const uint32_t gen = (uint32_t)((uint64_t)id >> 32);
    const int k = (int)(((uint64_t)id >> 24) & 0xff), e = (int)(id & 0xffffff);
    if (k >= LST_RESULT_SLOTS) return LST_ERR_ARG;
    lst_ctx::Slot& sl = c->slot[k];
    if (sl.gen != gen || sl.held == 0 || e >= sl.n_ev || sl.released[e]) return LST_ERR_ARG;
    sl.released[e] = 1;
    --sl.held;
    return LST_OK;
}

int32_t lst_last_launch_count(lst_ctx* c) { return c ? c->launches : 0; }

int32_t lst_query(lst_ctx* c) {
    if (!c) return LST_ERR_ARG;
    if (!c->ran) return 0;
    if (cudaSetDevice(c->device) != cudaSuccess) return LST_ERR_CUDA;
    cudaError_t e = cudaEventQuery(c->done);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return LST_ERR_CUDA;
}

int64_t lst_device_bytes(lst_ctx* c) { return c ? (int64_t)c->dev_bytes : 0; }

lst_status lst_set_profiling(lst_ctx* c, int32_t enable) {
    if (!c) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (enable && !c->prof_ev[0])
        for (cudaEvent_t& e : c->prof_ev) CK(cudaEventCreate(&e));
    if (c->ran) CK(cudaEventSynchronize(c->done));
    c->profiling = enable != 0;
    return LST_OK;
}

lst_status lst_get_kernel_times(lst_ctx* c, int32_t capacity, int32_t* n_out, const char** names, float* ms) {
    if (!c || capacity < 0) return LST_ERR_ARG;
    if (!c->ran || !c->profiling) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(c->done));
    const int n = std::min(c->launches, (int)lst_ctx::kMaxProf);
    if (n_out) *n_out = n;
    for (int i = 0; i < std::min(n, (int)capacity); ++i) {
        if (names) names[i] = c->prof_name[i];
        if (ms) CK(cudaEventElapsedTime(ms + i, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
    }
    return n > capacity ? LST_WARN_TRUNCATED : LST_OK;
}

static const void* launch_fn(int id) {
    switch (id) {
        case L_RESET: return (const void*)k_reset;
        case L_BIN_COUNT: return (const void*)k_bin_count;
        case L_BIN_SCAN: return (const void*)k_bin_scan;
        case L_BIN_SCATTER: return (const void*)k_bin_scatter;
        case L_BIN_SORT: return (const void*)k_bin_sort;
        case L_MD_PLAN: return (const void*)k_md_plan;
        case L_MD: return (const void*)k_md_search;
        case L_MD_WRITE: return (const void*)k_md_write;
        case L_LS: return (const void*)k_ls;
        case L_T3: return (const void*)k_t3;
        case L_T5: return (const void*)k_t5;
        case L_T5_PLAN: return (const void*)k_t5_plan;
        case L_T5_GATHER: return (const void*)k_t5_gather;
        case L_T5_REFINE: return (const void*)k_t5_refine;
        case L_T3_FEAT: return (const void*)k_t3_features;
        case L_T3_SCORE: return (const void*)k_t3_score;
        case L_T5_MLP: return (const void*)k_mlp_forward;
        case L_T5_MLP_SELECT: return (const void*)k_t5_mlp_select;
        case L_PLS: return (const void*)k_pls;
        case L_PT_PLAN: return (const void*)k_pt_plan;
        case L_T3_ORDER: return (const void*)k_t3_order;
        case L_PT5: return (const void*)k_pt5;
        case L_PT5_REFINE: return (const void*)k_pt5_refine;
        case L_PT3: return (const void*)k_pt3;
        case L_PT3_REFINE: return (const void*)k_pt3_refine;
        case L_CLEAN_KEYS: case L_CLEAN_KEEP: return (const void*)k_clean_keys;
        case L_CLEAN_PT5: return (const void*)k_clean_pt5;
        case L_CLEAN_PT3_CROSS: return (const void*)k_clean_pt3_cross;
        case L_CLEAN_PT3_MARK: return (const void*)k_clean_pt3_mark;
        case L_CLEAN_T5: return (const void*)k_clean_t5;
        case L_CLEAN_PLS: return (const void*)k_clean_pls;
        case L_TC_PACK: return (const void*)k_tc_pack;
        default: return nullptr;
    }
}

// Is (blocks per SM, block) a valid shape for the stage? 0 keeps the default.
static lst_status check_shape(int id, int bpsm, int block) {
    if (id < 0 || id >= kNumLaunch || bpsm < 0 || bpsm > 64 || block < 0) return LST_ERR_ARG;
    const LaunchInfo& k = kLaunch[id];
    if (bpsm && !k.tunable) return LST_ERR_ARG;
    if (block) {
        if (!k.generic || block % 32 || block > 1024) return LST_ERR_ARG;
        cudaFuncAttributes fa{};
        CK(cudaFuncGetAttributes(&fa, launch_fn(id)));
        if (block > fa.maxThreadsPerBlock) return LST_ERR_ARG;
    }
    return LST_OK;
}

static lst_status drop_graph(lst_ctx* c) {
    if (c->ran) CK(cudaEventSynchronize(c->done));
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return LST_OK;
}

lst_status lst_set_compact_storage(lst_ctx* c, int32_t enable) {
    if (!c || enable < 0 || enable > 1) return LST_ERR_ARG;
    lst_status s = drop_graph(c);
    c->A.compact = enable;
    return s;
}

lst_status lst_set_fp64_fit(lst_ctx* c, int32_t enable) {
    if (!c || enable < 0 || enable > 1) return LST_ERR_ARG;
    lst_status s = drop_graph(c);
    c->dc.fp64_fit = enable;
    return s;
}

lst_status lst_set_stage_limits(lst_ctx* c, int32_t t5, int32_t pt) {
    if (!c || t5 < 0 || t5 > kT5Stage || pt < 0 || pt > kPtStage) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    lst_status s = drop_graph(c);
    if (s != LST_OK) return s;
    c->dc.t5_stage = t5 > 0 ? t5 : kT5Stage;
    c->dc.pt_stage = pt > 0 ? pt : kPtStage;
    return LST_OK;
}

int32_t lst_launch_stage_count(void) { return kNumLaunch; }

lst_status lst_get_launch_config(lst_ctx* c, int32_t stage, const char** name, int32_t* blocks_per_sm,
                                 int32_t* block, int32_t* flags) {
    if (!c || stage < 0 || stage >= kNumLaunch) return LST_ERR_ARG;
    const LaunchInfo& k = kLaunch[stage];
    if (name) *name = k.name;
    if (blocks_per_sm) *blocks_per_sm = k.tunable ? (c->tune[stage].bpsm > 0 ? c->tune[stage].bpsm : k.bpsm) : 0;
    if (block) *block = block_of(c, stage);
    if (flags) *flags = (k.tunable ? 1 : 0) | (k.generic ? 2 : 0);
    return LST_OK;
}

lst_status lst_set_launch_config(lst_ctx* c, int32_t stage, int32_t blocks_per_sm, int32_t block) {
    if (!c) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    lst_status s = check_shape(stage, blocks_per_sm, block);
    if (s != LST_OK) return s;
    s = drop_graph(c);
    if (s != LST_OK) return s;
    c->tune[stage].bpsm = blocks_per_sm;
    c->tune[stage].block = block;
    return LST_OK;
}

// Median device time of every stage over `reps` profiled runs of the batch.
static lst_status time_stages(lst_ctx* c, const lst_hits* hits, const int32_t* hit_off, const lst_seeds* seeds,
                              const int32_t* seed_off, int32_t n_ev, int32_t mem_is_device, void* stream, int reps,
                              float* med, float* total) {
    std::vector<float> t[kNumLaunch];
    float tot = 0.f;
    for (int r = 0; r < reps; ++r) {
        lst_status s = lst_run_batch(c, hits, hit_off, seeds, seed_off, n_ev, mem_is_device, stream, nullptr);
        if (s != LST_OK) return s;
        CK(cudaEventSynchronize(c->done));
        CK(cudaGetLastError());
        const int n = std::min(c->launches, (int)lst_ctx::kMaxProf);
        for (int i = 0; i < n; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
            t[c->prof_id[i]].push_back(ms);
            tot += ms;
        }
    }
    for (int id = 0; id < kNumLaunch; ++id) {
        auto& v = t[id];
        if (v.empty()) {
            med[id] = 0.f;
            continue;
        }
        std::sort(v.begin(), v.end());
        med[id] = v[v.size() / 2];
    }
    if (total) *total = tot / reps;
    return LST_OK;
}

lst_status lst_autotune(lst_ctx* c, const lst_hits* hits, const int32_t* hit_off, const lst_seeds* seeds,
                        const int32_t* seed_off, int32_t n_ev, int32_t mem_is_device, void* stream, int32_t reps,
                        float* ms_before, float* ms_after) {
    if (!c || reps <= 0 || reps > 64) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    const bool was_profiling = c->profiling;
    lst_status s = lst_set_profiling(c, 1);
    if (s != LST_OK) return s;
    LaunchCfg start[kNumLaunch], best_cfg[kNumLaunch];
    float best[kNumLaunch], med[kNumLaunch];
    std::copy(c->tune, c->tune + kNumLaunch, start);
    std::copy(c->tune, c->tune + kNumLaunch, best_cfg);
    float t0 = 0.f;
    s = time_stages(c, hits, hit_off, seeds, seed_off, n_ev, mem_is_device, stream, reps, best, &t0);
    static const int kBpsm[] = {1, 2, 3, 4, 6, 8, 12, 16};
    static const int kBlock[] = {0, 64, 128, 256, 512};
    for (int bi = 0; s == LST_OK && bi < (int)(sizeof(kBlock) / sizeof(int)); ++bi) {
        for (int m : kBpsm) {
            const int b = kBlock[bi];
            if (b * m > 4096) continue;
            bool any = false;
            for (int id = 0; id < kNumLaunch; ++id) {
                c->tune[id] = start[id];
                if (!kLaunch[id].tunable || (b && !kLaunch[id].generic)) continue;
                if (check_shape(id, m, b) != LST_OK) continue;
                c->tune[id] = LaunchCfg{m, b};
                any = true;
            }
            if (!any) continue;
            s = time_stages(c, hits, hit_off, seeds, seed_off, n_ev, mem_is_device, stream, reps, med, nullptr);
            if (s != LST_OK) break;
            for (int id = 0; id < kNumLaunch; ++id) {
                const LaunchCfg& t = c->tune[id];
                if (t.bpsm != m || t.block != b || med[id] <= 0.f) continue;
                if (med[id] < best[id]) {
                    best[id] = med[id];
                    best_cfg[id] = t;
                }
            }
        }
    }
    std::copy(s == LST_OK ? best_cfg : start, (s == LST_OK ? best_cfg : start) + kNumLaunch, c->tune);
    float t1 = 0.f;
    if (s == LST_OK && ms_after)
        s = time_stages(c, hits, hit_off, seeds, seed_off, n_ev, mem_is_device, stream, reps, med, &t1);
    lst_status s2 = lst_set_profiling(c, was_profiling ? 1 : 0);
    lst_status s3 = drop_graph(c);
    if (ms_before) *ms_before = t0;
    if (ms_after) *ms_after = t1;
    if (s != LST_OK) return s;
    return s2 != LST_OK ? s2 : s3;
}

// The slot k and event e of `id`: a handle of a held batch, or an event index
// (0 <= id < n_events) of the last batch. Waits for that batch.
static lst_status resolve(lst_ctx* c, lst_event_id id, int& k, int& e) {
    if (!c || !c->ran || c->last < 0 || id < 0) return LST_ERR_ARG;
    if ((id >> 32) == 0) {
        k = c->last;
        e = (int)id;
        if (e >= c->slot[k].n_ev) return LST_ERR_ARG;
    } else {
        const uint32_t gen = (uint32_t)((uint64_t)id >> 32);
        k = (int)(((uint64_t)id >> 24) & 0xff);
        e = (int)(id & 0xffffff);
        if (k >= LST_RESULT_SLOTS) return LST_ERR_ARG;
        const lst_ctx::Slot& sl = c->slot[k];
        if (sl.gen != gen || sl.held == 0 || e >= sl.n_ev || sl.released[e]) return LST_ERR_ARG;
    }
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(c->slot[k].done));
    CK(cudaGetLastError());
    return LST_OK;
}

// As resolve, for the intermediate objects: only the last batch has them.
static lst_status wait_batch(lst_ctx* c, lst_event_id id, int32_t& event) {
    int k = 0, e = 0;
    lst_status s = resolve(c, id, k, e);
    if (s != LST_OK) return s;
    if (k != c->last) return LST_ERR_ARG;
    CK(cudaEventSynchronize(c->done));
    event = e;
    return LST_OK;
}


#define FETCH(v, d, n)                          \
    do {                                        \
        lst_status s__ = fetch(v, d, n);        \
        if (s__ != LST_OK) return s__;          \
    } while (0)

lst_status lst_set_t5_selection(lst_ctx* c, const lst_mlp* mlp, float threshold, float prefilter_scale,
                                int32_t capture_features) {
    if (!c || !(prefilter_scale >= 1.0f)) return LST_ERR_ARG;
    if (c->ran) CK(cudaEventSynchronize(c->done));
    c->mlp = mlp;
    c->dc.use_mlp = mlp ? 1 : 0;
    c->dc.features_on = (mlp || capture_features) ? 1 : 0;
    c->dc.prefit_scale = prefilter_scale;
    c->dc.mlp_threshold = threshold;
    derive_fp32(c->dc);
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return LST_OK;
}

lst_status lst_set_t3_selection(lst_ctx* c, const lst_mlp* mlp, float threshold, int32_t capture_features) {
    if (!c) return LST_ERR_ARG;
    if (!c->geometry) return LST_ERR_NO_GEOMETRY;
    if (c->ran) CK(cudaEventSynchronize(c->done));
    const bool feat = mlp || capture_features;
    if (feat && !c->t3_mem) {
        const size_t T3 = (size_t)c->A.t3_cap;
        const size_t bytes = T3 * (48 * sizeof(float) + sizeof(float) + 1) + 512;
        CK(cudaSetDevice(c->device));
        if (cudaMalloc(&c->t3_mem, bytes) != cudaSuccess) {
            c->t3_mem = nullptr;
            return LST_ERR_OOM;
        }
        char* p = static_cast<char*>(c->t3_mem);
        c->A.t3_feat = reinterpret_cast<float*>(p);
        c->A.t3_mlp = reinterpret_cast<float*>(p + T3 * 48 * sizeof(float));
        c->A.t3_ok = reinterpret_cast<uint8_t*>(p + T3 * 49 * sizeof(float));
    }
    c->mlp3 = mlp;
    c->t3_features = c->t3_features || feat;
    c->t3_capture = capture_features != 0;
    c->A.t3_sel = mlp ? 1 : 0;
    c->dc.t3_threshold = threshold;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return LST_OK;
}

lst_status lst_get_t3_candidates(lst_ctx* c, lst_event_id id, int32_t capacity, int32_t* n_out, float* features,
                                 int32_t* hits, float* score, int32_t* kept) {
    int32_t event = 0;
    lst_status s = wait_batch(c, id, event);
    if (s != LST_OK) return s;
    if (capacity < 0) return LST_ERR_ARG;
    const Arena& A = c->A;
    int cnt[32];
    CK(cudaMemcpy(cnt, A.counters, sizeof cnt, cudaMemcpyDeviceToHost));
    const int n = std::min(cnt[2], A.t3_cap), n_md = std::min(cnt[0], A.md_cap);
    std::vector<int4> t3md;
    std::vector<int> gm, lo, up;
    FETCH(t3md, A.t3_md, n);
    FETCH(gm, A.md_gmod, n_md); FETCH(lo, A.md_lo, n_md); FETCH(up, A.md_up, n_md);
    std::vector<int> rows;
    for (int i = 0; i < n; ++i)
        if (gm[t3md[i].x] / A.n_mod == event) rows.push_back(i);
    const int k = std::min((int)rows.size(), (int)capacity);
    if (n_out) *n_out = (int)rows.size();
    if (features && k) {
        if (!c->t3_capture) return LST_ERR_ARG;
        std::vector<float> f;
        FETCH(f, A.t3_feat, (size_t)48 * n);
        for (int r = 0; r < k; ++r) std::memcpy(features + 48 * (size_t)r, f.data() + 48 * (size_t)rows[r], 48 * 4);
    }
    if (score && k) {
        if (!c->mlp3) return LST_ERR_ARG;
        std::vector<float> sc;
        FETCH(sc, A.t3_mlp, n);
        for (int r = 0; r < k; ++r) score[r] = sc[rows[r]];
    }
    if (kept && k) {
        std::vector<uint8_t> ok;
        if (c->mlp3) FETCH(ok, A.t3_ok, n);
        for (int r = 0; r < k; ++r) kept[r] = c->mlp3 ? ok[rows[r]] : 1;
    }
    if (hits)
        for (int r = 0; r < k; ++r) {
            const int4 q = t3md[rows[r]];
            const int md[3] = {q.x, q.y, q.z};
            for (int j = 0; j < 3; ++j) {
                hits[6 * r + 2 * j] = lo[md[j]];
                hits[6 * r + 2 * j + 1] = up[md[j]];
            }
        }
    return (int)rows.size() > capacity ? LST_WARN_TRUNCATED : LST_OK;
}

lst_status lst_get_t5_candidates(lst_ctx* c, lst_event_id id, int32_t capacity, int32_t* n_out, float* features,
                                 int32_t* hits, int32_t* cut_pass, float* score) {
    int32_t event = 0;
    lst_status s = wait_batch(c, id, event);
    if (s != LST_OK) return s;
    if (capacity < 0) return LST_ERR_ARG;
    const Arena& A = c->A;
    int cnt[32];
    CK(cudaMemcpy(cnt, A.counters, sizeof cnt, cudaMemcpyDeviceToHost));
    const int n = std::min(cnt[3], A.t5_cap);
    const int n_md = std::min(cnt[0], A.md_cap), n_t3 = std::min(cnt[2], A.t3_cap);
    std::vector<int> ti, to, m0, m1, m2, gm, lo, up;
    std::vector<uint8_t> cp;
    std::vector<int4> t3md;
    FETCH(ti, A.t5_in, n); FETCH(to, A.t5_out, n); FETCH(cp, A.t5_cut, n);
    FETCH(t3md, A.t3_md, n_t3);
    for (const int4& q : t3md) {
        m0.push_back(q.x);
        m1.push_back(q.y);
        m2.push_back(q.z);
    }
    FETCH(gm, A.md_gmod, n_md); FETCH(lo, A.md_lo, n_md); FETCH(up, A.md_up, n_md);
    std::vector<int> rows;
    for (int i = 0; i < n; ++i)
        if (gm[m0[ti[i]]] / A.n_mod == event) rows.push_back(i);
    const int k = std::min((int)rows.size(), (int)capacity);
    if (n_out) *n_out = (int)rows.size();
    if (features && k) {
        std::vector<float> f;
        FETCH(f, A.t5_feat, (size_t)48 * n);
        for (int r = 0; r < k; ++r) std::memcpy(features + 48 * (size_t)r, f.data() + 48 * (size_t)rows[r], 48 * 4);
    }
    if (score && k) {
        std::vector<float> sc;
        FETCH(sc, A.t5_mlp, n);
        for (int r = 0; r < k; ++r) score[r] = sc[rows[r]];
    }
    for (int r = 0; r < k; ++r) {
        const int i = rows[r];
        const int md[5] = {m0[ti[i]], m1[ti[i]], m2[ti[i]], m1[to[i]], m2[to[i]]};
        if (hits)
            for (int j = 0; j < 5; ++j) {
                hits[10 * r + 2 * j] = lo[md[j]];
                hits[10 * r + 2 * j + 1] = up[md[j]];
            }
        if (cut_pass) cut_pass[r] = cp[i];
    }
    return (int)rows.size() > capacity ? LST_WARN_TRUNCATED : LST_OK;
}

lst_status lst_get_counters(lst_ctx* c, int32_t* out, int32_t n) {
    if (!c || !out || n < 0 || n > 32) return LST_ERR_ARG;
    if (!c->ran) return LST_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(c->done));
    if (n) CK(cudaMemcpy(out, c->A.counters, sizeof(int) * n, cudaMemcpyDeviceToHost));
    return LST_OK;
}

lst_status lst_get_stats(lst_ctx* c, lst_event_id id, lst_stats* out) {
    int k = 0, e = 0;
    lst_status s = resolve(c, id, k, e);
    if (s != LST_OK) return s;
    if (!out) return LST_ERR_ARG;
    int st[kSlotStats];
    CK(cudaMemcpy(st, c->slot[k].stats + kSlotStats * (size_t)e, sizeof st, cudaMemcpyDeviceToHost));
    for (int j = 0; j < 8; ++j) { out->counts[j] = st[j]; out->dropped[j] = st[8 + j]; }
    out->counts[7] = st[16];
    return LST_OK;
}

static_assert(sizeof(lst_tc) == sizeof(TcRec), "lst_tc mirrors the packed record");

lst_status lst_get_track_candidates(lst_ctx* c, lst_event_id id, int32_t capacity, int32_t* n_out, int32_t* type,
                                    int32_t* seed, int32_t* hits, float* pet) {
    int k = 0, e = 0;
    lst_status s = resolve(c, id, k, e);
    if (s != LST_OK) return s;
    if (capacity < 0) return LST_ERR_ARG;
    int off[2];
    CK(cudaMemcpy(off, c->slot[k].off + e, sizeof off, cudaMemcpyDeviceToHost));
    const int n = off[1] - off[0];
    if (n_out) *n_out = n;
    const int m = std::min(n, (int)capacity);
    if (m > 0 && (type || seed || hits || pet)) {
        std::vector<lst_tc> r(m);
        CK(cudaMemcpy(r.data(), c->slot[k].rec + off[0], sizeof(lst_tc) * (size_t)m, cudaMemcpyDeviceToHost));
        for (int i = 0; i < m; ++i) {
            if (type) type[i] = r[i].type;
            if (seed) seed[i] = r[i].seed;
            if (hits) std::memcpy(hits + 10 * (size_t)i, r[i].hits, sizeof r[i].hits);
            if (pet) { pet[3 * i] = r[i].pt; pet[3 * i + 1] = r[i].eta; pet[3 * i + 2] = r[i].phi0; }
        }
    }
    return n > capacity ? LST_WARN_TRUNCATED : LST_OK;
}

lst_status lst_get_batch_track_candidates(lst_ctx* c, int32_t capacity, int32_t* offsets, lst_tc* out) {
    if (!c || !offsets || capacity < 0 || (capacity > 0 && !out)) return LST_ERR_ARG;
    if (!c->ran || c->last < 0) return LST_ERR_ARG;
    const lst_ctx::Slot& sl = c->slot[c->last];
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(sl.done));
    CK(cudaGetLastError());
    CK(cudaMemcpy(offsets, sl.off, sizeof(int) * (sl.n_ev + 1), cudaMemcpyDeviceToHost));
    const int total = offsets[sl.n_ev];
    const int m = std::min(total, (int)capacity);
    if (m > 0) CK(cudaMemcpy(out, sl.rec, sizeof(lst_tc) * (size_t)m, cudaMemcpyDeviceToHost));
    return total > capacity ? LST_WARN_TRUNCATED : LST_OK;
}

lst_status lst_object_columns(int32_t kind, int32_t* ni, int32_t* nf) {
    static const int NI[] = {3, 2, 2, 2, 3, 2, 2};
    static const int NF[] = {2, 1, 3, 7, 6, 5, 5};
    if (kind < 0 || kind > 6 || !ni || !nf) return LST_ERR_ARG;
    *ni = NI[kind];
    *nf = NF[kind];
    return LST_OK;
}

lst_status lst_get_objects(lst_ctx* c, lst_event_id id, int32_t kind, int32_t capacity, int32_t* n_out, int32_t* I,
                           float* F) {
    int32_t event = 0;
    lst_status s = wait_batch(c, id, event);
    if (s != LST_OK) return s;
    if (kind < 0 || kind > 6 || capacity < 0) return LST_ERR_ARG;
    const Arena& A = c->A;
    int cnt[32];
    CK(cudaMemcpy(cnt, A.counters, sizeof cnt, cudaMemcpyDeviceToHost));
    const int n_md = std::min(cnt[0], A.md_cap), n_ls = std::min(cnt[1], A.ls_cap);
    const int n_t3 = std::min(cnt[2], A.t3_cap), n_t5 = std::min(cnt[3], A.t5_cap);
    const int n_p5 = std::min(cnt[4], A.pt5_cap), n_p3 = std::min(cnt[5], A.pt3_cap);
    std::vector<int> iv;        // rows: ints
    std::vector<float> fv;      // rows: floats
    int ni = 0, nf = 0;
    lst_object_columns(kind, &ni, &nf);
    // MD rows of this event (and their global -> row map) are needed by all kinds but pLS
    std::vector<int> md_row, ls_row, t3_row, t5_row;
    std::vector<int> gmod;
    FETCH(gmod, A.md_gmod, n_md);
    md_row.assign(n_md, -1);
    int r = 0;
    for (int i = 0; i < n_md; ++i)
        if (gmod[i] / A.n_mod == event) md_row[i] = r++;
    const int s0 = c->seed_off_host[event], s1 = c->seed_off_host[event + 1];
    if (kind == 0) {
        std::vector<int> lo, up;
        std::vector<float> dp, dl;
        FETCH(lo, A.md_lo, n_md); FETCH(up, A.md_up, n_md); FETCH(dp, A.md_dphi, n_md); FETCH(dl, A.md_dlong, n_md);
        for (int i = 0; i < n_md; ++i)
            if (md_row[i] >= 0) {
                iv.insert(iv.end(), {lo[i], up[i], gmod[i] % A.n_mod});
                fv.insert(fv.end(), {dp[i], dl[i]});
            }
    }
    std::vector<int> li, lo2;
    if (kind >= 1 && kind != 4) {
        FETCH(li, A.ls_in, n_ls);
        FETCH(lo2, A.ls_out, n_ls);
        ls_row.assign(n_ls, -1);
        r = 0;
        for (int i = 0; i < n_ls; ++i)
            if (md_row[li[i]] >= 0) ls_row[i] = r++;
    }
    if (kind == 1) {
        std::vector<float> dp;
        FETCH(dp, A.ls_dphi, n_ls);
        for (int i = 0; i < n_ls; ++i)
            if (ls_row[i] >= 0) {
                iv.insert(iv.end(), {md_row[li[i]], md_row[lo2[i]]});
                fv.push_back(dp[i]);
            }
    }
    std::vector<int> t3i, t3o;
    if (kind == 2 || kind == 3 || kind == 5 || kind == 6) {
        FETCH(t3i, A.t3_lsin, n_t3);
        FETCH(t3o, A.t3_lsout, n_t3);
        t3_row.assign(n_t3, -1);
        r = 0;
        for (int i = 0; i < n_t3; ++i)
            if (ls_row[t3i[i]] >= 0) t3_row[i] = r++;
    }
    if (kind == 2) {
        std::vector<float> b;
        std::vector<float2> ks;
        FETCH(b, A.t3_beta, n_t3); FETCH(ks, A.t3_ks, n_t3);
        for (int i = 0; i < n_t3; ++i)
            if (t3_row[i] >= 0) {
                iv.insert(iv.end(), {ls_row[t3i[i]], ls_row[t3o[i]]});
                fv.insert(fv.end(), {b[i], ks[i].x, ks[i].y});
            }
    }
    std::vector<int> t5i, t5o;
    if (kind == 3 || kind == 5) {
        FETCH(t5i, A.t5_in, n_t5);
        FETCH(t5o, A.t5_out, n_t5);
        std::vector<uint8_t> v5;
        FETCH(v5, A.t5_valid, n_t5);
        t5_row.assign(n_t5, -1);
        r = 0;
        for (int i = 0; i < n_t5; ++i)
            if (v5[i] && t3_row[t5i[i]] >= 0) t5_row[i] = r++;
    }
    if (kind == 3) {
        std::vector<double> k, et, ph;
        std::vector<float> c2, cz, sc, pt;
        FETCH(k, A.t5_kappa, n_t5); FETCH(et, A.t5_eta, n_t5); FETCH(ph, A.t5_phi, n_t5);
        FETCH(c2, A.t5_chi2, n_t5); FETCH(cz, A.t5_chi2z, n_t5); FETCH(sc, A.t5_score, n_t5); FETCH(pt, A.t5_pt, n_t5);
        for (int i = 0; i < n_t5; ++i)
            if (t5_row[i] >= 0) {
                iv.insert(iv.end(), {t3_row[t5i[i]], t3_row[t5o[i]]});
                fv.insert(fv.end(), {float(k[i]), c2[i], cz[i], float(et[i]), float(ph[i]), pt[i], sc[i]});
            }
    }
    if (kind == 4) {
        int n = s1 - s0;
        std::vector<int> ps, sb;
        std::vector<double> k, sk, et, ph;
        std::vector<float> z0, pt;
        FETCH(ps, A.pls_pass + s0, n); FETCH(sb, A.pls_sb + s0, n);
        FETCH(k, A.pls_kappa + s0, n); FETCH(sk, A.pls_sigk + s0, n); FETCH(et, A.pls_eta + s0, n);
        FETCH(ph, A.pls_phi + s0, n); FETCH(z0, A.pls_z0 + s0, n); FETCH(pt, A.pls_pt + s0, n);
        for (int i = 0; i < n; ++i) {
            iv.insert(iv.end(), {i, ps[i], sb[i]});
            fv.insert(fv.end(), {float(k[i]), float(sk[i]), float(et[i]), float(ph[i]), z0[i], pt[i]});
        }
    }
    if (kind == 5 || kind == 6) {
        const int n = kind == 5 ? n_p5 : n_p3;
        std::vector<int> sd, ob;
        std::vector<uint8_t> vv;
        std::vector<float> k, c2, cz, sc, pt;
        FETCH(vv, kind == 5 ? A.pt5_valid : A.pt3_valid, n);
        FETCH(sd, kind == 5 ? A.pt5_seed : A.pt3_seed, n); FETCH(ob, kind == 5 ? A.pt5_obj : A.pt3_obj, n);
        FETCH(k, kind == 5 ? A.pt5_kappa : A.pt3_kappa, n); FETCH(c2, kind == 5 ? A.pt5_chi2 : A.pt3_chi2, n);
        FETCH(cz, kind == 5 ? A.pt5_chi2z : A.pt3_chi2z, n); FETCH(sc, kind == 5 ? A.pt5_score : A.pt3_score, n);
        FETCH(pt, kind == 5 ? A.pt5_pt : A.pt3_pt, n);
        for (int i = 0; i < n; ++i)
            if (vv[i] && sd[i] >= s0 && sd[i] < s1) {
                iv.insert(iv.end(), {sd[i] - s0, kind == 5 ? t5_row[ob[i]] : t3_row[ob[i]]});
                fv.insert(fv.end(), {k[i], c2[i], cz[i], sc[i], pt[i]});
            }
    }
    const int rows = ni ? (int)(iv.size() / ni) : 0;
    if (n_out) *n_out = rows;
    const int k = std::min(rows, (int)capacity);
    if (I && k) std::memcpy(I, iv.data(), sizeof(int) * ni * (size_t)k);
    if (F && k) std::memcpy(F, fv.data(), sizeof(float) * nf * (size_t)k);
    return rows > capacity ? LST_WARN_TRUNCATED : LST_OK;
}

}  // extern "C"
