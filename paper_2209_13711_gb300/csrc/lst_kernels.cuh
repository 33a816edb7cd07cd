// Kernel declarations and per-unit occupancy bounds of the device chain.
#pragma once

#include "lst_device.cuh"
#include "lst_mlp.cuh"

namespace lst {

// Per-unit stage sizes. MD, LS and T3: the most objects one unit may produce
// (occupancy truncation; excess objects are counted as dropped). T5 and pT:
// shared-memory staging per work item; an item with more survivors is
// enumerated a second time and written directly, so nothing is dropped.
constexpr int kMaxHits = 256;     // hits per sensor of one module
constexpr int kMdStage = 1024;    // MDs per module
constexpr int kLsStage = 256;     // LS per inner MD
constexpr int kT3Stage = 512;     // T3 per inner MD
constexpr int kT5Pre = 256;       // FP32-prefiltered T5 candidates held before an FP64 pass
constexpr int kT5Stage = 512;     // T5 survivors staged per work item (more: the item is enumerated again)
constexpr int kPtPre = 128;       // prefiltered pT3/pT5 candidates held before an FP64 pass
constexpr int kPtStage = 256;     // pT3/pT5 survivors staged per work item (more: enumerated again)

constexpr int kMdWarps = 4;
constexpr int kLsWarps = 8;
constexpr int kT3Warps = 8;
constexpr int kT5Warps = 4;
constexpr int kPtWarps = 4;
constexpr int kPtChunk = 8;        // superbin modules per pT search work item (<= 32)

__global__ void k_reset(Arena A);
__global__ void k_bin_count(Arena A);
__global__ void k_bin_scan(Arena A);
__global__ void k_bin_scatter(Arena A);
__global__ void k_md(Arena A, DevCfg c);
__global__ void k_bin_sort(Arena A);
__global__ void k_md_plan(Arena A);
__global__ void k_md_search(Arena A, DevCfg c);
__global__ void k_md_write(Arena A, DevCfg c);
__global__ void k_ls(Arena A, DevCfg c);
__global__ void k_t3(Arena A, DevCfg c);
__global__ void k_t5(Arena A, DevCfg c);
__global__ void k_t5_plan(Arena A);
__global__ void k_t5_gather(Arena A);
__global__ void k_t5_refine(Arena A, DevCfg c);
__global__ void k_t5_mlp_select(Arena A, DevCfg c);
__global__ void k_pls(Arena A, DevCfg c);
__global__ void k_pt_plan(Arena A);
__global__ void k_t3_order(Arena A);
__global__ void k_pt5(Arena A, DevCfg c);
__global__ void k_pt3(Arena A, DevCfg c);
__global__ void k_pt5_refine(Arena A, DevCfg c);
__global__ void k_pt3_refine(Arena A, DevCfg c);
__global__ void k_clean_keys(Arena A, int pass);
size_t t5_plan_smem_bytes(int max_events);
__global__ void k_t3_features(Arena A, DevCfg c);
__global__ void k_t3_score(Arena A, DevCfg c, MlpParams P);
__global__ void k_clean_pt5(Arena A);
__global__ void k_clean_pt3_cross(Arena A, DevCfg c);
__global__ void k_clean_pt3_mark(Arena A);
__global__ void k_clean_t5(Arena A, DevCfg c);
__global__ void k_clean_pls(Arena A, DevCfg c);
__global__ void k_tc_pack(Arena A);

size_t md_smem_bytes();

}  // namespace lst
