/*
 * lst.h -- C ABI of the GB300 Segment Linking (Line Segment Tracking) library.
 *
 * The library builds, for one event or a batch of events, the object chain
 * of Segment Linking (arXiv:2209.13711, Section 2.1, kernel order of
 * Fig. KernelFlow): mini-doublets (stubs) from hit pairs in one pT module,
 * line segments between mini-doublets of connected modules (Fig.
 * CompModules), triplets and quintuplets from segments / triplets sharing a
 * mini-doublet (Figs. Triplet, Quintuplet, GeomReqs), pixel line segments
 * from pixel seeds and their links to triplets and quintuplets (pT3, pT5),
 * the cross-cleaning of Section 2.1 and the track-candidate collection. All
 * of it runs in CUDA kernels on one GPU (sm_103a); the host side only stages
 * inputs and launches.
 *
 * Conventions
 *   Units: cm, GeV, tesla, radians. A hit index is the position of the hit in
 *   the caller's per-event input arrays. Pixel seeds are three space points;
 *   seed s of an event owns pixel hits 3s, 3s+1, 3s+2.
 *   Every function returns an lst_status: 0 success, > 0 warning, < 0 error.
 *   Nothing is thrown across the ABI.
 *   Ownership: the caller owns every buffer it passes. Input arrays in
 *   pageable host memory must stay valid until the call returns (the copy is
 *   staged during the call); arrays in pinned host memory or device memory
 *   until the stream reaches the work (the copies are asynchronous). The
 *   library copies the geometry and keeps it until lst_destroy.
 *   Threading: one context per host thread; a context runs one batch at a
 *   time (a new run waits on the host for the previous batch to finish).
 *   Results: a run may return one lst_event_id per event (a handle). The
 *   track candidates and statistics of a batch run with handles are kept in
 *   one of LST_RESULT_SLOTS result slots until every event of the batch has
 *   been released (lst_release_event), across later runs; a batch run
 *   without handles gives its slot up to the next run. The intermediate
 *   objects (lst_get_objects, lst_get_t5_candidates) belong to the last batch
 *   only. Every getter takes an lst_event_id: a handle, or the index
 *   (0 <= event < n_events) of an event in the last batch.
 */
#ifndef LST_H
#define LST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lst_status;

/* An event handle: opaque, nonzero in its high 32 bits (a generation), so it
 * never equals an event index. Stale or released handles are refused with
 * LST_ERR_ARG. */
typedef int64_t lst_event_id;
#define LST_RESULT_SLOTS 4
enum {
    LST_OK = 0,
    LST_WARN_TRUNCATED = 1,      /* an occupancy cap dropped objects (counted in lst_stats) */
    LST_ERR_ARG = -1,            /* a null pointer, a negative size or an out-of-range id */
    LST_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    LST_ERR_OOM = -3,            /* device allocation failed at creation */
    LST_ERR_NO_GEOMETRY = -4,    /* lst_run_batch before lst_load_geometry */
    LST_ERR_TIMEOUT = -5,        /* reserved: a bounded device wait ran out */
    LST_ERR_CAPACITY = -6        /* the batch exceeds the context's event / hit / seed capacity, or every
                                    result slot holds unreleased events */
};

/* Cut constants of the chain. The paper fixes only pt_min = 0.8 GeV (Section 2);
 * every other value is this library's reading, filled by lst_config_default. */
typedef struct lst_config {
    double pt_min, k_field, b_field, z_lumi;
    double n_md, n_ls, n_t3, n_t5, n_pt;
    double tol_r;
    double chi2_rphi_t5, chi2_rz_t5, chi2_rphi_pt3, chi2_rz_pt3, chi2_rphi_pt5, chi2_rz_pt5;
    double pls_pt_tol, sig_pix;
    double sb_eta_max;
    int32_t sb_n_eta, sb_n_phi;
    double dr_clean;
} lst_config;

/* Capacities, fixed at creation; all device memory is allocated once. */
typedef struct lst_capacity {
    int32_t max_events;          /* events per batch, 1 .. 8192 */
    int32_t max_hits;            /* outer-tracker hits per batch */
    int32_t max_seeds;           /* pixel seeds per batch */
    int32_t md_per_event, ls_per_event, t3_per_event, t5_per_event;
    int32_t pt3_per_event, pt5_per_event, tc_per_event;
} lst_capacity;

/* One row of the module table (the geometry of Section 2: paired-sensor pT modules). */
typedef struct lst_module {
    int32_t subdet;              /* 0 barrel, 1 endcap */
    int32_t layer;               /* barrel layer 1..6 or endcap disk 1..5 */
    float dsep;                  /* sensor separation (cm) */
    float sig_rphi;              /* r-phi resolution (cm) */
    float sig_long;              /* resolution along the strip: z in the barrel, r in the endcap (cm) */
} lst_module;

/* Outer-tracker hits of a batch, concatenated event after event (SoA). */
typedef struct lst_hits {
    const float* x;
    const float* y;
    const float* z;
    const int32_t* module;       /* module id, 0 <= module < n_mod */
    const uint8_t* side;         /* 0 lower sensor (nearer the interaction point), 1 upper */
    int32_t n;                   /* total hits */
} lst_hits;

/* Pixel seeds of a batch: seed i has points (xyz[9i+3j .. 9i+3j+2]), j = 0, 1, 2,
 * ordered by increasing radius. */
typedef struct lst_seeds {
    const float* xyz;
    int32_t n;
} lst_seeds;

/* Per-event statistics. counts[k] and dropped[k] for k = 0 MD, 1 LS, 2 T3, 3 T5,
 * 4 pLS (passing), 5 pT5, 6 pT3, 7 TC. */
typedef struct lst_stats {
    int32_t counts[8];
    int32_t dropped[8];
} lst_stats;

typedef struct lst_ctx lst_ctx;

/* Fill *cfg with the library defaults. */
lst_status lst_config_default(lst_config* cfg);
/* Default capacities for `max_events` events shaped like a 200-pileup event. */
lst_status lst_capacity_default(lst_capacity* cap, int32_t max_events);

/* Create a context on CUDA device `device`; cfg and cap are copied. Allocates
 * every device buffer. On failure *out is NULL. */
lst_status lst_create(lst_ctx** out, const lst_config* cfg, const lst_capacity* cap, int32_t device);
void lst_destroy(lst_ctx* ctx);

/* Copy the geometry (host arrays) to the device: n_mod module rows, the
 * module connectivity map as CSR (conn_offsets[n_mod + 1], conn_targets: for
 * each module the modules of the next layer a pT >= pt_min helix can reach,
 * Fig. CompModules) and the pixel superbin map as CSR (sb_offsets[n_sb + 1],
 * sb_targets: modules a seed of that superbin can link to). n_sb must equal
 * sb_n_eta * sb_n_phi * 2. Synchronous. */
lst_status lst_load_geometry(lst_ctx* ctx, const lst_module* modules, int32_t n_mod,
                             const int32_t* conn_offsets, const int32_t* conn_targets,
                             const int32_t* sb_offsets, const int32_t* sb_targets, int32_t n_sb);

/* Enqueue the whole chain for a batch of n_events events on `cuda_stream`
 * (a cudaStream_t; NULL for the legacy default stream). hit_offsets and
 * seed_offsets are HOST arrays of n_events + 1 prefix offsets into the
 * concatenated hits and seeds. mem_is_device = 0: hits and seeds are host
 * pointers and are copied (pinned host memory makes the copy asynchronous);
 * 1: they are device pointers read in place. Returns when the work is
 * enqueued; results are read with lst_get_track_candidates / lst_get_objects.
 * The chain is one CUDA graph per context, captured on the first call (and
 * again after a change of launch shapes, stage limits or T5 selection) and
 * replayed on `cuda_stream`; with profiling on, the kernels are launched
 * one by one instead.
 *   ids: NULL, or a HOST array of n_events that receives one handle per event
 *   (the batch then holds its result slot until each event is released). With
 *   every slot held, LST_ERR_CAPACITY is returned before anything is enqueued.
 *   The chain's last stage writes the track candidates and statistics
 *   straight into the slot: handles cost no copy. */
lst_status lst_run_batch(lst_ctx* ctx, const lst_hits* hits, const int32_t* hit_offsets,
                         const lst_seeds* seeds, const int32_t* seed_offsets, int32_t n_events,
                         int32_t mem_is_device, void* cuda_stream, lst_event_id* ids);

/* A batch given event by event: hits[e] and seeds[e] (n_events entries, HOST
 * arrays of structs) point at each event's own arrays, host (mem_is_device =
 * 0; pinned memory makes the copies asynchronous) or device (1). The library
 * gathers them into its input staging with one copy per array and event on
 * `cuda_stream`, then runs the chain as lst_run_batch does. The event arrays
 * must stay valid until the stream reaches the copies. For serving loops whose
 * requests arrive with their own buffers. ids as for lst_run_batch. */
lst_status lst_run_events(lst_ctx* ctx, const lst_hits* hits, const lst_seeds* seeds, int32_t n_events,
                          int32_t mem_is_device, void* cuda_stream, lst_event_id* ids);

/* One event (the call of the paper's per-event processing, Section 2.2): the
 * chain of Section 2.1 / Fig. KernelFlow on one event's hits and pixel
 * seeds, enqueued on cuda_stream; lst_run_batch with n_events = 1. id: NULL
 * or a HOST lst_event_id that receives the event's handle. */
lst_status lst_run_event(lst_ctx* ctx, const lst_hits* hits, const lst_seeds* seeds, int32_t mem_is_device,
                         void* cuda_stream, lst_event_id* id);

/* Release one event of a batch run with handles; the batch's result slot is
 * free again once all its events are released. LST_ERR_ARG for an index, a
 * stale handle or one released before. Does not wait for the device. */
lst_status lst_release_event(lst_ctx* ctx, lst_event_id id);

/* Wait for the event's batch and copy the track candidates of `event` (a
 * handle, or an index in the last batch) into caller-owned arrays (HOST
 * memory): type[i] (0 pT5,
 * 1 pT3, 2 T5, 3 pLS), seed[i] (pixel seed index in the event, -1 for T5),
 * hits[10 i .. 10 i + 9] (outer-tracker hit indices in the event, -1 padded),
 * pt_eta_phi[3 i .. 3 i + 2]. Any output pointer may be NULL. At most
 * `capacity` rows are written; *n_out receives the true count and
 * LST_WARN_TRUNCATED is returned when it exceeds capacity. Candidate order is
 * unspecified. */
lst_status lst_get_track_candidates(lst_ctx* ctx, lst_event_id event, int32_t capacity, int32_t* n_out,
                                    int32_t* type, int32_t* seed, int32_t* hits, float* pt_eta_phi);

/* One track candidate of a batch, as packed by the chain's last stage. */
typedef struct lst_tc {
    int32_t type;        /* 0 pT5, 1 pT3, 2 T5, 3 pLS */
    int32_t seed;        /* pixel seed index in the event, -1 for T5 */
    int32_t hits[10];    /* outer-tracker hit indices in the event, -1 padded */
    float pt, eta, phi0;
    int32_t reserved;
} lst_tc;

/* Wait for the last batch and copy every event's track candidates with two
 * copies: offsets[0 .. n_events] (HOST, caller-owned; event e owns records
 * offsets[e] .. offsets[e + 1] - 1) and at most `capacity` records into `out`
 * (HOST; may be NULL when capacity is 0). LST_WARN_TRUNCATED when the batch
 * holds more than `capacity` records. Candidate order within an event is
 * unspecified. */
lst_status lst_get_batch_track_candidates(lst_ctx* ctx, int32_t capacity, int32_t* offsets, lst_tc* out);

/* Wait for the batch and copy one intermediate collection of event `event`
 * (for parity tests), which must belong to the last batch (LST_ERR_ARG
 * otherwise: a later run has overwritten the objects). kind: 0 MD, 1 LS, 2
 * T3, 3 T5, 4 pLS, 5 pT5, 6 pT3.
 * Rows are ints[ni * i ..] and floats[nf * i ..] (host memory) with
 *   MD : ints {lower hit, upper hit, module}              floats {dphi, dlong}
 *   LS : ints {inner MD row, outer MD row}                floats {dphi}
 *   T3 : ints {inner LS row, outer LS row}                floats {beta, kappa, sigk}
 *   T5 : ints {inner T3 row, outer T3 row}                floats {kappa, chi2_rphi, chi2_rz, eta, phi0, pt, score}
 *   pLS: ints {seed, pass, superbin}                      floats {kappa, sigk, eta, phi0, z0, pt}
 *   pT5: ints {seed, T5 row}                              floats {kappa, chi2_rphi, chi2_rz, score, pt}
 *   pT3: ints {seed, T3 row}                              floats {kappa, chi2_rphi, chi2_rz, score, pt}
 * where "row" indexes the rows returned for the same event and kind.
 * lst_object_columns gives ni and nf. Behaviour on capacity as above. */
lst_status lst_object_columns(int32_t kind, int32_t* ni, int32_t* nf);
lst_status lst_get_objects(lst_ctx* ctx, lst_event_id event, int32_t kind, int32_t capacity, int32_t* n_out,
                           int32_t* ints, float* floats);

/* Wait for the event's batch and copy its statistics (kept with the track
 * candidates in the result slot). */
lst_status lst_get_stats(lst_ctx* ctx, lst_event_id event, lst_stats* out);

/* Non-blocking: 1 when the last batch has finished on the device, 0 while it
 * runs (or when no batch was run), < 0 on error. */
int32_t lst_query(lst_ctx* ctx);
/* Device memory held by the context (bytes). */
int64_t lst_device_bytes(lst_ctx* ctx);

/* Launch shapes and the autotuner (batching, with per-event offsets and one
 * graph per batch, replaces the paper's one-event-per-stream overlap of
 * Section 2.2; the launch shape of each stage is this library's own knob, the
 * paper fixes none).
 *
 * The chain is a fixed sequence of stages (lst_launch_stage_count of them,
 * in Fig. KernelFlow order). Every stage whose flags have bit 0 set loops over
 * its units with a grid-stride loop, so its grid (n_SM x blocks_per_sm) may be
 * any size; bit 1 set means the stage indexes threads only through blockDim,
 * so its block may be any multiple of 32 up to the kernel's limit. Results do
 * not depend on the launch shape (object sets are identical; the order of
 * objects within an event's arrays may differ).
 *
 * lst_get_launch_config: the stage's name (static storage), its current
 *   blocks per SM (0 for a stage with a fixed grid), threads per block and flags.
 * lst_set_launch_config: 0 restores the default; LST_ERR_ARG for a stage out
 *   of range, a shape the stage does not allow, or a block above what the
 *   kernel can launch. Waits for the running batch; the next lst_run_batch
 *   captures a new graph.
 * lst_autotune: runs the given batch (same arguments as lst_run_batch) `reps`
 *   times (1..64) per candidate shape with profiling on, and keeps for every
 *   stage the shape with the smallest median device time (candidates: 1, 2, 3,
 *   4, 6, 8, 12 or 16 blocks per SM, with the default block or, for generic
 *   stages, 64, 128, 256 or 512 threads). *ms_before / *ms_after (optional):
 *   summed stage times of one run before and after. Synchronous; leaves the
 *   profiling switch as it found it and the context's results are those of the
 *   last tuning run of the batch. */
/* Survivors a search work item stages in shared memory before it falls back
 * to enumerating its candidates a second time and writing them directly: t5
 * for a T5 item (1..512, 0 restores 512), pt for a pT5 / pT3 item (1..256, 0
 * restores 256). Results do not depend on them; small limits exercise the
 * fallback. Waits for the running batch; the next batch captures a new graph. */
lst_status lst_set_stage_limits(lst_ctx* ctx, int32_t t5, int32_t pt);
/* Compact (16-bit) storage, off by default (half-precision object
 * properties are the paper's future work, Section 3). On: the triplets'
 * (curvature, sigma) pair is also stored in FP16 (scaled by 1/(2a)) and the
 * T5 and pT3 searches read that copy, with their FP32 prefilter slack widened
 * by the FP16 rounding; the cleaning's eta-phi lists hold 16-bit fixed-point
 * (eta, phi) pairs instead of FP32 ones, with the FP64 re-test band widened to
 * cover their rounding. Every decision is still taken by the FP32 / FP64
 * values, so the objects are those of the default storage. Waits for the
 * running batch; the next run captures a new graph. */
lst_status lst_set_compact_storage(lst_ctx* ctx, int32_t enable);
/* Precision of the refine fits (the five-point T5 fit, Section 2.1, and the
 * pT5 / pT3 fits, Section 2.2: the chord-frame circle fit, the residual chi2
 * and the r-z line fit). 0 (the default): float-float arithmetic (pairs of
 * FP32 numbers, about 48 significant bits) on the FP32 pipe from the FP32
 * hit coordinates; 1: FP64 as before. The two agree to about 1e-10 relative,
 * far inside the 1e-5 parity tolerance, so the objects are the same. Waits
 * for the running batch; the next run captures a new graph. */
lst_status lst_set_fp64_fit(lst_ctx* ctx, int32_t enable);
int32_t lst_launch_stage_count(void);
lst_status lst_get_launch_config(lst_ctx* ctx, int32_t stage, const char** name, int32_t* blocks_per_sm,
                                 int32_t* block, int32_t* flags);
lst_status lst_set_launch_config(lst_ctx* ctx, int32_t stage, int32_t blocks_per_sm, int32_t block);
lst_status lst_autotune(lst_ctx* ctx, const lst_hits* hits, const int32_t* hit_off, const lst_seeds* seeds,
                        const int32_t* seed_off, int32_t n_events, int32_t mem_is_device, void* stream,
                        int32_t reps, float* ms_before, float* ms_after);

/* Number of kernel launches enqueued by the last lst_run_batch. */
int32_t lst_last_launch_count(lst_ctx* ctx);

/* Profiling: when enabled, lst_run_batch records a CUDA event pair around
 * every kernel launch (on the batch's stream). lst_get_kernel_times waits for
 * the batch and returns, for each launch of the last batch in launch order,
 * its name (static storage) and its device time in milliseconds; at most
 * `capacity` entries, *n_out = the number of launches. Off by default. */
lst_status lst_set_profiling(lst_ctx* ctx, int32_t enable);
lst_status lst_get_kernel_times(lst_ctx* ctx, int32_t capacity, int32_t* n_out, const char** names, float* ms);

/* Allocation-free mini-doublet builder (the paper has no counterpart; this
 * is a library service). For callers that cannot allocate device memory: a
 * host framework that owns the device budget through its own pool and forbids
 * its plugins from calling cudaMalloc, or a latency-critical loop that must
 * not pay for an allocation. It runs the hit binning of lst_run_batch
 * (including the per-sensor sort by input index) and a one-warp-per-module
 * mini-doublet kernel with the same predicates on one event, and allocates
 * nothing: its scratch (bucket counters, sorted hits, module table in device
 * layout, MD anchors) lives in one file-scope device array of about 9 MB that
 * every device loading the library keeps until the process exits.
 *   All pointers except cfg are DEVICE memory owned by the caller: modules
 *   (n_mod rows), the event's hits (x, y, z, module, side; n_hits), and the
 *   outputs md_lower / md_upper (hit indices), md_module, md_dphi, md_dlong
 *   with room for md_capacity rows, md_count (one int: rows written) and
 *   md_dropped (one int, may be NULL: MDs lost to the per-module bounds or to
 *   md_capacity, plus hits ignored for a module id outside [0, n_mod) or a
 *   side above 1; nonzero means the rows are not the complete set). Rows
 *   match lst_get_objects(kind = 0) of the same event as a set (their order
 *   may differ), truncation included: a sensor with more than 256 hits keeps
 *   its 256 lowest input indices in both.
 *   Limits: n_hits <= 262144, n_mod <= 16384, md_capacity <= 131072; larger
 *   sizes return LST_ERR_CAPACITY before any work is enqueued.
 *   The first call on a device looks up the array's device address (on the
 *   current device); make that first call before any stream capture. Every
 *   call reuses the same array and clears what must start at zero; calls that
 *   overlap on the GPU race on it and must be serialized by the caller.
 *   Asynchronous on cuda_stream (NULL: legacy default stream). */
lst_status lst_build_mini_doublets_static(const lst_config* cfg, const lst_module* modules, int32_t n_mod,
                                          const float* x, const float* y, const float* z, const int32_t* module,
                                          const uint8_t* side, int32_t n_hits, int32_t md_capacity,
                                          int32_t* md_lower, int32_t* md_upper, int32_t* md_module, float* md_dphi,
                                          float* md_dlong, int32_t* md_count, int32_t* md_dropped,
                                          void* cuda_stream);

/* Wait for the batch and copy the batch-wide device counters: [0..5] objects
 * reserved (MD, LS, T3, T5 candidates, pT5 candidates, pT3 candidates), [10]
 * / [11] the LS / T3 searches' inner-MD cursors, [16]
 * hits with an invalid module or side, [20] T5 search work items (chunks of 8, 16
 * or 32 T3 of one inner MD, by batch size) whose survivors exceeded the shared-memory stage
 * and were enumerated a second time, [21] T5 search survivors, [22] + [23] T5
 * work items, [24] the T5 search's event pointer (items are taken event by
 * event; n_events once done), [25] pT work items (seed, superbin module),
 * [26] / [27] the pT5 / pT3 searches' item cursors, [28] pT work items
 * enumerated a second time. At most n (<= 32) values. */
lst_status lst_get_counters(lst_ctx* ctx, int32_t* out, int32_t n);

/* ---- learned T5 selection (an optional scoring network; the paper's own
 * selection is the hand-set cuts of Section 2.1, which stay the default, the
 * fallback and the yardstick of its efficiency) ---------------------------
 * Network: LST_MLP_INPUTS inputs (LST_MLP_FEATURES features, zero padded) ->
 * 64 -> 64 -> 32 -> 1, ReLU hidden, sigmoid output; BF16 weights and layer
 * inputs on tensor cores with FP32 accumulation. Parameters are FP32, laid out
 * as W1[64][48], b1[64], W2[64][64], b2[64], W3[32][64], b3[32], W4[32], b4. */
#define LST_MLP_FEATURES 38
#define LST_MLP_INPUTS 48
#define LST_MLP_PARAMS 9409
typedef struct lst_mlp lst_mlp;

/* A network on `device` able to take gradients over batches of up to
 * max_batch samples; parameters start at zero (set them). */
lst_status lst_mlp_create(lst_mlp** out, int32_t device, int32_t max_batch);
void lst_mlp_destroy(lst_mlp* m);
/* Host parameter vector in / out (LST_MLP_PARAMS floats); set resets Adam. */
lst_status lst_mlp_set_params(lst_mlp* m, const float* params);
lst_status lst_mlp_get_params(lst_mlp* m, float* params);
/* The whole training state, for checkpoints: parameters, Adam's first and
 * second moments (HOST arrays of LST_MLP_PARAMS floats each) and its step
 * count (the bias corrections depend on it). A network given the state of
 * another continues its training exactly as the other would. Synchronous. */
lst_status lst_mlp_get_state(lst_mlp* m, float* params, float* adam_m, float* adam_v, int64_t* step);
lst_status lst_mlp_set_state(lst_mlp* m, const float* params, const float* adam_m, const float* adam_v,
                             int64_t step);
/* scores[i] = network(features[i]) for n samples (DEVICE pointers, features
 * [n][LST_MLP_INPUTS]); asynchronous on stream. */
lst_status lst_mlp_forward(lst_mlp* m, const float* features, int32_t n, float* scores, void* stream);
/* Gradient of the mean binary cross-entropy over n <= max_batch samples
 * (features, labels in {0,1}: DEVICE); grad (LST_MLP_PARAMS) and loss are
 * HOST outputs (either may be NULL). Synchronous. */
lst_status lst_mlp_gradient(lst_mlp* m, const float* features, const float* labels, int32_t n, float* grad,
                            float* loss, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on that loss;
 * loss (HOST, may be NULL) receives the loss before the step (synchronizes
 * only when requested). */
lst_status lst_mlp_train_step(lst_mlp* m, const float* features, const float* labels, int32_t n, float lr,
                              float* loss, void* stream);

/* T5 selection of a context: mlp = NULL keeps the hand-set cuts; otherwise a
 * T5 candidate is valid when its network score >= threshold (and its fitted
 * curvature is within the pT window). prefilter_scale >= 1 widens the FP32
 * fit prefilter of the T5 search (more candidates for the network);
 * capture_features = 1 computes the features even without a network (for
 * training). The network must outlive its use by the context. */
lst_status lst_set_t5_selection(lst_ctx* ctx, const lst_mlp* mlp, float threshold, float prefilter_scale,
                                int32_t capture_features);
/* Learned triplet selection (optional; the default keeps every T3 that passes
 * the hand-set cuts). mlp = NULL: no network; otherwise every T3 is scored
 * (LST_MLP_FEATURES features of the triplet in the T5's slots, the missing
 * ones zero) and the T5 search skips the T3s whose score is below threshold,
 * which saves its combinatorics (the pT3 search, on its own branch of the
 * graph, keeps every T3 and starts without waiting for the scores). capture_features = 1 computes
 * the features without a network (for training). The first call that needs
 * them allocates the feature buffer (t3_per_event x max_events x 197 bytes;
 * LST_ERR_OOM if that fails). The network must outlive its use. Waits for the
 * running batch; the next run captures a new graph. */
lst_status lst_set_t3_selection(lst_ctx* ctx, const lst_mlp* mlp, float threshold, int32_t capture_features);
/* All T3s of an event of the last batch, HOST outputs (any may be NULL):
 * features [n][LST_MLP_INPUTS] (only when computed), hits [n][6] (lower,
 * upper of the three MDs), score [n] (with a network), kept [n] (1 when the
 * searches use the T3). */
lst_status lst_get_t3_candidates(lst_ctx* ctx, lst_event_id event, int32_t capacity, int32_t* n_out,
                                 float* features, int32_t* hits, float* score, int32_t* kept);
/* All T5 candidates of an event of the last batch (before the validity decision), HOST outputs:
 * features [n][LST_MLP_INPUTS] (when captured), hits [n][10] (lower, upper
 * of the five MDs), cut_pass [n] (the hand-set cut decision), score [n] (the
 * network score when attached). Any output may be NULL. */
lst_status lst_get_t5_candidates(lst_ctx* ctx, lst_event_id event, int32_t capacity, int32_t* n_out, float* features,
                                 int32_t* hits, int32_t* cut_pass, float* score);

/* ---- calibration (measurement support; not on the track-finding path) ----
 * Rates of the device measured with the library's own kernels, the
 * denominators of the per-kernel ALU and atomic fractions:
 *   fp32_tflops / fp64_tflops: FMA chains (2 flops per lane and FMA),
 *     8 (FP32) or 4 (FP64) independent chains per thread;
 *   atom_warp_gops: single-lane atomicAdd instructions with a used return,
 *     one per warp and iteration, each on its own 128-byte line (the form of
 *     the chain's warp-aggregated counters), per second, in 1e9;
 *   atom_same_gops: the same on one address shared by every warp;
 *   red_lane_gops: per-lane atomicAdd without a used return (reductions) to
 *     consecutive words;
 *   ms: best of three launches of each probe, in that order; sm_count;
 *   clock_khz: the device's reported maximum SM clock.
 * Each probe runs 8 blocks of 256 threads per SM for a fixed number of
 * iterations. Synchronous; allocates and frees 16 MB on `device` (which
 * becomes the calling thread's current device). LST_ERR_ARG for a negative
 * device or a NULL out, LST_ERR_OOM / LST_ERR_CUDA on a failed call. */
typedef struct lst_peaks {
    double fp32_tflops, fp64_tflops;
    double atom_warp_gops, atom_same_gops, red_lane_gops;
    float ms[5];
    int32_t sm_count, clock_khz;
} lst_peaks;
lst_status lst_measure_peaks(int32_t device, lst_peaks* out);

/* Message of a status code (static storage). */
const char* lst_status_str(lst_status s);

#ifdef __cplusplus
}
#endif
#endif /* LST_H */
