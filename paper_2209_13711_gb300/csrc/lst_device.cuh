// Device-side types and cut arithmetic of the Segment Linking chain.
//
// Every candidate test is written once as a template over the arithmetic
// type T. The float instantiation is the fast path: each cut "v <= thr" is
// decided in FP32 unless v lies within kBand * |thr| of its threshold, in
// which case the candidate is re-evaluated with T = double and that decision
// stands (a filtered predicate). The double instantiation decides every cut
// exactly as written. Quantities whose FP32 rounding is too coarse for a
// 1e-5 relative agreement (circle-fit residuals of 26 um against 100 cm
// coordinates) are only ever computed in double.
//
// The cut formulas are this library's reading of Section 2.1 of the paper
// (which gives the cut concepts, not formulas):
//   MD  (Section 2, Fig. pTModule): position-angle change between the two
//       sensors bounded by a pT_min helix, and the hits' z (barrel) or r
//       (endcap) consistent with a track from the luminous region.
//   LS  (Fig. CompModules): r-z pointing to |z0| <= z_lumi, position-angle
//       change and stub-vs-segment angles bounded by a pT_min helix.
//   T3  (Figs. Triplet, GeomReqs): relative angle beta of the two segments
//       bounded by a pT_min helix, r-z residual of the three anchors.
//   T5  (Fig. Quintuplet): inner/outer triplet curvature agreement, circle
//       fit chi2 and curvature, r-z line chi2.
//   pLS, pT3, pT5 (Section 2.1): seed curvature and z0 cuts, superbin,
//       pLS/T-object curvature agreement, joint circle and r-z fits.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lst_ff.cuh"
#include "lst_pdl.cuh"

namespace lst {

constexpr float kBand = 5e-4f;   // relative width of the FP32 undecided band around a threshold
constexpr double kPi = 3.14159265358979323846;

// Cut constants as seen by the kernels (derived on the host from lst_config).
// Limits of the conservative FP32 verdict on the fit cuts: a candidate is
// rejected only when a cut fails by far more than FP32 rounding can explain
// (|kappa| above 1.01 kmax + 1e-5, a chi2 above rel * max + abs; the
// per-object slack is set on the host).
struct FitLimits {
    float kappa, chi2, chi2z;
};

// FP32 copies of the constants the FP32 predicates use, converted once on the
// host (a double-to-float conversion per candidate would run on the FP64 pipe).
struct CfgF {
    float a, z_lumi, n_md, n_ls, n_t3, n_t5, n_pt, sig_pix;
};

struct DevCfg {
    double a;              // 1 / (2 R_min), R_min = 100 pT_min / (k B) cm
    double z_lumi, n_md, n_ls, n_t3, n_t5, n_pt, tol_r;
    double chi2_rphi_t5, chi2_rz_t5, chi2_rphi_pt3, chi2_rz_pt3, chi2_rphi_pt5, chi2_rz_pt5;
    double pls_pt_tol, sig_pix, sb_eta_max;
    int sb_n_eta, sb_n_phi;
    double dr_clean, k_field, b_field;
    int features_on;       // the T5 refine also writes the 38 scoring features
    int use_mlp;           // T5 validity from the network score instead of the cuts
    int fp64_fit;          // refine fits in FP64 (default: float-float on the FP32 pipe)
    float prefit_scale;    // widening of the T5 FP32 prefilter (1: conservative for the cuts)
    float mlp_threshold;
    float t3_threshold;    // learned triplet selection: keep a T3 when its score reaches this
    int t5_stage;          // T5 survivors staged per work item before the re-enumeration path
    int pt_stage;          // the same for the pT5 / pT3 search
    CfgF f;
    FitLimits lim_t5, lim_pt5, lim_pt3;   // FP32 prefilter limits (T5 widened by prefit_scale)
};

// The constant in the predicate's precision: FP32 predicates take the host-made copy.
template <typename T> __device__ __forceinline__ T cval(double d, float f);
template <> __device__ __forceinline__ float cval<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double cval<double>(double d, float) { return d; }

// Shape and inputs of the batch being processed (device memory).
// Per-event statistics a result slot keeps: counts[8], dropped[8], track
// candidates (the lst_stats kinds).
constexpr int kSlotStats = 17;
constexpr int kCellSlots = 8;      // list positions held per eta-phi cell
constexpr float kCellEta = 4.f;    // the cells cover |eta| < kCellEta

struct BatchDesc {
    int n_ev, n_hits, n_seeds, pad;
    const float* hx;
    const float* hy;
    const float* hz;
    const int* hmod;
    const uint8_t* hside;
    const float* seeds;           // [n_seeds][9]
    // the batch's result slot (chosen per run; the last stage writes it)
    struct TcRec* out_rec;        // packed track candidates, event after event
    int* out_off;                 // [n_ev + 1] record offsets
    int* out_stats;               // [n_ev][kSlotStats]
};

// Device buffers of one context (all preallocated; flat object arenas with
// per-unit segments).
struct Arena {
    // geometry
    int n_mod, n_sb;
    const float4* mod;            // {dsep, sig_rphi, sig_long, subdet}
    const int* mod_layer;
    const int* conn_off;
    const int* conn_tgt;
    const int* sb_off;
    const int* sb_tgt;
    // batch: shape and input pointers are read from device memory so that one
    // captured launch sequence serves every batch
    const struct BatchDesc* bd;
    int max_events;
    const int* hit_off;           // [n_ev + 1]
    const int* seed_off;          // [n_ev + 1]
    // hit binning: bucket (e, module, side) = e * 2 n_mod + 2 module + side
    int* bcnt;                    // [n_ev * 2 n_mod]: counts, then scatter cursors
    int* boff;                    // [n_ev * (2 n_mod + 1)]: offsets relative to hit_off[e]
    float* sx;
    float* sy;
    float* sz;
    int* sidx;                    // original hit index within the event
    // counters: [0] MD [1] LS [2] T3 [3] T5 [4] pT5 [5] pT3, [16] bad hits, [20] T5 overflow units
    int* counters;
    int* ev_counts;               // [n_ev][8]
    int* ev_drop;                 // [n_ev][8]
    // MD
    int md_cap;
    int* md_lo;
    int* md_up;
    int* md_gmod;                 // e * n_mod + module
    float4* md_p4;                // anchor (lower hit) x, y, z and +sig_z (barrel) / -sig_r (endcap)
    float2* md_sr;                // anchor {r-phi resolution, r = sqrtf(x^2 + y^2)}
    float4* md_lsc;               // FP32 LS terms of the MD (ls_terms_f32)
    float* md_dx;
    float* md_dy;
    float* md_dphi;
    float* md_dlong;
    // MD search work items: chunks of a module's lower hits
    int md_item_cap;
    int2* md_items;               // {unit, first lower rank | chunk length << 16}
    int* md_chunk_off;            // [max_hits] by the chunk's first lower-hit position
    int* md_chunk_cnt;
    int2* md_tmp;                 // [md_cap] passing (lower, upper) sorted-hit positions by chunk
    int* md_moff;                 // [n_ev * n_mod]
    int* md_mcnt;
    // LS
    int ls_cap;
    int* ls_in;
    int* ls_out;
    float* ls_dphi;
    int* ls_off;                  // [md_cap] segment of LS whose inner MD is this MD
    int* ls_cnt;
    // T3
    int t3_cap;
    int* t3_lsin;
    int* t3_lsout;
    float* t3_beta;
    float2* t3_ks;                // {curvature, its sigma} (FP32)
    __half2* t3_ksh;              // the same over 2a in FP16 (compact storage: the searches' copy)
    float two_a;                  // 2a in FP32 (the FP16 copy's scale)
    int compact;                  // 16-bit storage: FP16 triplet curvatures for the T5 / pT3 searches and
                                  // fixed-point eta-phi lists for the cleaning (decisions unchanged)
    // optional learned triplet selection (a network scores every T3; the T5 and pT3 searches skip the
    // T3s it rejects)
    int t3_sel;                   // 1: t3_ok gates the searches
    float* t3_feat;               // [T3][48] scoring features (allocated when enabled)
    float* t3_mlp;                // [T3] network score
    uint8_t* t3_ok;               // [T3] score >= threshold
    int4* t3_md;                  // the three MDs {inner, middle, outer, 0}
    int* t3_off;                  // [md_cap] by inner MD
    int* t3_cnt;
    int* t3_perm;                 // [t3_cap] the pT3 search's view: each inner MD's T3s in curvature order
    float2* t3_kord;              // [t3_cap] their (curvature, sigma) as the searches read them, in that order
    float* t3_smax;               // [md_cap] the largest such sigma of the MD's T3s; < 0: view not ordered
    // T5
    int t5_cap;
    int* t5_in;
    int* t5_out;
    double* t5_kappa;
    float* t5_chi2;
    float* t5_chi2z;
    float* t5_score;
    float* t5_pt;
    double* t5_sigk;
    double* t5_eta;
    double* t5_phi;
    uint8_t* t5_valid;            // the FP64 test passed (entries are FP32-prefiltered candidates)
    uint8_t* t5_cut;              // the hand-set cuts passed (== t5_valid without the network)
    float* t5_feat;               // [t5_cap][48] scoring features
    float* t5_mlp;                // network score
    float2* t5_ks;                // FP32 {curvature, sigma} of each T5 (the pT5 search's prefilter)
    int* t5_evf;                  // [n_ev] T5 work items at the front of each event's region (split units)
    int* t5_evb;                  // [n_ev] ... at its back (single-chunk units)
    int* t5_evc;                  // [n_ev] claim cursor of each event's items
    int* t5_evbase;               // [n_ev + 1] first item slot of each event's region
    int* t5_off;                  // [md_cap] by inner MD
    int* t5_cnt;
    // T5 search work items: chunks of 8, 16 or 32 T3_1 of one inner MD,
    // named by the T3 index of their first T3_1
    int* t5_items;                // [t3_cap] split units from the front, whole units from the back
    int* t5_chunk_off;            // [t3_cap] by chunk start: the chunk's segment of t5_tmp
    int* t5_chunk_cnt;
    int2* t5_tmp;                 // [t5_cap] survivors in chunk segments
    // pLS, per seed
    int* pls_pass;
    int* pls_sb;
    double* pls_kappa;
    double* pls_sigk;
    float* pls_z0;
    float* pls_pt;
    double* pls_eta;
    double* pls_phi;
    // pT5 / pT3
    int pt_item_cap;
    int2* pt_items;               // pT search work items: (seed, index into sb_tgt)
    int pt5_cap;
    int* pt5_seed;
    int* pt5_obj;
    float* pt5_kappa;
    float* pt5_chi2;
    float* pt5_chi2z;
    float* pt5_score;
    float* pt5_pt;
    uint8_t* pt5_valid;
    int pt3_cap;
    int* pt3_seed;
    int* pt3_obj;
    float* pt3_kappa;
    float* pt3_chi2;
    float* pt3_chi2z;
    float* pt3_score;
    float* pt3_pt;
    uint8_t* pt3_valid;
    // cleaning
    unsigned long long* best;     // [3][n_keys]: n_keys = n_hits + 3 n_seeds
    int* mark;                    // [n_keys] bit 0: used by a kept pT5, bit 1: by a kept pT3
    // per object (flat index over pT5, pT3, T5), written by the first cleaning
    // pass: its key, (event << 4) | number of hits, and its hits' key slots
    unsigned long long* obj_key;
    int* obj_meta;
    int* obj_slot;                // [16 per object]
    uint8_t* keep_pt5;
    uint8_t* keep_pt3;
    uint8_t* keep_t5;
    int* seed_link;               // [n_seeds]
    int list_cap;                 // per event
    int* list_cnt;                // [n_ev][2]: list 0 = kept pT5 + pT3, list 1 = kept T5
    float2* list_ef;              // [n_ev][2][list_cap] (eta, phi) float
    int* list_ref;                // [n_ev][2][list_cap] (category << 28) | index
    unsigned* list_q;             // compact storage: (eta, phi) as two 16-bit fixed-point halves
    // eta-phi cells over each list (|eta| < kCellEta, cell sides >= 2 (dr_clean + 1e-3)), so that a
    // query reads the entries of at most 2 x 2 cells; entries past kCellSlots in a cell, or outside the
    // eta range, go to the list's overflow, which every query scans
    int cell_ne, cell_np;         // cells in eta and in phi
    float cell_we, cell_wp;       // cell widths
    int* cell_cnt;                // [n_ev][2][cell_ne * cell_np]
    int* cell_idx;                // [n_ev][2][cells][kCellSlots]: list positions
    int* ovf_cnt;                 // [n_ev][2]
    int* ovf_idx;                 // [n_ev][2][list_cap]
    // track candidates, per-event slabs
    int tc_cap;
    int* tc_cnt;                  // [n_ev]
    int* tc_type;
    int* tc_seed;
    int* tc_obj;
    int* tc_hits;                 // [n_ev * tc_cap][10]
    float* tc_pt;
    float* tc_eta;
    float* tc_phi;
    // the batch's track candidates packed event after event (the last stage)
};

// One packed track candidate; the layout of lst_tc in the C ABI.
struct __align__(16) TcRec {
    int type, seed, hits[10];
    float pt, eta, phi;
    int reserved;
};
static_assert(sizeof(TcRec) == 64, "packed track candidate is 64 bytes");

// ---------------------------------------------------------------------------
// arithmetic helpers (float and double overloads)
// ---------------------------------------------------------------------------
// FP32 square roots and divisions are the approximate ones (rsqrtf,
// __fdividef: a few ulp). Every FP32 quantity here either feeds a decision
// that is retested in FP64 within a band far wider than that error, or is
// compared with a limit that carries slack for it; FP64 stays exact.
__device__ __forceinline__ float m_sqrt(float v) { return v > 1e-30f ? v * rsqrtf(v) : sqrtf(v); }
__device__ __forceinline__ double m_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ float m_asin(float v) { return asinf(v); }
__device__ __forceinline__ double m_asin(double v) { return asin(v); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
// Coordinates and their differences are bounded (|x| < 1e4 cm), so the
// plain root of the sum of squares neither overflows nor underflows.
__device__ __forceinline__ float m_hypot(float a, float b) { return m_sqrt(a * a + b * b); }
__device__ __forceinline__ double m_hypot(double a, double b) { return sqrt(a * a + b * b); }
__device__ __forceinline__ float m_abs(float v) { return fabsf(v); }
__device__ __forceinline__ double m_abs(double v) { return fabs(v); }
__device__ __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double m_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double m_min(double a, double b) { return fmin(a, b); }

template <typename T> __device__ __forceinline__ T sq(T v) { return v * v; }
template <typename T> __device__ __forceinline__ T asinc(T v) { return m_asin(m_min(T(1), m_max(T(0), v))); }
// transverse arc length of a chord c on a circle of curvature k
template <typename T> __device__ __forceinline__ T arc(T c, T k) {
    return k > T(0) ? m_div(T(2) * m_asin(m_min(T(1), c * k / T(2))), k) : c;
}
// angle in (-pi, pi]; loop-free (a non-finite input gives NaN)
__device__ __forceinline__ double wrap_pi(double p) {
    double q = p - 2 * kPi * rint(p / (2 * kPi));
    if (q <= -kPi) q += 2 * kPi;
    if (q > kPi) q -= 2 * kPi;
    return q;
}

// Filtered cut bookkeeping: state 1 accept, 0 reject, 2 undecided (FP32 only).
template <typename T> struct Cuts {
    bool fail = false;
    bool near = false;
    __device__ __forceinline__ void operator()(T v, T thr) {
        if (sizeof(T) == 4) {
            T band = T(kBand) * m_abs(thr);
            if (m_abs(v - thr) <= band) near = true;
            else if (!(v <= thr)) fail = true;        // also rejects NaN
        } else {
            if (!(v <= thr)) fail = true;
        }
    }
    __device__ __forceinline__ int state() const { return fail ? 0 : (near ? 2 : 1); }
};

// A measured point with its resolutions (along phi-hat, z, r-hat).
template <typename T> struct Pt {
    T x, y, z, r, srphi, sz, sr;
};

template <typename T> __device__ __forceinline__ Pt<T> hit_pt(float x, float y, float z, float4 mi) {
    Pt<T> p;
    p.x = T(x); p.y = T(y); p.z = T(z);
    p.r = m_hypot(p.x, p.y);
    p.srphi = T(mi.y);
    bool barrel = mi.w < 0.5f;
    p.sz = barrel ? T(mi.z) : T(0);
    p.sr = barrel ? T(0) : T(mi.z);
    return p;
}

template <typename T, typename S> __device__ __forceinline__ Pt<T> pix_pt(const float* q, S sig_pix) {
    Pt<T> p;
    p.x = T(q[0]); p.y = T(q[1]); p.z = T(q[2]);
    p.r = m_hypot(p.x, p.y);
    p.srphi = T(sig_pix); p.sz = T(sig_pix); p.sr = T(0);
    return p;
}

// MD anchor as a measured point
template <typename T> __device__ __forceinline__ Pt<T> md_point(const Arena& A, int i) {
    float4 p = A.md_p4[i];
    Pt<T> q;
    const float2 sr = A.md_sr[i];
    q.x = T(p.x); q.y = T(p.y); q.z = T(p.z);
    // FP32: the radius stored with the MD (the same sqrtf value); FP64: recomputed
    q.r = sizeof(T) == 4 ? T(sr.y) : m_hypot(q.x, q.y);
    q.srphi = T(sr.x);
    q.sz = p.w > 0.f ? T(p.w) : T(0);
    q.sr = p.w > 0.f ? T(0) : T(-p.w);
    return q;
}

// a b - c d with one rounding (Kahan's difference of products with an FMA)
__device__ __forceinline__ float m_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double m_fma(double a, double b, double c) { return fma(a, b, c); }
template <typename T> __device__ __forceinline__ T diff_prod(T a, T b, T c, T d) {
    const T w = c * d;
    return m_fma(a, b, -w) + m_fma(-c, d, w);
}

// error of P perpendicular to a chord of unit direction (cx, cy); across =
// |chord x r-hat|, passed in because it is computed from the exact
// coordinates of the chord's end points (|A x B| / (|AB| r_P)): for a chord
// nearly parallel to r-hat the rounded unit vectors would lose it
template <typename T> __device__ __forceinline__ T sigma_perp(const Pt<T>& P, T cx, T cy, T across) {
    T ir = m_div(T(1), P.r);
    T along = (cx * P.x + cy * P.y) * ir;
    return m_sqrt(sq(P.srphi * along) + sq(P.sr * across));
}

// ---------------------------------------------------------------------------
// MD: lower hit L, upper hit U of one module (mi = module row)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int md_eval(const DevCfg& c, float4 mi, const Pt<T>& L, const Pt<T>& U, T& dphi_o,
                                       T& dlong_o) {
    const T a = cval<T>(c.a, c.f.a);
    T dx = U.x - L.x, dy = U.y - L.y, dz = U.z - L.z;
    T rL = L.r;
    T dsep = T(mi.x), srphi = T(mi.y), sl = T(mi.z);
    T dphi = m_atan2(L.x * dy - L.y * dx, L.x * U.x + L.y * U.y);
    T dlong, thr_phi, thr_long;
    const T rt2 = T(1.4142135623730951);
    if (mi.w < 0.5f) {
        thr_phi = asinc((rL + dsep) * a) - asinc(rL * a) + cval<T>(c.n_md, c.f.n_md) * rt2 * srphi / rL;
        dlong = dz - dsep * L.z / rL;
        thr_long = cval<T>(c.n_md, c.f.n_md) * rt2 * sl + dsep * cval<T>(c.z_lumi, c.f.z_lumi) / rL;
    } else {
        T az = m_abs(L.z);
        // r_U - r_L from the exact coordinate differences (no cancellation)
        T dr = (dx * (U.x + L.x) + dy * (U.y + L.y)) / (U.r + rL);
        dlong = dr - dsep * rL / az;
        thr_long = cval<T>(c.n_md, c.f.n_md) * rt2 * sl;
        T ds_max = T(1.2) * dsep * (rL + cval<T>(c.n_md, c.f.n_md) * sl) / (az - cval<T>(c.z_lumi, c.f.z_lumi));
        thr_phi = a * ds_max + cval<T>(c.n_md, c.f.n_md) * rt2 * srphi / rL;
    }
    Cuts<T> cut;
    cut(m_abs(dphi), thr_phi);
    if (!cut.fail) cut(m_abs(dlong), thr_long);
    dphi_o = dphi;
    dlong_o = dlong;
    return cut.state();
}

// ---------------------------------------------------------------------------
// LS between MD A (anchor PA, stub sA, module mA) and MD B
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int ls_eval(const DevCfg& c, const Pt<T>& P, T sAx, T sAy, float4 mA, const Pt<T>& Q,
                                       T sBx, T sBy, float4 mB, T& dphi_o) {
    const T a = cval<T>(c.a, c.f.a);
    const T n = cval<T>(c.n_ls, c.f.n_ls);
    Cuts<T> cut;
    T num = P.z * Q.r - Q.z * P.r;
    T den = Q.r - P.r;
    T sig_num = m_sqrt(sq(Q.r * P.sz) + sq(P.r * Q.sz) + sq(Q.z * P.sr) + sq(P.z * Q.sr));
    cut(m_abs(num), cval<T>(c.z_lumi, c.f.z_lumi) * m_abs(den) + n * sig_num);
    // P x Q as P x (Q - P): products of the anchor with the short segment
    T ux = Q.x - P.x, uy = Q.y - P.y;
    T dphi = m_atan2(P.x * uy - P.y * ux, P.x * Q.x + P.y * Q.y);
    dphi_o = dphi;
    if (cut.fail) return 0;
    T lo = asinc(m_max(T(0), P.r - n * P.sr) * a);
    T thr_phi = asinc((Q.r + n * Q.sr) * a) - lo + n * m_sqrt(sq(P.srphi / P.r) + sq(Q.srphi / Q.r));
    cut(m_abs(dphi), thr_phi);
    if (cut.fail) return 0;
    T lu = m_hypot(ux, uy);
    T base = asinc((Q.r + T(mB.x) + n * Q.sr) * a) - lo;
    T rt2 = T(1.4142135623730951);
    if (mA.w < 0.5f) {
        T ls_ = m_hypot(sAx, sAy);
        T al = m_atan2(sAx * uy - sAy * ux, sAx * ux + sAy * uy);
        cut(m_abs(al), base + n * (m_div(rt2 * P.srphi, ls_) + m_div(P.sr + Q.sr, lu)));
        if (cut.fail) return 0;
    }
    if (mB.w < 0.5f) {
        T ls_ = m_hypot(sBx, sBy);
        T al = m_atan2(sBx * uy - sBy * ux, sBx * ux + sBy * uy);
        cut(m_abs(al), base + n * (m_div(rt2 * Q.srphi, ls_) + m_div(P.sr + Q.sr, lu)));
    }
    return cut.state();
}

// The per-MD terms of the LS test in FP32, computed once when the MD is
// written: {asinc((r + n sr) a), asinc((r + dsep + n sr) a),
// asinc(max(0, r - n sr) a), srphi / r}.
__device__ __forceinline__ float4 ls_terms_f32(const DevCfg& c, const Pt<float>& P, float dsep) {
    const float a = c.f.a, n = c.f.n_ls;
    return make_float4(asinc((P.r + n * P.sr) * a), asinc((P.r + dsep + n * P.sr) * a),
                       asinc(m_max(0.f, P.r - n * P.sr) * a), P.srphi / P.r);
}

// ls_eval<float> with the per-MD terms of anchor (tP) and candidate (tQ)
// taken from the MD records; the same cuts in the same order.
__device__ __forceinline__ int ls_eval_f32(const DevCfg& c, const Pt<float>& P, float4 tP, float sAx, float sAy,
                                           float4 mA, const Pt<float>& Q, float4 tQ, float sBx, float sBy,
                                           float4 mB, float& dphi_o) {
    const float n = c.f.n_ls;
    Cuts<float> cut;
    float num = P.z * Q.r - Q.z * P.r;
    float den = Q.r - P.r;
    float sig_num = m_sqrt(sq(Q.r * P.sz) + sq(P.r * Q.sz) + sq(Q.z * P.sr) + sq(P.z * Q.sr));
    cut(m_abs(num), c.f.z_lumi * m_abs(den) + n * sig_num);
    float ux = Q.x - P.x, uy = Q.y - P.y;
    float dphi = m_atan2(P.x * uy - P.y * ux, P.x * Q.x + P.y * Q.y);
    dphi_o = dphi;
    if (cut.fail) return 0;
    const float lo = tP.z;
    float thr_phi = tQ.x - lo + n * m_sqrt(sq(tP.w) + sq(tQ.w));
    cut(m_abs(dphi), thr_phi);
    if (cut.fail) return 0;
    float lu = m_hypot(ux, uy);
    float base = tQ.y - lo;
    const float rt2 = 1.4142135623730951f;
    if (mA.w < 0.5f) {
        float ls_ = m_hypot(sAx, sAy);
        float al = m_atan2(sAx * uy - sAy * ux, sAx * ux + sAy * uy);
        cut(m_abs(al), base + n * (m_div(rt2 * P.srphi, ls_) + m_div(P.sr + Q.sr, lu)));
        if (cut.fail) return 0;
    }
    if (mB.w < 0.5f) {
        float ls_ = m_hypot(sBx, sBy);
        float al = m_atan2(sBx * uy - sBy * ux, sBx * ux + sBy * uy);
        cut(m_abs(al), base + n * (m_div(rt2 * Q.srphi, ls_) + m_div(P.sr + Q.sr, lu)));
    }
    return cut.state();
}

// ---------------------------------------------------------------------------
// three-point quantities
// ---------------------------------------------------------------------------
template <typename T> struct Tri {
    T lu, lv, lw, beta, sig_beta, kappa, sigk;
};

template <typename T> __device__ __forceinline__ Tri<T> tri(const Pt<T>& A, const Pt<T>& B, const Pt<T>& C) {
    Tri<T> t;
    T ux = B.x - A.x, uy = B.y - A.y;
    T vx = C.x - B.x, vy = C.y - B.y;
    T wx = C.x - A.x, wy = C.y - A.y;
    t.lu = m_hypot(ux, uy);
    t.lv = m_hypot(vx, vy);
    t.lw = m_hypot(wx, wy);
    t.beta = m_atan2(ux * vy - uy * vx, ux * vx + uy * vy);
    T iu = m_div(T(1), t.lu), iv = m_div(T(1), t.lv);
    const T xAB = m_abs(diff_prod(A.x, B.y, A.y, B.x)) * iu;   // |A x B| / |AB|
    const T xBC = m_abs(diff_prod(B.x, C.y, B.y, C.x)) * iv;
    T sAu = sigma_perp(A, ux * iu, uy * iu, m_div(xAB, A.r));
    T sBu = sigma_perp(B, ux * iu, uy * iu, m_div(xAB, B.r));
    T sBv = sigma_perp(B, vx * iv, vy * iv, m_div(xBC, B.r));
    T sCv = sigma_perp(C, vx * iv, vy * iv, m_div(xBC, C.r));
    t.sig_beta = m_sqrt(sq(sAu * iu) + sq(sBu * iu + sBv * iv) + sq(sCv * iv));
    t.kappa = m_div(T(2) * (ux * wy - uy * wx), t.lu * t.lv * t.lw);
    t.sigk = m_div(T(2) * t.sig_beta, t.lu + t.lv);
    return t;
}

template <typename T>
__device__ __forceinline__ int t3_eval(const DevCfg& c, const Pt<T>& A, const Pt<T>& B, const Pt<T>& C, T& beta_o,
                                       T& kappa_o, T& rz_o, T& sigk_o) {
    const T a = cval<T>(c.a, c.f.a);
    Tri<T> t = tri(A, B, C);
    Cuts<T> cut;
    beta_o = t.beta;
    kappa_o = t.kappa;
    sigk_o = t.sigk;
    cut(m_abs(t.beta), asinc(t.lu * a) + asinc(t.lv * a) + cval<T>(c.n_t3, c.f.n_t3) * t.sig_beta);
    T ka = m_abs(t.kappa);
    T sB = arc(t.lu, ka), sC = arc(t.lw, ka);
    T d = (B.z - A.z) * sC - (C.z - A.z) * sB;
    rz_o = d;
    if (cut.fail) return 0;
    T sig_d = m_sqrt(sq((sB - sC) * A.sz) + sq(sC * B.sz) + sq(sB * C.sz) + sq((C.z - B.z) * A.sr) +
                     sq((C.z - A.z) * B.sr) + sq((B.z - A.z) * C.sr));
    cut(m_abs(d), cval<T>(c.n_t3, c.f.n_t3) * sig_d);
    return cut.state();
}

// ---------------------------------------------------------------------------
// circle fit in the chord frame + r-z line fit (double only)
// ---------------------------------------------------------------------------
struct Fit {
    double kappa, chi2_rphi, chi2_rz, tanl;
};

// Full output of the chord-frame fit: circle g (xi^2+eta^2) + h xi + k - eta = 0
// in the frame (origin O, x-hat (xx, xy)), S = sqrt(1 + h^2 - 4gk), and the
// r-z line z = c0 + t s (s: arc length from P[0]) with its t_hat.
struct FitFull {
    double gg, hh, kk, S, xx, xy, ox, oy, c0, t, t_hat, kappa, chi2, chi2z;
};

// Pf (optional) holds the same points in FP32. With it, the quantities that
// are well conditioned given the FP64 residual u -- the geometric residual e
// from u, the circle normal, the error projected on it and the r-z weights --
// are computed in FP32 (relative error ~1e-7 of chi2); the fit itself, the
// residuals and the arc lengths stay FP64. Without it everything is FP64.
template <int N> __device__ inline Fit fit_track(const Pt<double>* P, FitFull* full = nullptr,
                                                 const Pt<float>* Pf = nullptr) {
    Fit f;
    const Pt<double>& O = P[N / 2];
    double ex = P[N - 1].x - P[0].x, ey = P[N - 1].y - P[0].y;
    double il = rsqrt(ex * ex + ey * ey);
    double xx = ex * il, xy = ey * il;
    double yx = -xy, yy = xx;
    double xi[N], et[N], rho2[N];
    double mr = 0.0, mx = 0.0, me = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double dx = P[i].x - O.x, dy = P[i].y - O.y;
        xi[i] = dx * xx + dy * xy;
        et[i] = dx * yx + dy * yy;
        rho2[i] = xi[i] * xi[i] + et[i] * et[i];
        mr += rho2[i]; mx += xi[i]; me += et[i];
    }
    // least squares of et ~ gg rho2 + hh xi + kk through the centred moments
    // (the normal equations with the intercept eliminated)
    mr *= 1.0 / N; mx *= 1.0 / N; me *= 1.0 / N;
    double saa = 0.0, sab = 0.0, sbb = 0.0, sac = 0.0, sbc = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double a = rho2[i] - mr, b = xi[i] - mx, cc = et[i] - me;
        saa += a * a; sab += a * b; sbb += b * b; sac += a * cc; sbc += b * cc;
    }
    const double det = saa * sbb - sab * sab;
    if (!(det > 0.0)) {
        f.kappa = 1e30; f.chi2_rphi = 1e30; f.chi2_rz = 1e30; f.tanl = 0;
        if (full) *full = FitFull{0, 0, 0, 1, xx, xy, O.x, O.y, 0, 0, 0, 1e30, 1e30, 1e30};
        return f;
    }
    const double idet = 1.0 / det;
    double gg = (sac * sbb - sab * sbc) * idet, hh = (saa * sbc - sab * sac) * idet;
    double kk = me - gg * mr - hh * mx;
    double S = sqrt(fmax(0.0, 1.0 + hh * hh - 4.0 * gg * kk));
    f.kappa = 2.0 * gg / S;
    double chi2 = 0.0;
    if (Pf) {
        const float gf = float(gg), hf = float(hh), Sf = float(S), xxf = float(xx), xyf = float(xy);
        const float oxf = Pf[N / 2].x, oyf = Pf[N / 2].y;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const float uf = float(gg * rho2[i] + hh * xi[i] + kk - et[i]);
            const float e = 2.f * uf / (Sf + sqrtf(fmaxf(0.f, Sf * Sf + 4.f * gf * uf)));
            const float dxf = Pf[i].x - oxf, dyf = Pf[i].y - oyf;
            const float xif = dxf * xxf + dyf * xyf, etf = dyf * xxf - dxf * xyf;
            if (Pf[i].sr > 0.f) {
                // endcap strip: sr >> srphi, so the radial component of the
                // normal (small, from a cancelling dot product) needs FP64
                const double nlx = 2.0 * gg * xi[i] + hh, nly = 2.0 * gg * et[i] - 1.0;
                const double nx = nlx * xx - nly * xy, ny = nlx * xy + nly * xx;
                const double nn2 = nx * nx + ny * ny;
                const double ir = 1.0 / P[i].r;
                const double rx = P[i].x * ir, ry = P[i].y * ir;
                const double n_phi = ny * rx - nx * ry, n_r = nx * rx + ny * ry;
                const double s2 = fmax(sq(P[i].srphi * n_phi) + sq(P[i].sr * n_r), sq(0.01 * P[i].srphi) * nn2);
                chi2 += double(e) * double(e) * nn2 / s2;
                continue;
            }
            const float nlx = 2.f * gf * xif + hf, nly = 2.f * gf * etf - 1.f;
            const float nx = nlx * xxf - nly * xyf, ny = nlx * xyf + nly * xxf;
            const float nn2 = nx * nx + ny * ny;
            const float ir = 1.f / Pf[i].r;
            const float rx = Pf[i].x * ir, ry = Pf[i].y * ir;
            const float n_phi = ny * rx - nx * ry;
            const float s2 = fmaxf(sq(Pf[i].srphi * n_phi), sq(0.01f * Pf[i].srphi) * nn2);
            chi2 += double(e * e * nn2 / s2);
        }
    } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        // geometric residual e, and the point's error projected on the circle
        // normal; the normal is left unnormalised and the squared norm divides
        // once: s2 = (srphi^2 n_phi^2 + sr^2 n_r^2) / |n|^2 (|n| >= ~1 here)
        double u = gg * rho2[i] + hh * xi[i] + kk - et[i];
        double e = 2.0 * u / (S + sqrt(fmax(0.0, S * S + 4.0 * gg * u)));
        double nlx = 2.0 * gg * xi[i] + hh, nly = 2.0 * gg * et[i] - 1.0;
        double nx = nlx * xx + nly * yx, ny = nlx * xy + nly * yy;
        double nn2 = nx * nx + ny * ny;
        double ir = 1.0 / P[i].r;
        double rx = P[i].x * ir, ry = P[i].y * ir;
        double n_phi = -nx * ry + ny * rx;
        double n_r = nx * rx + ny * ry;
        double s2 = fmax(sq(P[i].srphi * n_phi) + sq(P[i].sr * n_r), sq(0.01 * P[i].srphi) * nn2);
        chi2 += e * e * nn2 / s2;
    }
    }
    f.chi2_rphi = chi2;
    double ka = fabs(f.kappa);
    // arc lengths from the first point (arc(): 2 asin(c ka / 2) / ka), the
    // division by ka taken once
    const double k2 = 0.5 * ka, ik = ka > 0.0 ? 2.0 / ka : 0.0;
    double s[N];
    s[0] = 0.0;
#pragma unroll
    for (int i = 1; i < N; ++i) {
        const double c = sqrt(sq(P[i].x - P[0].x) + sq(P[i].y - P[0].y));
        s[i] = ka > 0.0 ? asin(fmin(1.0, c * k2)) * ik : c;
    }
    double t_hat = (P[N - 1].z - P[0].z) / s[N - 1];
    double w[N], W = 0, Ws = 0, Wz = 0;
    const float tf = float(t_hat);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        w[i] = Pf ? double(1.f / fmaxf(1e-12f, sq(Pf[i].sz) + sq(tf * Pf[i].sr)))
                  : 1.0 / fmax(1e-12, sq(P[i].sz) + sq(t_hat * P[i].sr));
        W += w[i];
        Ws += w[i] * s[i];
        Wz += w[i] * P[i].z;
    }
    const double iW = 1.0 / W;
    double sbar = Ws * iW, zbar = Wz * iW, Sss = 0, Ssz = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        Sss += w[i] * sq(s[i] - sbar);
        Ssz += w[i] * (s[i] - sbar) * (P[i].z - zbar);
    }
    double t = Ssz / Sss, c0 = zbar - t * sbar, chi2z = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) chi2z += w[i] * sq(P[i].z - c0 - t * s[i]);
    f.chi2_rz = chi2z;
    f.tanl = t;
    if (full) {
        full->gg = gg; full->hh = hh; full->kk = kk; full->S = S; full->xx = xx; full->xy = xy;
        full->ox = O.x; full->oy = O.y; full->c0 = c0; full->t = t; full->t_hat = t_hat;
        full->kappa = f.kappa; full->chi2 = chi2; full->chi2z = chi2z;
    }
    return f;
}

// r-phi chi2 term of point Q (scaled-frame coordinates xi, et, rho2) for the
// circle (gg, hh, kk) of fit_track_ff: the geometric residual from u and the
// error projected on the circle normal, as in fit_track with FP32 points, with
// the radial component of the normal at a strip point in float-float.
__device__ __forceinline__ float ff_rphi_term(const Pt<float>& Q, ff xi, ff et, ff rho2, ff gg, ff hh, ff kk, ff ex,
                                              ff ey, float Sf, float iLf) {
    const float gf = gg.hi, hf = hh.hi, exf = ex.hi, eyf = ey.hi;
    const float u = (gg * rho2 + hh * xi + kk - et).hi;
    const float e = 2.f * u / (Sf + sqrtf(fmaxf(0.f, Sf * Sf + 4.f * gf * u))) * iLf;
    // the normal (nlx, nly) in the chord frame; n_phi, n_r against the radial direction
    const float nlx = 2.f * gf * xi.hi + hf, nly = 2.f * gf * et.hi - 1.f;
    const float nn2 = nlx * nlx + nly * nly;
    const float ilr = iLf / Q.r;
    const float n_phi = ((nlx * eyf + nly * exf) * Q.x - (nlx * exf - nly * eyf) * Q.y) * ilr;
    float s2;
    if (Q.sr > 0.f) {
        const ff lx = gg * xi * 2.f + hh, ly = gg * et * 2.f - 1.f;
        const float n_r = ((lx * ex - ly * ey) * Q.x + (lx * ey + ly * ex) * Q.y).hi * ilr;
        s2 = fmaxf(sq(Q.srphi * n_phi) + sq(Q.sr * n_r), sq(0.01f * Q.srphi) * nn2);
    } else {
        s2 = fmaxf(sq(Q.srphi * n_phi), sq(0.01f * Q.srphi) * nn2);
    }
    return e * e * nn2 / s2;
}

// fit_track in float-float on the FP32 pipe, from the FP32 points (the
// coordinates are FP32 in memory, so the FP64 fit sees the same numbers).
// The frame axis is the exact chord (the differences of the end points as
// float-float), left unnormalised: the chord frame scaled by the chord length
// L, to which the algebraic circle fit is invariant (curvature and residuals
// scale by L and 1/L). The axis must be exact: the fit is not invariant under
// a turn of the frame, and a turn by the FP32 rounding of the chord (~1e-7
// rad) moves the curvature of a nearly straight candidate by ~2e-11 /cm, 1e-4
// of a curvature of 2e-7 /cm. The residuals, the arc lengths and the r-z line
// fit are float-float; the geometric residual from u, the error projection on
// the circle normal and the r-z weights are FP32, as in fit_track with FP32
// points, except the radial component of the normal at strip points (a
// cancelling dot product), which is float-float. The point loops stay rolled:
// unrolled, the float-float code outgrows the instruction cache (measured:
// instruction-fetch stalls dominated the refine).
template <int N> __device__ inline Fit fit_track_ff(const Pt<float>* P) {
    Fit f;
    const float ox = P[N / 2].x, oy = P[N / 2].y;
    const ff ex = two_sum(P[N - 1].x, -P[0].x), ey = two_sum(P[N - 1].y, -P[0].y);
    const ff L2 = ex * ex + ey * ey;
    ff xi[N], et[N], rho2[N];
    ff mr{0.f, 0.f}, mx{0.f, 0.f}, me{0.f, 0.f};
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        const ff dx = two_sum(P[i].x, -ox), dy = two_sum(P[i].y, -oy);
        xi[i] = dx * ex + dy * ey;
        et[i] = dy * ex - dx * ey;
        rho2[i] = (dx * dx + dy * dy) * L2;
        mr = mr + rho2[i]; mx = mx + xi[i]; me = me + et[i];
    }
    mr = mr / float(N); mx = mx / float(N); me = me / float(N);
    ff saa{0.f, 0.f}, sab{0.f, 0.f}, sbb{0.f, 0.f}, sac{0.f, 0.f}, sbc{0.f, 0.f};
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        const ff a = rho2[i] - mr, b = xi[i] - mx, cc = et[i] - me;
        saa = saa + a * a; sab = sab + a * b; sbb = sbb + b * b; sac = sac + a * cc; sbc = sbc + b * cc;
    }
    const ff det = saa * sbb - sab * sab;
    if (!(det.hi > 0.f)) {
        f.kappa = 1e30; f.chi2_rphi = 1e30; f.chi2_rz = 1e30; f.tanl = 0;
        return f;
    }
    // the circle in the scaled frame; curvature and residuals scale by L, 1/L
    const ff gg = (sac * sbb - sab * sbc) / det, hh = (saa * sbc - sab * sac) / det;
    const ff kk = me - gg * mr - hh * mx;
    const ff S = ff_sqrt(hh * hh + 1.f - gg * kk * 4.f);
    const ff L = ff_sqrt(L2);
    const ff kappa = gg * L * 2.f / S;
    f.kappa = ff_d(kappa);
    const float iLf = 1.f / L.hi;
    float chi2 = 0.f;
#pragma unroll 1
    for (int i = 0; i < N; ++i) chi2 += ff_rphi_term(P[i], xi[i], et[i], rho2[i], gg, hh, kk, ex, ey, S.hi, iLf);
    f.chi2_rphi = chi2;
    // r-z: arc lengths from the first point, weighted line z = c0 + t s
    const ff ka = ff_abs(kappa);
    ff s[N];
    s[0] = ff{0.f, 0.f};
#pragma unroll 1
    for (int i = 1; i < N; ++i) {
        const ff cx = two_sum(P[i].x, -P[0].x), cy = two_sum(P[i].y, -P[0].y);
        s[i] = ff_arc(ff_sqrt(cx * cx + cy * cy), ka);
    }
    const float t_hat = (P[N - 1].z - P[0].z) / s[N - 1].hi;
    float w[N];
    ff W{0.f, 0.f}, Ws{0.f, 0.f}, Wz{0.f, 0.f};
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        w[i] = 1.f / fmaxf(1e-12f, sq(P[i].sz) + sq(t_hat * P[i].sr));
        W = W + w[i];
        Ws = Ws + s[i] * w[i];
        Wz = Wz + two_prod(w[i], P[i].z);
    }
    const ff sbar = Ws / W, zbar = Wz / W;
    ff Sss{0.f, 0.f}, Ssz{0.f, 0.f};
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        const ff ds = s[i] - sbar, dz = ff_of(P[i].z) - zbar;
        Sss = Sss + ds * ds * w[i];
        Ssz = Ssz + ds * dz * w[i];
    }
    const ff t = Ssz / Sss, c0 = zbar - t * sbar;
    float chi2z = 0.f;
#pragma unroll 1
    for (int i = 0; i < N; ++i) {
        const float r = (ff_of(P[i].z) - c0 - t * s[i]).hi;
        chi2z += w[i] * r * r;
    }
    f.chi2_rz = chi2z;
    f.tanl = ff_d(t);
    return f;
}

// The same fit with one candidate per group of 8 lanes: lane j of the group
// holds point j (j < N) in FP64 (Q) and FP32 (Qf); the per-point work runs in
// parallel, the sums are taken with shuffles and every lane of the group
// returns the fit. For kernels with few candidates, where one thread per
// candidate would leave the FP64 latency exposed. All 32 lanes must call.
__device__ __forceinline__ double grp_sum8(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
    return v;
}

template <int N> __device__ inline Fit fit_track_group(const Pt<double>& Q, const Pt<float>& Qf, int j) {
    static_assert(N <= 8, "one point per lane of a group of 8");
    const unsigned F = 0xffffffffu;
    const bool act = j < N;
    Fit f;
    const double x0 = __shfl_sync(F, Q.x, 0, 8), y0 = __shfl_sync(F, Q.y, 0, 8), z0 = __shfl_sync(F, Q.z, 0, 8);
    const double xn = __shfl_sync(F, Q.x, N - 1, 8), yn = __shfl_sync(F, Q.y, N - 1, 8);
    const double zn = __shfl_sync(F, Q.z, N - 1, 8);
    const double ox = __shfl_sync(F, Q.x, N / 2, 8), oy = __shfl_sync(F, Q.y, N / 2, 8);
    const float oxf = __shfl_sync(F, Qf.x, N / 2, 8), oyf = __shfl_sync(F, Qf.y, N / 2, 8);
    const double ex = xn - x0, ey = yn - y0;
    const double il = rsqrt(ex * ex + ey * ey);
    const double xx = ex * il, xy = ey * il, yx = -xy, yy = xx;
    const double dx = Q.x - ox, dy = Q.y - oy;
    const double xi = dx * xx + dy * xy, et = dx * yx + dy * yy, rho2 = xi * xi + et * et;
    const double w1 = act ? 1.0 : 0.0;
    // centred least squares, as in fit_track
    const double mr = grp_sum8(w1 * rho2) * (1.0 / N), mx = grp_sum8(w1 * xi) * (1.0 / N);
    const double me = grp_sum8(w1 * et) * (1.0 / N);
    const double ca = w1 * (rho2 - mr), cb = w1 * (xi - mx), cc = w1 * (et - me);
    const double saa = grp_sum8(ca * ca), sab = grp_sum8(ca * cb), sbb = grp_sum8(cb * cb);
    const double sac = grp_sum8(ca * cc), sbc = grp_sum8(cb * cc);
    const double det = saa * sbb - sab * sab;
    if (!(det > 0.0)) {
        f.kappa = 1e30; f.chi2_rphi = 1e30; f.chi2_rz = 1e30; f.tanl = 0;
        return f;
    }
    const double idet = 1.0 / det;
    const double gg = (sac * sbb - sab * sbc) * idet, hh = (saa * sbc - sab * sac) * idet;
    const double kk = me - gg * mr - hh * mx;
    const double S = sqrt(fmax(0.0, 1.0 + hh * hh - 4.0 * gg * kk));
    f.kappa = 2.0 * gg / S;
    // residual and error projection of this lane's point (as in fit_track with Pf)
    double term = 0.0;
    {
        const float gf = float(gg), hf = float(hh), Sf = float(S), xxf = float(xx), xyf = float(xy);
        const float uf = float(gg * rho2 + hh * xi + kk - et);
        const float e = 2.f * uf / (Sf + sqrtf(fmaxf(0.f, Sf * Sf + 4.f * gf * uf)));
        if (Qf.sr > 0.f) {
            const double nlx = 2.0 * gg * xi + hh, nly = 2.0 * gg * et - 1.0;
            const double nx = nlx * xx - nly * xy, ny = nlx * xy + nly * xx;
            const double nn2 = nx * nx + ny * ny;
            const double ir = 1.0 / Q.r;
            const double rx = Q.x * ir, ry = Q.y * ir;
            const double n_phi = ny * rx - nx * ry, n_r = nx * rx + ny * ry;
            const double s2 = fmax(sq(Q.srphi * n_phi) + sq(Q.sr * n_r), sq(0.01 * Q.srphi) * nn2);
            term = double(e) * double(e) * nn2 / s2;
        } else {
            const float dxf = Qf.x - oxf, dyf = Qf.y - oyf;
            const float xif = dxf * xxf + dyf * xyf, etf = dyf * xxf - dxf * xyf;
            const float nlx = 2.f * gf * xif + hf, nly = 2.f * gf * etf - 1.f;
            const float nx = nlx * xxf - nly * xyf, ny = nlx * xyf + nly * xxf;
            const float nn2 = nx * nx + ny * ny;
            const float ir = 1.f / Qf.r;
            const float rx = Qf.x * ir, ry = Qf.y * ir;
            const float n_phi = ny * rx - nx * ry;
            const float s2 = fmaxf(sq(Qf.srphi * n_phi), sq(0.01f * Qf.srphi) * nn2);
            term = double(e * e * nn2 / s2);
        }
    }
    f.chi2_rphi = grp_sum8(act ? term : 0.0);
    const double ka = fabs(f.kappa);
    const double sj = arc(sqrt(sq(Q.x - x0) + sq(Q.y - y0)), ka);
    const double sn = __shfl_sync(F, sj, N - 1, 8);
    const double t_hat = (zn - z0) / sn;
    const float tf = float(t_hat);
    const double w = act ? double(1.f / fmaxf(1e-12f, sq(Qf.sz) + sq(tf * Qf.sr))) : 0.0;
    const double W = grp_sum8(w), Ws = grp_sum8(w * sj), Wz = grp_sum8(w * Q.z);
    const double iW = 1.0 / W;
    const double sbar = Ws * iW, zbar = Wz * iW;
    const double Sss = grp_sum8(w * sq(sj - sbar)), Ssz = grp_sum8(w * (sj - sbar) * (Q.z - zbar));
    const double t = Ssz / Sss, c0 = zbar - t * sbar;
    f.chi2_rz = grp_sum8(w * sq(Q.z - c0 - t * sj));
    f.tanl = t;
    return f;
}

// Sum over a group of 8 lanes (float-float)
__device__ __forceinline__ ff grp_sum8(ff v) {
#pragma unroll
    for (int d = 4; d; d >>= 1)
        v = v + ff{__shfl_xor_sync(0xffffffffu, v.hi, d, 8), __shfl_xor_sync(0xffffffffu, v.lo, d, 8)};
    return v;
}
__device__ __forceinline__ float grp_sum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
    return v;
}

// fit_track_ff with one candidate per group of 8 lanes, lane j holding point j
// (j < N); every lane of the group returns the fit. For kernels with few
// candidates, where a thread per candidate leaves the dependent float-float
// chain exposed. All 32 lanes must call.
template <int N> __device__ inline Fit fit_track_group_ff(const Pt<float>& Q, int j) {
    static_assert(N <= 8, "one point per lane of a group of 8");
    const unsigned F = 0xffffffffu;
    const bool act = j < N;
    const ff zero{0.f, 0.f};
    Fit f;
    const float x0 = __shfl_sync(F, Q.x, 0, 8), y0 = __shfl_sync(F, Q.y, 0, 8), z0 = __shfl_sync(F, Q.z, 0, 8);
    const float xn = __shfl_sync(F, Q.x, N - 1, 8), yn = __shfl_sync(F, Q.y, N - 1, 8);
    const float zn = __shfl_sync(F, Q.z, N - 1, 8);
    const float ox = __shfl_sync(F, Q.x, N / 2, 8), oy = __shfl_sync(F, Q.y, N / 2, 8);
    const ff ex = two_sum(xn, -x0), ey = two_sum(yn, -y0);
    const ff L2 = ex * ex + ey * ey;
    const ff dx = two_sum(Q.x, -ox), dy = two_sum(Q.y, -oy);
    const ff xi = dx * ex + dy * ey, et = dy * ex - dx * ey, rho2 = (dx * dx + dy * dy) * L2;
    const ff mr = grp_sum8(act ? rho2 : zero) / float(N), mx = grp_sum8(act ? xi : zero) / float(N);
    const ff me = grp_sum8(act ? et : zero) / float(N);
    const ff ca = act ? rho2 - mr : zero, cb = act ? xi - mx : zero, cc = act ? et - me : zero;
    const ff saa = grp_sum8(ca * ca), sab = grp_sum8(ca * cb), sbb = grp_sum8(cb * cb);
    const ff sac = grp_sum8(ca * cc), sbc = grp_sum8(cb * cc);
    const ff det = saa * sbb - sab * sab;
    if (!(det.hi > 0.f)) {
        f.kappa = 1e30; f.chi2_rphi = 1e30; f.chi2_rz = 1e30; f.tanl = 0;
        return f;
    }
    const ff gg = (sac * sbb - sab * sbc) / det, hh = (saa * sbc - sab * sac) / det;
    const ff kk = me - gg * mr - hh * mx;
    const ff S = ff_sqrt(hh * hh + 1.f - gg * kk * 4.f);
    const ff L = ff_sqrt(L2);
    const ff kappa = gg * L * 2.f / S;
    f.kappa = ff_d(kappa);
    const float term = act ? ff_rphi_term(Q, xi, et, rho2, gg, hh, kk, ex, ey, S.hi, 1.f / L.hi) : 0.f;
    f.chi2_rphi = grp_sum8(term);
    const ff cx = two_sum(Q.x, -x0), cy = two_sum(Q.y, -y0);
    const ff sj = ff_arc(ff_sqrt(cx * cx + cy * cy), ff_abs(kappa));
    const float sn = __shfl_sync(F, sj.hi, N - 1, 8);
    const float t_hat = (zn - z0) / sn;
    const float w = act ? 1.f / fmaxf(1e-12f, sq(Q.sz) + sq(t_hat * Q.sr)) : 0.f;
    const ff W = grp_sum8(ff{w, 0.f}), Ws = grp_sum8(sj * w), Wz = grp_sum8(two_prod(w, Q.z));
    const ff sbar = Ws / W, zbar = Wz / W;
    const ff ds = sj - sbar, dz = ff_of(Q.z) - zbar;
    const ff Sss = grp_sum8(ds * ds * w), Ssz = grp_sum8(ds * dz * w);
    const ff t = Ssz / Sss, c0 = zbar - t * sbar;
    const float r = (ff_of(Q.z) - c0 - t * sj).hi;
    f.chi2_rz = grp_sum8(w * r * r);
    f.tanl = ff_d(t);
    return f;
}

// Square root through the approximate reciprocal square root (a few ulp;
// the FP32 prefilters carry far larger slack); 0 for x <= 0.
__device__ __forceinline__ float fast_sqrtf(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// FP32 twin of fit_track (same chord-frame circle fit, geometric residuals and
// r-z line fit), evaluated cut by cut: the curvature is tested right after the
// circle solve, chi2_rphi after the residuals, and the r-z fit runs only for
// candidates that passed both. The verdict equals testing all three at the end.
// Divisions and square roots are the approximate ones (__fdividef, rsqrtf: a
// few ulp each), well inside the slack of the limits (prefit_limits).
template <int N> __device__ inline bool fit_may_pass_f32(const Pt<float>* P, const FitLimits& L) {
    const Pt<float>& O = P[N / 2];
    float ex = P[N - 1].x - P[0].x, ey = P[N - 1].y - P[0].y;
    float il = rsqrtf(ex * ex + ey * ey);
    float xx = ex * il, xy = ey * il, yx = -xy, yy = xx;
    float xi[N], et[N], rho2[N];
    float mr = 0.f, mx = 0.f, me = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float dx = P[i].x - O.x, dy = P[i].y - O.y;
        xi[i] = dx * xx + dy * xy;
        et[i] = dx * yx + dy * yy;
        rho2[i] = xi[i] * xi[i] + et[i] * et[i];
        mr += rho2[i]; mx += xi[i]; me += et[i];
    }
    mr *= 1.0f / N; mx *= 1.0f / N; me *= 1.0f / N;
    float saa = 0.f, sab = 0.f, sbb = 0.f, sac = 0.f, sbc = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float a = rho2[i] - mr, b = xi[i] - mx, cc = et[i] - me;
        saa += a * a; sab += a * b; sbb += b * b; sac += a * cc; sbc += b * cc;
    }
    float det = saa * sbb - sab * sab;
    if (!(det > 0.f)) return false;
    const float idet = __fdividef(1.f, det);
    float gg = (sac * sbb - sab * sbc) * idet;
    float hh = (saa * sbc - sab * sac) * idet;
    float kk = me - gg * mr - hh * mx;
    float S = fast_sqrtf(1.f + hh * hh - 4.f * gg * kk);
    float kappa = __fdividef(2.f * gg, S);
    if (!(fabsf(kappa) <= L.kappa)) return false;
    float c2 = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float u = gg * rho2[i] + hh * xi[i] + kk - et[i];
        float e = __fdividef(2.f * u, S + fast_sqrtf(S * S + 4.f * gg * u));
        float nlx = 2.f * gg * xi[i] + hh, nly = 2.f * gg * et[i] - 1.f;
        float nx = nlx * xx + nly * yx, ny = nlx * xy + nly * yy;
        float inn = rsqrtf(nx * nx + ny * ny);
        nx *= inn; ny *= inn;
        float ir = __fdividef(1.f, P[i].r);
        float rx = P[i].x * ir, ry = P[i].y * ir;
        float n_phi = -nx * ry + ny * rx, n_r = nx * rx + ny * ry;
        float s2 = fmaxf(sq(P[i].srphi * n_phi) + sq(P[i].sr * n_r), sq(0.01f * P[i].srphi));
        c2 += __fdividef(e * e, s2);
    }
    if (!(c2 <= L.chi2)) return false;
    float ka = fabsf(kappa);
    float s[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float c = fast_sqrtf(sq(P[i].x - P[0].x) + sq(P[i].y - P[0].y));
        s[i] = ka > 0.f ? __fdividef(2.f * asinf(fminf(1.f, 0.5f * c * ka)), ka) : c;
    }
    float t_hat = __fdividef(P[N - 1].z - P[0].z, s[N - 1]);
    float w[N], W = 0.f, Ws = 0.f, Wz = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        w[i] = __fdividef(1.f, fmaxf(1e-12f, sq(P[i].sz) + sq(t_hat * P[i].sr)));
        W += w[i]; Ws += w[i] * s[i]; Wz += w[i] * P[i].z;
    }
    const float iW = __fdividef(1.f, W);
    float sbar = Ws * iW, zbar = Wz * iW, Sss = 0.f, Ssz = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        Sss += w[i] * sq(s[i] - sbar);
        Ssz += w[i] * (s[i] - sbar) * (P[i].z - zbar);
    }
    float t = __fdividef(Ssz, Sss), c0 = zbar - t * sbar, cz = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) cz += w[i] * sq(P[i].z - c0 - t * s[i]);
    return cz <= L.chi2z;
}

__device__ __forceinline__ double phi0_of(const Pt<double>& P, double kappa) {
    double s = kappa < 0 ? -1.0 : 1.0;
    return wrap_pi(atan2(P.y, P.x) - s * asinc(P.r * fabs(kappa) / 2.0));
}

__device__ __forceinline__ double pt_of(const DevCfg& c, double kappa) {
    double ka = fabs(kappa);
    return ka > 0 ? c.k_field * c.b_field / (100.0 * ka) : 1e30;
}

// Scoring features of a T5 candidate (FP64, stored as FP32): hits H[0..9] =
// (lower, upper) of the five MDs, P[0..4] = the lower hits (anchors), layer
// codes (layer + 6 subdet). f[0..9] r-phi pulls of the ten hits to the fitted
// circle, f[10..19] r-z pulls to the fitted line (both clipped to +-50),
// f[20..24] anchor radii / 100, f[25..27] inner, outer and fitted curvature
// over 2a, f[28..29] log(1 + chi2) (r-phi, r-z), f[30..31] 10 beta of the two
// triplets, f[32] eta, f[33..37] layer codes / 11, f[38..47] zero.
__device__ inline void t5_features(const DevCfg& c, const Pt<double>* P, const Pt<double>* H, const int* code,
                                   float* f) {
    FitFull F;
    fit_track<5>(P, &F);
    Tri<double> ti = tri(P[0], P[1], P[2]);
    Tri<double> to = tri(P[2], P[3], P[4]);
    const double ka = fabs(F.kappa);
    const double yx = -F.xy, yy = F.xx;
    for (int j = 0; j < 10; ++j) {
        const Pt<double>& Q = H[j];
        double dx = Q.x - F.ox, dy = Q.y - F.oy;
        double xi = dx * F.xx + dy * F.xy, et = dx * yx + dy * yy;
        double rho2 = xi * xi + et * et;
        double u = F.gg * rho2 + F.hh * xi + F.kk - et;
        double e = 2.0 * u / (F.S + sqrt(fmax(0.0, F.S * F.S + 4.0 * F.gg * u)));
        double nlx = 2.0 * F.gg * xi + F.hh, nly = 2.0 * F.gg * et - 1.0;
        double nx = nlx * F.xx + nly * yx, ny = nlx * F.xy + nly * yy;
        double nn = hypot(nx, ny);
        nx /= nn;
        ny /= nn;
        double rx = Q.x / Q.r, ry = Q.y / Q.r;
        double s2 = fmax(sq(Q.srphi * (-nx * ry + ny * rx)) + sq(Q.sr * (nx * rx + ny * ry)), sq(0.01 * Q.srphi));
        double pr = e / sqrt(s2);
        double sj = arc(hypot(Q.x - P[0].x, Q.y - P[0].y), ka);
        double w = 1.0 / fmax(1e-12, sq(Q.sz) + sq(F.t_hat * Q.sr));
        double pz = (Q.z - F.c0 - F.t * sj) * sqrt(w);
        f[j] = float(fmin(50.0, fmax(-50.0, pr)));
        f[10 + j] = float(fmin(50.0, fmax(-50.0, pz)));
    }
    for (int j = 0; j < 5; ++j) f[20 + j] = float(P[j].r / 100.0);
    const double two_a = 2.0 * c.a;
    f[25] = float(ti.kappa / two_a);
    f[26] = float(to.kappa / two_a);
    f[27] = float(F.kappa / two_a);
    f[28] = float(log1p(fmin(F.chi2, 1e30)));
    f[29] = float(log1p(fmin(F.chi2z, 1e30)));
    f[30] = float(10.0 * ti.beta);
    f[31] = float(10.0 * to.beta);
    f[32] = float(asinh(F.t));
    for (int j = 0; j < 5; ++j) f[33 + j] = float(code[j] / 11.0);
    for (int j = 38; j < 48; ++j) f[j] = 0.f;
}

// FP32 chord-frame fit of N points with every output (the same algebra as
// fit_track, no early exit): the triplet features' fit. IEEE division and
// square root; FP32 is ample for features the network reads in BF16.
struct FitF {
    float gg, hh, kk, S, xx, xy, ox, oy, c0, t, t_hat, kappa, chi2, chi2z;
};
template <int N> __device__ inline FitF fit_f32(const Pt<float>* P) {
    FitF F;
    const Pt<float>& O = P[N / 2];
    const float ex = P[N - 1].x - P[0].x, ey = P[N - 1].y - P[0].y;
    const float il = 1.f / sqrtf(ex * ex + ey * ey);
    const float xx = ex * il, xy = ey * il;
    float xi[N], et[N], rho2[N], mr = 0.f, mx = 0.f, me = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float dx = P[i].x - O.x, dy = P[i].y - O.y;
        xi[i] = dx * xx + dy * xy;
        et[i] = dy * xx - dx * xy;
        rho2[i] = xi[i] * xi[i] + et[i] * et[i];
        mr += rho2[i]; mx += xi[i]; me += et[i];
    }
    mr *= 1.f / N; mx *= 1.f / N; me *= 1.f / N;
    float saa = 0.f, sab = 0.f, sbb = 0.f, sac = 0.f, sbc = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float a = rho2[i] - mr, b = xi[i] - mx, cc = et[i] - me;
        saa += a * a; sab += a * b; sbb += b * b; sac += a * cc; sbc += b * cc;
    }
    const float det = saa * sbb - sab * sab;
    F.xx = xx; F.xy = xy; F.ox = O.x; F.oy = O.y;
    if (!(det > 0.f)) {
        F.gg = F.hh = F.kk = 0.f; F.S = 1.f; F.kappa = 0.f; F.chi2 = F.chi2z = 1e30f; F.c0 = F.t = F.t_hat = 0.f;
        return F;
    }
    F.gg = (sac * sbb - sab * sbc) / det;
    F.hh = (saa * sbc - sab * sac) / det;
    F.kk = me - F.gg * mr - F.hh * mx;
    F.S = sqrtf(fmaxf(0.f, 1.f + F.hh * F.hh - 4.f * F.gg * F.kk));
    F.kappa = 2.f * F.gg / F.S;
    float chi2 = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float u = F.gg * rho2[i] + F.hh * xi[i] + F.kk - et[i];
        const float e = 2.f * u / (F.S + sqrtf(fmaxf(0.f, F.S * F.S + 4.f * F.gg * u)));
        const float nlx = 2.f * F.gg * xi[i] + F.hh, nly = 2.f * F.gg * et[i] - 1.f;
        const float nx = nlx * xx - nly * xy, ny = nlx * xy + nly * xx;
        const float nn2 = nx * nx + ny * ny;
        const float rx = P[i].x / P[i].r, ry = P[i].y / P[i].r;
        const float n_phi = ny * rx - nx * ry, n_r = nx * rx + ny * ry;
        const float s2 = fmaxf(sq(P[i].srphi * n_phi) + sq(P[i].sr * n_r), sq(0.01f * P[i].srphi) * nn2);
        chi2 += e * e * nn2 / s2;
    }
    F.chi2 = chi2;
    const float ka = fabsf(F.kappa);
    float s[N], w[N], W = 0.f, Ws = 0.f, Wz = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) s[i] = arc(sqrtf(sq(P[i].x - P[0].x) + sq(P[i].y - P[0].y)), ka);
    F.t_hat = (P[N - 1].z - P[0].z) / s[N - 1];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        w[i] = 1.f / fmaxf(1e-12f, sq(P[i].sz) + sq(F.t_hat * P[i].sr));
        W += w[i]; Ws += w[i] * s[i]; Wz += w[i] * P[i].z;
    }
    const float sbar = Ws / W, zbar = Wz / W;
    float Sss = 0.f, Ssz = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        Sss += w[i] * sq(s[i] - sbar);
        Ssz += w[i] * (s[i] - sbar) * (P[i].z - zbar);
    }
    F.t = Ssz / Sss;
    F.c0 = zbar - F.t * sbar;
    float cz = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) cz += w[i] * sq(P[i].z - F.c0 - F.t * s[i]);
    F.chi2z = cz;
    return F;
}

// Scoring features of a T3 (FP32), in the T5's slots with the missing ones
// zero: hits H[0..5] = (lower, upper) of the three MDs, anchors P = the lower
// hits. f[0..5] r-phi pulls of the six hits to the anchors' circle, f[10..15]
// r-z pulls to the fitted line (both clipped to +-50), f[20..22] anchor
// radius / 100, f[25] the triplet's curvature / 2a, f[27] the fit's,
// f[28..29] log(1 + chi2_rphi), log(1 + chi2_rz), f[30] 10 x beta, f[32] eta,
// f[33..35] layer code / 11; every other slot 0.
__device__ inline void t3_features(const DevCfg& c, const Pt<float>* P, const Pt<float>* H, const int* code,
                                   float (&v)[48]) {
    const FitF F = fit_f32<3>(P);
    const Tri<float> t = tri(P[0], P[1], P[2]);
    const float ka = fabsf(F.kappa);
#pragma unroll
    for (int j = 0; j < 48; ++j) v[j] = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const Pt<float>& Q = H[j];
        const float dx = Q.x - F.ox, dy = Q.y - F.oy;
        const float xi = dx * F.xx + dy * F.xy, et = dy * F.xx - dx * F.xy;
        const float u = F.gg * (xi * xi + et * et) + F.hh * xi + F.kk - et;
        const float e = 2.f * u / (F.S + sqrtf(fmaxf(0.f, F.S * F.S + 4.f * F.gg * u)));
        const float nlx = 2.f * F.gg * xi + F.hh, nly = 2.f * F.gg * et - 1.f;
        const float nx = nlx * F.xx - nly * F.xy, ny = nlx * F.xy + nly * F.xx;
        const float nn2 = nx * nx + ny * ny;
        const float rx = Q.x / Q.r, ry = Q.y / Q.r;
        const float n_phi = ny * rx - nx * ry, n_r = nx * rx + ny * ry;
        const float s2 = fmaxf(sq(Q.srphi * n_phi) + sq(Q.sr * n_r), sq(0.01f * Q.srphi) * nn2) / nn2;
        v[j] = fminf(50.f, fmaxf(-50.f, e / sqrtf(s2)));
        const float sj = arc(sqrtf(sq(Q.x - P[0].x) + sq(Q.y - P[0].y)), ka);
        const float w = 1.f / fmaxf(1e-12f, sq(Q.sz) + sq(F.t_hat * Q.sr));
        v[10 + j] = fminf(50.f, fmaxf(-50.f, (Q.z - F.c0 - F.t * sj) * sqrtf(w)));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) v[20 + j] = P[j].r / 100.f;
    const float two_a = 2.f * c.f.a;
    v[25] = t.kappa / two_a;
    v[27] = F.kappa / two_a;
    v[28] = log1pf(fminf(F.chi2, 1e30f));
    v[29] = log1pf(fminf(F.chi2z, 1e30f));
    v[30] = 10.f * t.beta;
    v[32] = asinhf(F.t);
#pragma unroll
    for (int j = 0; j < 3; ++j) v[33 + j] = code[j] / 11.f;
}

// Inputs of the scoring features of T3 i: anchors P (the MDs' lower hits),
// hits H (lower, upper of each MD) and layer codes (layer, +6 on a 2S module).
__device__ inline void t3_feature_inputs(const Arena& A, int i, Pt<float>* P, Pt<float>* H, int* code) {
    const int4 q = A.t3_md[i];
    const int m[3] = {q.x, q.y, q.z};
    const int h0 = A.hit_off[A.md_gmod[m[0]] / A.n_mod];
    const BatchDesc* B = A.bd;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        P[j] = md_point<float>(A, m[j]);
        H[2 * j] = P[j];
        Pt<float> U = P[j];
        const int hu = h0 + A.md_up[m[j]];
        U.x = B->hx[hu];
        U.y = B->hy[hu];
        U.z = B->hz[hu];
        U.r = sqrtf(U.x * U.x + U.y * U.y);
        H[2 * j + 1] = U;
        const int mod = A.md_gmod[m[j]] % A.n_mod;
        code[j] = A.mod_layer[mod] + (A.mod[mod].w > 0.5f ? 6 : 0);
    }
}

// T5 on anchors P[0..4]; outputs in double
struct T5Out {
    double kappa, chi2_rphi, chi2_rz, eta, phi0, pt, score, sigk;
};

// Curvature consistency |k1 - k2| <= n sqrt(s1^2 + s2^2) on FP32 inputs: 1 or
// 0 when the FP32 values are farther from the threshold than their rounding
// can move them (a band of 2e-3 of the threshold), -1 (undecided) otherwise.
__device__ __forceinline__ int kappa_test_f32(float k1, float s1, float k2, float s2, float n) {
    const float d = fabsf(k1 - k2), thr = n * fast_sqrtf(s1 * s1 + s2 * s2);
    const float band = 2e-3f * thr + 1e-7f;
    if (d < thr - band) return 1;
    if (d > thr + band) return 0;
    return -1;
}

// The FP64 twin of an FP32 point: the coordinates convert exactly and r is
// recomputed in FP64, as md_point<double> does.
__device__ __forceinline__ Pt<double> pt_f64(const Pt<float>& q) {
    Pt<double> p;
    p.x = q.x; p.y = q.y; p.z = q.z;
    p.r = m_hypot(p.x, p.y);
    p.srphi = q.srphi; p.sz = q.sz; p.sr = q.sr;
    return p;
}

// FP64 curvature consistency of a T5's two triplets, recomputed from the
// anchors Pf[0..4] (for a test the stored FP32 curvatures leave undecided);
// sigk receives the T5's curvature error.
__device__ inline bool t5_kc_fp64(const DevCfg& c, const Pt<float>* Pf, double& sigk) {
    const Pt<double> P0 = pt_f64(Pf[0]), P1 = pt_f64(Pf[1]), P2 = pt_f64(Pf[2]);
    const Pt<double> P3 = pt_f64(Pf[3]), P4 = pt_f64(Pf[4]);
    const Tri<double> ti = tri(P0, P1, P2), to = tri(P2, P3, P4);
    sigk = 0.5 * sqrt(sq(ti.sigk) + sq(to.sigk));
    return fabs(ti.kappa - to.kappa) <= c.n_t5 * sqrt(sq(ti.sigk) + sq(to.sigk));
}

// A T5's verdict and outputs from its fit f, its curvature consistency kc and
// its first anchor P0 (o.sigk already set). all_outputs = false leaves the
// outputs of a candidate that fails kc at zero and skips eta, phi0 and pT of
// a rejected one.
__device__ inline bool t5_finish(const DevCfg& c, const Pt<float>& P0, const Fit& f, bool kc, bool all_outputs,
                                 T5Out& o) {
    if (!kc && !all_outputs) return false;
    o.kappa = f.kappa;
    o.chi2_rphi = f.chi2_rphi;
    o.chi2_rz = f.chi2_rz;
    o.score = f.chi2_rphi + f.chi2_rz;
    const bool pass = kc && fabs(f.kappa) <= (1.0 + c.tol_r) * 2.0 * c.a && f.chi2_rphi <= c.chi2_rphi_t5 &&
                      f.chi2_rz <= c.chi2_rz_t5;
    if (pass || all_outputs) {
        // direction in FP32 (well conditioned; ~1e-7 rad): eta from the fitted
        // r-z slope, phi0 from the first anchor and the fitted curvature
        o.eta = double(asinhf(float(f.tanl)));
        const float kf = float(f.kappa);
        const float turn = asinf(fminf(1.f, fmaxf(0.f, P0.r * fabsf(kf) * 0.5f)));
        float ph = atan2f(P0.y, P0.x) - (kf < 0.f ? -turn : turn);
        if (ph > float(kPi)) ph -= float(2 * kPi);
        if (ph <= -float(kPi)) ph += float(2 * kPi);
        o.phi0 = double(ph);
        o.pt = pt_of(c, f.kappa);
    }
    return pass;
}

// T5 on anchors Pf[0..4]; the two triplets' curvatures (k, s) come from the
// T3 arrays (FP32) and decide the consistency test unless it is undecided, in
// which case both triplets are recomputed in FP64. The fit is float-float, or
// FP64 with c.fp64_fit.
__device__ inline bool t5_eval(const DevCfg& c, const Pt<float>* Pf, float k1, float s1, float k2, float s2,
                               bool all_outputs, T5Out& o) {
    o = T5Out{};
    o.sigk = 0.5 * sqrt(sq(double(s1)) + sq(double(s2)));
    int kc = kappa_test_f32(k1, s1, k2, s2, c.f.n_t5);
    if (kc < 0) kc = t5_kc_fp64(c, Pf, o.sigk);
    if (!kc && !all_outputs) return false;
    Fit f;
    if (c.fp64_fit) {
        Pt<double> P[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) P[j] = pt_f64(Pf[j]);
        f = fit_track<5>(P, nullptr, Pf);
    } else {
        f = fit_track_ff<5>(Pf);
    }
    return t5_finish(c, Pf[0], f, kc != 0, all_outputs, o);
}

struct PTOut {
    double kappa, chi2_rphi, chi2_rz, score, pt;
};

// pT5 / pT3 with the curvature-consistency verdict kc decided by the caller;
// the fit is float-float, or FP64 on P with c.fp64_fit (P is read only then).
template <int N>
__device__ inline bool pt_eval(const DevCfg& c, const Pt<double>* P, const Pt<float>* Pf, bool kc,
                               double chi2_rphi_max, double chi2_rz_max, PTOut& o) {
    o = PTOut{};
    if (!kc) return false;
    const Fit f = c.fp64_fit ? fit_track<N>(P, nullptr, Pf) : fit_track_ff<N>(Pf);
    o.kappa = f.kappa;
    o.chi2_rphi = f.chi2_rphi;
    o.chi2_rz = f.chi2_rz;
    o.score = f.chi2_rphi + f.chi2_rz;
    o.pt = pt_of(c, f.kappa);
    if (!(fabs(f.kappa) <= (1.0 + c.tol_r) * 2.0 * c.a)) return false;
    if (!(f.chi2_rphi <= chi2_rphi_max)) return false;
    if (!(f.chi2_rz <= chi2_rz_max)) return false;
    return true;
}

// ---------------------------------------------------------------------------
// small device utilities
// ---------------------------------------------------------------------------
// ---- compact (16-bit) storage ---------------------------------------------
// A triplet's stored (curvature, sigma) as the T5 and pT3 searches read it:
// FP32, or the FP16 copy scaled by 1/(2a) (|kappa| / 2a <= 1 + tol for a
// triplet, so the copy stays in FP16's normal range). A search prefilter that
// reads the copy widens its slack by ks_slack: each FP16 value is within
// 2^-11 of its FP32 value (relative), subnormals within 1e-9 absolute after
// rescaling, both far inside 1e-3 relative plus the 1e-7 absolute term.
__device__ __forceinline__ float2 t3_ks_search(const Arena& A, int t) {
    if (!A.compact) return A.t3_ks[t];
    const float2 v = __half22float2(A.t3_ksh[t]);
    return make_float2(v.x * A.two_a, v.y * A.two_a);
}
__device__ __forceinline__ float ks_slack(const Arena& A) { return A.compact ? 1e-3f : 1e-5f; }

// Curvature window of the searches' prefilter |k - kt| <= 1.01 n sqrt(s^2 + st^2) + rel (|k| + |kt|) + 1e-7
// against objects whose sigma st is at most smax: with sqrt(s^2 + st^2) <= s + st and |kt| <= |k| + |k - kt|,
// every kt that can pass lies within the returned w of k (the factors 1.001 and 1e-7 cover the FP32 rounding
// of both sides).
__device__ __forceinline__ float ks_window(float k, float s, float smax, float n, float rel) {
    return (1.01f * n * (s + smax) + 2.f * rel * fabsf(k) + 1e-7f) / (1.f - rel) * 1.001f + 1e-7f;
}

// First position in [lo, hi) of curvature-ordered (curvature, sigma) pairs whose curvature is >= x (> x with
// upper).
__device__ __forceinline__ int ks_bound(const float2* ks, int lo, int hi, float x, bool upper) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float v = ks[mid].x;
        if (upper ? !(v > x) : (v < x)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Fixed-point eta-phi: 1e-4 per step in eta (|eta| < 3.2767) and pi / 32767
// in phi; an eta outside that range is stored as the sentinel -32768, which
// the list scan always re-tests in FP64.
constexpr float kEtaQ = 1e-4f;
constexpr float kPhiQ = 3.14159265358979f / 32767.f;
__device__ __forceinline__ unsigned pack_eta_phi(float eta, float phi) {
    const float qe = eta / kEtaQ;
    const int ie = fabsf(qe) < 32767.f ? __float2int_rn(qe) : -32768;
    const int ip = max(-32767, min(32767, __float2int_rn(phi / kPhiQ)));
    return (unsigned(ie) & 0xffffu) | (unsigned(ip) << 16);
}
__device__ __forceinline__ float2 unpack_eta_phi(unsigned q, bool& sentinel) {
    const int ie = int(short(q & 0xffffu)), ip = int(short(q >> 16));
    sentinel = ie == -32768;
    return make_float2(float(ie) * kEtaQ, float(ip) * kPhiQ);
}

__device__ __forceinline__ int event_of(const int* off, int n_ev, int i) {
    int lo = 0, hi = n_ev;            // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// exclusive prefix of `flag` across the warp, and the warp total
__device__ __forceinline__ int warp_rank(bool flag, int& total) {
    unsigned m = __ballot_sync(0xffffffffu, flag);
    total = __popc(m);
    return __popc(m & ((1u << lane_id()) - 1u));
}

}  // namespace lst
