// Pixel-seeded objects (pLS, pT5, pT3) and the cross-cleaning that forms the
// track-candidate collection (Section 2.1; pT5 is launched before pT3, as in
// Fig. KernelFlow).
#include "lst_kernels.cuh"
#include "lst_warp.cuh"

namespace lst {

// ---------------------------------------------------------------------------
// pLS: one thread per seed, FP64 (three-point circle, r-z line, superbin)
// ---------------------------------------------------------------------------
__global__ void k_pls(Arena A, DevCfg c) {
    pdl_begin();
    const BatchDesc B = *A.bd;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < B.n_seeds; g += gridDim.x * blockDim.x) {
        const float* q = B.seeds + 9 * (size_t)g;
        Pt<double> Q[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) Q[j] = pix_pt<double>(q + 3 * j, c.sig_pix);
        Tri<double> t = tri(Q[0], Q[1], Q[2]);
        double ka = fabs(t.kappa);
        double s1 = arc(t.lu, ka), s2 = arc(t.lw, ka);
        double sbar = (s1 + s2) / 3.0, zbar = (Q[0].z + Q[1].z + Q[2].z) / 3.0;
        double Sss = sq(0.0 - sbar) + sq(s1 - sbar) + sq(s2 - sbar);
        double Ssz = (0.0 - sbar) * (Q[0].z - zbar) + (s1 - sbar) * (Q[1].z - zbar) + (s2 - sbar) * (Q[2].z - zbar);
        double tanl = Ssz / Sss;
        double zc = zbar - tanl * sbar;
        double z0 = zc - tanl * arc(Q[0].r, ka);
        double eta = asinh(tanl);
        double phi0 = phi0_of(Q[0], t.kappa);
        bool pass = (ka <= 2.0 * c.a / (1.0 - c.pls_pt_tol)) && (fabs(z0) <= c.z_lumi);
        double de = 2.0 * c.sb_eta_max / c.sb_n_eta;
        double dp = 2.0 * kPi / c.sb_n_phi;
        long ie = (long)floor((eta + c.sb_eta_max) / de);
        long ip = (long)floor((phi0 + kPi) / dp);
        ip = ip < 0 ? 0 : (ip > c.sb_n_phi - 1 ? c.sb_n_phi - 1 : ip);
        int iq = t.kappa < 0 ? 1 : 0;
        int sb = (ie >= 0 && ie < c.sb_n_eta) ? (int)((ie * c.sb_n_phi + ip) * 2 + iq) : -1;
        A.pls_pass[g] = pass;
        A.pls_sb[g] = sb;
        A.pls_kappa[g] = t.kappa;
        A.pls_sigk[g] = t.sigk;
        A.pls_z0[g] = float(z0);
        A.pls_pt[g] = float(pt_of(c, t.kappa));
        A.pls_eta[g] = eta;
        A.pls_phi[g] = phi0;
        if (pass) {
            int e = event_of(A.seed_off, B.n_ev, g);
            atomic_add_agg(&A.ev_counts[e * 8 + 4], 1);
        }
    }
}

// ---------------------------------------------------------------------------
// pT5 / pT3: candidates of a passing seed = T objects whose inner MD sits in
// a module listed under the seed's superbin.
// ---------------------------------------------------------------------------
struct PtSmem {
    int pre[32], off[32], pre2[32], off2[32];
    int cand[kPtPre];
    int stage[kPtStage];
};

template <int NT>
__device__ __forceinline__ void pt_mds(const Arena& A, int obj, int* m) {
    if (NT == 5) {
        int a = A.t5_in[obj], b = A.t5_out[obj];
        const int4 ta = A.t3_md[a], tb = A.t3_md[b];
        m[0] = ta.x; m[1] = ta.y; m[2] = ta.z; m[3] = tb.y; m[4] = tb.z;
    } else {
        const int4 t = A.t3_md[obj];
        m[0] = t.x; m[1] = t.y; m[2] = t.z;
    }
}

template <int NT>
__device__ __forceinline__ bool pt_prefit_f32(const Arena& A, const DevCfg& c, int g, int obj) {
    Pt<float> P[NT + 3];
    const float* sd = A.bd->seeds + 9 * (size_t)g;
#pragma unroll
    for (int j = 0; j < 3; ++j) P[j] = pix_pt<float>(sd + 3 * j, c.f.sig_pix);
    int m[NT];
    pt_mds<NT>(A, obj, m);
#pragma unroll
    for (int j = 0; j < NT; ++j) P[3 + j] = md_point<float>(A, m[j]);
    return fit_may_pass_f32<NT + 3>(P, NT == 5 ? c.lim_pt5 : c.lim_pt3);
}

// FP32 fit verdicts of one group of 32 candidates (one out-of-line copy).
template <int NT>
__device__ __noinline__ unsigned pt_prefit_group(const Arena& A, const DevCfg& c, int g, const int* cand, int q, int n) {
    bool keep = q < n && pt_prefit_f32<NT>(A, c, g, cand[q]);
    return __ballot_sync(kFull, keep);
}

// Collected candidates: FP32 fit prefilter; sink(keep, obj, rank, total) per
// group of 32, in candidate order.
template <int NT, typename Sink>
__device__ __forceinline__ void pt_flush(const Arena& A, const DevCfg& c, PtSmem& S, int g, int ncand, Sink& sink) {
    const int lane = lane_id();
    for (int base = 0; base < ncand; base += 32) {
        int q = base + lane;
        unsigned m = pt_prefit_group<NT>(A, c, g, S.cand, q, ncand);
        bool keep = (m >> lane) & 1u;
        int r = __popc(m & ((1u << lane) - 1u));
        sink(keep, q < ncand ? S.cand[q] : 0, r, __popc(m));
    }
    __syncwarp();
}

// Candidates of seed g (event e) among the T objects whose inner MD sits in
// the superbin modules sb_tgt[j_begin .. j_end) (at most 32), in a fixed
// order (module, MD, object): curvature prefilter, FP32 fit prefilter, then
// the sink. Two levels of flattening keep the lanes busy: modules -> MDs,
// then each group of 32 MDs -> their T objects.
template <int NT, typename Sink>
__device__ __forceinline__ void pt_enumerate(const Arena& A, const DevCfg& c, PtSmem& S, int g, int e, int j_begin,
                                             int j_end, Sink& sink) {
    const int lane = lane_id();
    const float nk = float(c.n_pt);
    const float kp = float(A.pls_kappa[g]), sp = float(A.pls_sigk[g]);
    int ncand = 0;
    int moff = 0, mcnt = 0;
    if (j_begin + lane < j_end) {
        const int u = e * A.n_mod + A.sb_tgt[j_begin + lane];
        moff = A.md_moff[u];
        mcnt = A.md_mcnt[u];
    }
    for_each_flat(moff, mcnt, S.pre, S.off, [&](bool mvalid, int, int md) {
        int oo = 0, on = 0;
        if (mvalid) {
            oo = NT == 5 ? A.t5_off[md] : A.t3_off[md];
            on = NT == 5 ? A.t5_cnt[md] : A.t3_cnt[md];
            if (NT == 3) {
                const float smax = A.t3_smax[md];
                if (smax >= 0.f) {
                    // the view is curvature-ordered: only the T3s inside the seed's window can pass
                    const float w = ks_window(kp, sp, smax, nk, ks_slack(A));
                    const int lo = ks_bound(A.t3_kord, oo, oo + on, kp - w, false);
                    on = ks_bound(A.t3_kord, lo, oo + on, kp + w, true) - lo;
                    oo = lo;
                }
            }
        }
        for_each_flat(oo, on, S.pre2, S.off2, [&](bool valid, int, int p) {
            bool pass = false;
            // pT3: p is a position of the ordered view, the T3 its permutation entry
            const int obj = NT == 5 ? p : (valid ? A.t3_perm[p] : 0);
            if (valid && (NT == 3 || A.t5_valid[obj])) {
                const float2 ks = NT == 5 ? A.t5_ks[obj] : A.t3_kord[p];
                const float kt = ks.x, st = ks.y;
                float thr = nk * fast_sqrtf(sp * sp + st * st);
                const float rel = NT == 5 ? 1e-5f : ks_slack(A);
                pass = fabsf(kp - kt) <= thr * 1.01f + rel * (fabsf(kp) + fabsf(kt)) + 1e-7f;
            }
            int tot;
            int r = warp_rank(pass, tot);
            if (pass) S.cand[ncand + r] = obj;
            ncand += tot;
            if (ncand > kPtPre - 32) {
                __syncwarp();
                pt_flush<NT>(A, c, S, g, ncand, sink);
                ncand = 0;
            }
        });
    });
    __syncwarp();
    if (ncand) pt_flush<NT>(A, c, S, g, ncand, sink);
}

// The pT3 search's curvature-ordered view of each inner MD's T3s, one warp
// per MD: the permutation, the (curvature, sigma) pairs in that order and the
// largest sigma, so that the search bounds the T3s that can pass its curvature
// prefilter by binary search (on a PU200 event 95 % of the (seed, T3) pairs
// fail it). An MD with more than kT3Order T3s keeps the identity order (its
// t3_smax < 0: no window). The T3 arrays themselves are not reordered: the T5
// search reads them at the same time on the graph's other branch.
constexpr int kT3Order = 128;
constexpr int kOrderWarps = 8;
__device__ __forceinline__ unsigned float_order_key(float v) {
    const unsigned u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // the FP32 order (NaNs at the ends)
}
__global__ void __launch_bounds__(kOrderWarps * 32) k_t3_order(Arena A) {
    pdl_begin();
    __shared__ unsigned key[kOrderWarps][kT3Order];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int n_md = min(A.counters[0], A.md_cap);
    const int warps = gridDim.x * kOrderWarps;
    for (int i = blockIdx.x * kOrderWarps + w; i < n_md; i += warps) {
        const int off = A.t3_off[i], n = A.t3_cnt[i];
        if (n == 0) continue;                        // the search never reads an empty MD's view
        if (n > kT3Order) {
            for (int k = lane; k < n; k += 32) {
                A.t3_perm[off + k] = off + k;
                A.t3_kord[off + k] = t3_ks_search(A, off + k);
            }
            if (lane == 0) A.t3_smax[i] = -1.f;
            continue;
        }
        float smax = 0.f;
        for (int k = lane; k < n; k += 32) {
            const float2 v = t3_ks_search(A, off + k);
            key[w][k] = float_order_key(v.x);
            smax = fmaxf(smax, v.y);
        }
        __syncwarp();
        for (int k = lane; k < n; k += 32) {
            const unsigned kk = key[w][k];
            int rank = 0;
            for (int j = 0; j < n; ++j) {
                const unsigned kj = key[w][j];
                rank += (kj < kk) || (kj == kk && j < k);
            }
            A.t3_perm[off + rank] = off + k;
            A.t3_kord[off + rank] = t3_ks_search(A, off + k);
        }
#pragma unroll
        for (int d = 16; d; d >>= 1) smax = fmaxf(smax, __shfl_xor_sync(kFull, smax, d));
        if (lane == 0) A.t3_smax[i] = smax;
        __syncwarp();
    }
}

// pT work items: (passing seed, a chunk of up to kPtChunk modules of its
// superbin list). The same list serves the pT5 and the pT3 search.
__global__ void k_pt_plan(Arena A) {
    pdl_begin();
    const int n_seeds = A.bd->n_seeds;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_seeds; g += gridDim.x * blockDim.x) {
        if (!A.pls_pass[g] || A.pls_sb[g] < 0) continue;
        const int sb = A.pls_sb[g];
        const int j0 = A.sb_off[sb], n = A.sb_off[sb + 1] - j0;
        if (n <= 0) continue;
        const int nch = (n + kPtChunk - 1) / kPtChunk;
        const int k = atomic_add_agg(&A.counters[25], nch);
        for (int j = 0; j < nch && k + j < A.pt_item_cap; ++j) A.pt_items[k + j] = make_int2(g, j0 + j * kPtChunk);
    }
}

// pT5 / pT3 search (FP32 only): each warp takes (seed, module chunk) work
// items from a shared cursor; a seed's candidates are the T objects whose
// inner MD sits in one of the chunk's modules. An item's survivors are staged and written as one
// segment; an item with more survivors than the stage holds is enumerated a
// second time and written directly. The pT refines decide (float-float fit).
template <int NT>
__device__ __forceinline__ void pt_kernel_body(Arena& A, const DevCfg& c) {
    __shared__ PtSmem sm[kPtWarps];
    PtSmem& S = sm[threadIdx.x >> 5];
    const int lane = lane_id();
    const int n_ev = A.bd->n_ev;
    const int n_items = min(A.counters[25], A.pt_item_cap);
    const int stage = min(max(c.pt_stage, 1), kPtStage);
    const int slot = NT == 5 ? 4 : 5;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&A.counters[NT == 5 ? 26 : 27], 1);
        k = __shfl_sync(kFull, k, 0);
        if (k >= n_items) break;
        const int2 it = A.pt_items[k];
        const int g = it.x;
        const int e = event_of(A.seed_off, n_ev, g);
        const int j_end = min(it.y + kPtChunk, A.sb_off[A.pls_sb[g] + 1]);
        int cnt = 0;
        auto stage_sink = [&](bool keep, int obj, int r, int tot) {
            if (keep && cnt + r < stage) S.stage[cnt + r] = obj;
            cnt += tot;
        };
        pt_enumerate<NT>(A, c, S, g, e, it.y, j_end, stage_sink);
        if (cnt == 0) continue;
        int n = cnt, dropped = 0;
        const int base = reserve(&A.counters[slot], NT == 5 ? A.pt5_cap : A.pt3_cap, n, dropped);
        int* seed_out = NT == 5 ? A.pt5_seed : A.pt3_seed;
        int* obj_out = NT == 5 ? A.pt5_obj : A.pt3_obj;
        if (cnt <= stage) {
            for (int q = lane; q < n; q += 32) {
                seed_out[base + q] = g;
                obj_out[base + q] = S.stage[q];
            }
        } else {
            if (lane == 0) atomicAdd(&A.counters[28], 1);
            int wr = 0;
            auto write_sink = [&](bool keep, int obj, int r, int tot) {
                if (keep && wr + r < n) {
                    seed_out[base + wr + r] = g;
                    obj_out[base + wr + r] = obj;
                }
                wr += tot;
            };
            pt_enumerate<NT>(A, c, S, g, e, it.y, j_end, write_sink);
        }
        if (lane == 0 && dropped) atomicAdd(&A.ev_drop[e * 8 + (NT == 5 ? 5 : 6)], dropped);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kPtWarps * 32, 8) k_pt5(Arena A, DevCfg c) {
    pdl_begin();
    pt_kernel_body<5>(A, c);
}
__global__ void __launch_bounds__(kPtWarps * 32, 8) k_pt3(Arena A, DevCfg c) {
    pdl_begin();
    pt_kernel_body<3>(A, c);
}

// A point from lane `src` of this lane's group of 8
__device__ __forceinline__ Pt<double> shfl_pt8(const Pt<double>& q, int src) {
    const unsigned F = 0xffffffffu;
    Pt<double> p;
    p.x = __shfl_sync(F, q.x, src, 8);
    p.y = __shfl_sync(F, q.y, src, 8);
    p.z = __shfl_sync(F, q.z, src, 8);
    p.r = __shfl_sync(F, q.r, src, 8);
    p.srphi = __shfl_sync(F, q.srphi, src, 8);
    p.sz = __shfl_sync(F, q.sz, src, 8);
    p.sr = __shfl_sync(F, q.sr, src, 8);
    return p;
}

// pT5 / pT3 refine, one candidate per group of 8 lanes, one point per lane
// (fit_track_group_ff, or fit_track_group in FP64): for few candidates (one
// event), where a thread per candidate would leave the fit's latency exposed.
template <int NT> __device__ __forceinline__ void pt_refine_group(Arena& A, const DevCfg& c, int n) {
    constexpr int N = NT + 3;
    const int lane = lane_id(), j = lane & 7;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (int i0 = warp * 4; i0 < n; i0 += warps * 4) {
        const int i_raw = i0 + (lane >> 3);
        const bool valid = i_raw < n;
        const int i = valid ? i_raw : n - 1;
        const int g = NT == 5 ? A.pt5_seed[i] : A.pt3_seed[i];
        const int obj = NT == 5 ? A.pt5_obj[i] : A.pt3_obj[i];
        const float* sd = A.bd->seeds + 9 * (size_t)g;
        Pt<double> Q;
        Pt<float> Qf;
        if (j >= 3 && j < N) {
            int m[NT];
            pt_mds<NT>(A, obj, m);
            Qf = md_point<float>(A, m[j - 3]);
            Q = pt_f64(Qf);
        } else {
            const int k = j < 3 ? j : 0;      // lanes past the last point repeat pixel point 0 (unused)
            Qf = pix_pt<float>(sd + 3 * k, c.f.sig_pix);
            Q = pix_pt<double>(sd + 3 * k, c.sig_pix);
        }
        const double kp = A.pls_kappa[g], sp = A.pls_sigk[g];
        // the triplet's points for an undecided pT3 curvature test (all lanes shuffle)
        const Pt<double> T0 = shfl_pt8(Q, 3), T1 = shfl_pt8(Q, 4), T2 = shfl_pt8(Q, 5 < N ? 5 : 3);
        bool kc;
        if (NT == 5) {
            kc = fabs(kp - A.t5_kappa[obj]) <= c.n_pt * sqrt(sq(sp) + sq(A.t5_sigk[obj]));
        } else {
            // the triplet's FP32 curvature decides unless undecided; then FP64
            const float2 ks = A.t3_ks[obj];
            int k = kappa_test_f32(float(kp), float(sp), ks.x, ks.y, c.f.n_pt);
            if (k < 0) {
                Tri<double> tt = tri(T0, T1, T2);
                k = fabs(kp - tt.kappa) <= c.n_pt * sqrt(sq(sp) + sq(tt.sigk));
            }
            kc = k != 0;
        }
        const Fit f = c.fp64_fit ? fit_track_group<N>(Q, Qf, j) : fit_track_group_ff<N>(Qf, j);
        const double chi2_max = NT == 5 ? c.chi2_rphi_pt5 : c.chi2_rphi_pt3;
        const double chi2z_max = NT == 5 ? c.chi2_rz_pt5 : c.chi2_rz_pt3;
        const bool pass = kc && fabs(f.kappa) <= (1.0 + c.tol_r) * 2.0 * c.a && f.chi2_rphi <= chi2_max &&
                          f.chi2_rz <= chi2z_max;
        if (valid && j == 0) {
            PTOut o{};
            if (kc) {
                o.kappa = f.kappa;
                o.chi2_rphi = f.chi2_rphi;
                o.chi2_rz = f.chi2_rz;
                o.score = f.chi2_rphi + f.chi2_rz;
                o.pt = pt_of(c, f.kappa);
            }
            if (NT == 5) {
                A.pt5_valid[i] = pass; A.pt5_kappa[i] = float(o.kappa); A.pt5_chi2[i] = float(o.chi2_rphi);
                A.pt5_chi2z[i] = float(o.chi2_rz); A.pt5_score[i] = float(o.score); A.pt5_pt[i] = float(o.pt);
            } else {
                A.pt3_valid[i] = pass; A.pt3_kappa[i] = float(o.kappa); A.pt3_chi2[i] = float(o.chi2_rphi);
                A.pt3_chi2z[i] = float(o.chi2_rz); A.pt3_score[i] = float(o.score); A.pt3_pt[i] = float(o.pt);
            }
            if (pass) atomic_add_agg(&A.ev_counts[event_of(A.seed_off, A.bd->n_ev, g) * 8 + (NT == 5 ? 5 : 6)], 1);
        }
    }
}

// pT5 / pT3 refine, one thread per candidate: for many candidates (batches),
// where the FP64 pipe is the bound and lanes should not repeat work.
template <int NT> __device__ __forceinline__ void pt_refine_thread(Arena& A, const DevCfg& c, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = NT == 5 ? A.pt5_seed[i] : A.pt3_seed[i];
        const int obj = NT == 5 ? A.pt5_obj[i] : A.pt3_obj[i];
        Pt<double> P[NT + 3];
        Pt<float> Pf[NT + 3];
        const float* sd = A.bd->seeds + 9 * (size_t)g;
#pragma unroll
        for (int j = 0; j < 3; ++j) Pf[j] = pix_pt<float>(sd + 3 * j, c.f.sig_pix);
        int m[NT];
        pt_mds<NT>(A, obj, m);
#pragma unroll
        for (int j = 0; j < NT; ++j) Pf[3 + j] = md_point<float>(A, m[j]);
        if (c.fp64_fit) {
            // the FP64 fit's own points (the pixel errors from the FP64 configuration)
#pragma unroll
            for (int j = 0; j < 3; ++j) P[j] = pix_pt<double>(sd + 3 * j, c.sig_pix);
#pragma unroll
            for (int j = 0; j < NT; ++j) P[3 + j] = pt_f64(Pf[3 + j]);
        }
        const double kp = A.pls_kappa[g], sp = A.pls_sigk[g];
        bool kc;
        if (NT == 5) {
            kc = fabs(kp - A.t5_kappa[obj]) <= c.n_pt * sqrt(sq(sp) + sq(A.t5_sigk[obj]));
        } else {
            // the triplet's FP32 curvature decides unless undecided; then FP64
            const float2 ks = A.t3_ks[obj];
            int k = kappa_test_f32(float(kp), float(sp), ks.x, ks.y, c.f.n_pt);
            if (k < 0) {
                Tri<double> tt = tri(pt_f64(Pf[3]), pt_f64(Pf[4]), pt_f64(Pf[5]));
                k = fabs(kp - tt.kappa) <= c.n_pt * sqrt(sq(sp) + sq(tt.sigk));
            }
            kc = k != 0;
        }
        PTOut o;
        bool pass = pt_eval<NT + 3>(c, P, Pf, kc, NT == 5 ? c.chi2_rphi_pt5 : c.chi2_rphi_pt3,
                                    NT == 5 ? c.chi2_rz_pt5 : c.chi2_rz_pt3, o);
        if (NT == 5) {
            A.pt5_valid[i] = pass; A.pt5_kappa[i] = float(o.kappa); A.pt5_chi2[i] = float(o.chi2_rphi);
            A.pt5_chi2z[i] = float(o.chi2_rz); A.pt5_score[i] = float(o.score); A.pt5_pt[i] = float(o.pt);
        } else {
            A.pt3_valid[i] = pass; A.pt3_kappa[i] = float(o.kappa); A.pt3_chi2[i] = float(o.chi2_rphi);
            A.pt3_chi2z[i] = float(o.chi2_rz); A.pt3_score[i] = float(o.score); A.pt3_pt[i] = float(o.pt);
        }
        if (pass) atomic_add_agg(&A.ev_counts[event_of(A.seed_off, A.bd->n_ev, g) * 8 + (NT == 5 ? 5 : 6)], 1);
    }
}

// Below this many candidates the grouped refine is faster (measured: one
// PU200 event has ~5k pT5 / ~8k pT3 candidates; 64 events ~50x more).
constexpr int kPtGroupRefineMax = 16384;

template <int NT> __device__ __forceinline__ void pt_refine_body(Arena& A, const DevCfg& c) {
    const int n = min(A.counters[NT == 5 ? 4 : 5], NT == 5 ? A.pt5_cap : A.pt3_cap);
    if (n <= kPtGroupRefineMax) pt_refine_group<NT>(A, c, n);
    else pt_refine_thread<NT>(A, c, n);
}

__global__ void k_pt5_refine(Arena A, DevCfg c) {
    pdl_begin();
    pt_refine_body<5>(A, c);
}
__global__ void k_pt3_refine(Arena A, DevCfg c) {
    pdl_begin();
    pt_refine_body<3>(A, c);
}

// ---------------------------------------------------------------------------
// cross-cleaning
// ---------------------------------------------------------------------------
// Categories: 0 pT5, 1 pT3, 2 T5. Hit ids of an object, local to its event:
// outer-tracker hits keep their input index; the pixel hits of seed s are
// n_hits(event) + 3 s + j. Global key slots: hit_off[e] + local for
// outer-tracker hits, n_hits(batch) + 3 seed_global + j for pixel hits.
struct ObjHits {
    int n, e;
    int ids[13];
    int slots[13];
    float score;
};

__device__ __forceinline__ void md_hits_into(const Arena& A, int md, int h0, ObjHits& o) {
    o.ids[o.n] = A.md_lo[md];
    o.slots[o.n++] = h0 + A.md_lo[md];
    o.ids[o.n] = A.md_up[md];
    o.slots[o.n++] = h0 + A.md_up[md];
}

__device__ __forceinline__ void object_hits(const Arena& A, int cat, int idx, ObjHits& o) {
    o.n = 0;
    int m[5];
    int nm;
    if (cat == 2) {
        pt_mds<5>(A, idx, m);
        nm = 5;
        o.e = A.md_gmod[m[0]] / A.n_mod;
        o.score = A.t5_score[idx];
    } else {
        int g = cat == 0 ? A.pt5_seed[idx] : A.pt3_seed[idx];
        o.e = event_of(A.seed_off, A.bd->n_ev, g);
        int nh = A.hit_off[o.e + 1] - A.hit_off[o.e];
        int sl = g - A.seed_off[o.e];
        for (int j = 0; j < 3; ++j) {
            o.ids[o.n] = nh + 3 * sl + j;
            o.slots[o.n++] = A.bd->n_hits + 3 * g + j;
        }
        if (cat == 0) { pt_mds<5>(A, A.pt5_obj[idx], m); nm = 5; o.score = A.pt5_score[idx]; }
        else { pt_mds<3>(A, A.pt3_obj[idx], m); nm = 3; o.score = A.pt3_score[idx]; }
    }
    int h0 = A.hit_off[o.e];
    for (int j = 0; j < nm; ++j) md_hits_into(A, m[j], h0, o);
}

// The cached hits of object f (written by the first cleaning pass).
struct CachedHits {
    int n, e;
    const int* slots;
};

__device__ __forceinline__ CachedHits cached_hits(const Arena& A, int f) {
    const int meta = A.obj_meta[f];
    return CachedHits{meta & 15, meta >> 4, A.obj_slot + 16 * (size_t)f};
}

// key = (score as FP32 bits, FNV-1a of the sorted local hit ids as 32-bit words)
__device__ __forceinline__ unsigned long long object_key(ObjHits& o) {
    int s[13];
    for (int i = 0; i < o.n; ++i) s[i] = o.ids[i];
    for (int i = 1; i < o.n; ++i) {
        int v = s[i], j = i - 1;
        while (j >= 0 && s[j] > v) { s[j + 1] = s[j]; --j; }
        s[j + 1] = v;
    }
    unsigned h = 2166136261u;
    for (int i = 0; i < o.n; ++i) {
        h ^= (unsigned)s[i];
        h *= 16777619u;
    }
    unsigned sb = __float_as_uint(o.score);
    return ((unsigned long long)sb << 32) | h;
}

// pass 0: per hit, the smallest key of each category; pass 1: keep an object
// when it holds the smallest key on every one of its hits.
__global__ void k_clean_keys(Arena A, int pass) {
    pdl_begin();
    const int n5 = min(A.counters[4], A.pt5_cap);
    const int n3 = min(A.counters[5], A.pt3_cap);
    const int nt = min(A.counters[3], A.t5_cap);
    const size_t n_keys = (size_t)A.bd->n_hits + 3 * (size_t)A.bd->n_seeds;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n5 + n3 + nt; f += gridDim.x * blockDim.x) {
        int cat = f < n5 ? 0 : (f < n5 + n3 ? 1 : 2);
        int idx = cat == 0 ? f : (cat == 1 ? f - n5 : f - n5 - n3);
        const uint8_t* vf = cat == 0 ? A.pt5_valid : (cat == 1 ? A.pt3_valid : A.t5_valid);
        uint8_t* kf = cat == 0 ? A.keep_pt5 : (cat == 1 ? A.keep_pt3 : A.keep_t5);
        if (!vf[idx]) {
            if (pass == 1) kf[idx] = 0;
            continue;
        }
        unsigned long long* best = A.best + cat * n_keys;
        if (pass == 0) {
            ObjHits o;
            object_hits(A, cat, idx, o);
            const unsigned long long key = object_key(o);
            for (int i = 0; i < o.n; ++i) atomicMin(best + o.slots[i], key);
            A.obj_key[f] = key;
            A.obj_meta[f] = (o.e << 4) | o.n;
            int* sl = A.obj_slot + 16 * (size_t)f;
            for (int i = 0; i < o.n; ++i) sl[i] = o.slots[i];
        } else {
            const CachedHits o = cached_hits(A, f);
            const unsigned long long key = A.obj_key[f];
            bool keep = true;
            for (int i = 0; i < o.n; ++i) keep &= best[o.slots[i]] == key;
            kf[idx] = keep;
        }
    }
}

// A track candidate from a cached object: its outer-tracker hits are the
// cached slots from `first` on, minus the event's hit offset.
__device__ __forceinline__ void tc_append(const Arena& A, int e, int type, int seed_local, int obj,
                                          const CachedHits& o, int first, float pt, float eta, float phi) {
    int k = atomicAdd(&A.tc_cnt[e], 1);
    if (k >= A.tc_cap) {
        atomicAdd(&A.ev_drop[e * 8 + 7], 1);
        return;
    }
    size_t t = (size_t)e * A.tc_cap + k;
    A.tc_type[t] = type;
    A.tc_seed[t] = seed_local;
    A.tc_obj[t] = obj;
    int* h = A.tc_hits + 10 * t;
    const int h0 = A.hit_off[e];
    for (int j = 0; j < 10; ++j) h[j] = first + j < o.n ? o.slots[first + j] - h0 : -1;
    A.tc_pt[t] = pt;
    A.tc_eta[t] = eta;
    A.tc_phi[t] = phi;
}

// pLS track candidate (no outer-tracker hits)
__device__ __forceinline__ void tc_append_pls(const Arena& A, int e, int seed_local, int g, float pt, float eta,
                                              float phi) {
    int k = atomicAdd(&A.tc_cnt[e], 1);
    if (k >= A.tc_cap) {
        atomicAdd(&A.ev_drop[e * 8 + 7], 1);
        return;
    }
    size_t t = (size_t)e * A.tc_cap + k;
    A.tc_type[t] = 3;
    A.tc_seed[t] = seed_local;
    A.tc_obj[t] = g;
    int* h = A.tc_hits + 10 * t;
    for (int j = 0; j < 10; ++j) h[j] = -1;
    A.tc_pt[t] = pt;
    A.tc_eta[t] = eta;
    A.tc_phi[t] = phi;
}

// eta-phi cell of a list entry, or -1 (the overflow) outside |eta| < kCellEta
__device__ __forceinline__ int cell_of(const Arena& A, float eta, float phi) {
    if (!(fabsf(eta) < kCellEta) || !(fabsf(phi) <= 4.f)) return -1;
    const int ie = min(A.cell_ne - 1, int(floorf((eta + kCellEta) / A.cell_we)));
    const int ip = (int(floorf((phi + float(kPi)) / A.cell_wp)) % A.cell_np + A.cell_np) % A.cell_np;
    return ie * A.cell_np + ip;
}

__device__ __forceinline__ void list_append(const Arena& A, int e, int list, float eta, float phi, int ref) {
    int k = atomicAdd(&A.list_cnt[e * 2 + list], 1);
    if (k < A.list_cap) {
        const size_t L = (size_t)e * 2 + list;
        size_t o = L * A.list_cap + k;
        if (A.compact)
            A.list_q[o] = pack_eta_phi(eta, phi);
        else
            A.list_ef[o] = make_float2(eta, phi);
        A.list_ref[o] = ref;
        const size_t NC = (size_t)A.cell_ne * A.cell_np;
        const int cell = cell_of(A, eta, phi);
        const int slot = cell >= 0 ? atomicAdd(&A.cell_cnt[L * NC + cell], 1) : kCellSlots;
        if (slot < kCellSlots)
            A.cell_idx[(L * NC + cell) * kCellSlots + slot] = k;
        else
            A.ovf_idx[L * A.list_cap + atomicAdd(&A.ovf_cnt[L], 1)] = k;
    }
}

__device__ __forceinline__ void ref_eta_phi(const Arena& A, int ref, double& eta, double& phi) {
    int cat = ref >> 28, idx = ref & 0x0fffffff;
    int g = -1;
    if (cat == 0) g = A.pt5_seed[idx];
    if (cat == 1) g = A.pt3_seed[idx];
    if (g >= 0) { eta = A.pls_eta[g]; phi = A.pls_phi[g]; }
    else { eta = A.t5_eta[idx]; phi = A.t5_phi[idx]; }
}

// Is list entry j (position in the event's list at base) within dr_clean of
// (eta, phi)? FP32 test with an FP64 re-test inside a band around the
// threshold: 1e-3 relative for FP32 entries; 2e-2 for the compact fixed-point
// entries, whose rounding (<= 5e-5 per coordinate) moves d^2 by at most
// 4e-6 = 1 % of the threshold's square wherever d is near the threshold.
__device__ __forceinline__ bool entry_close(const Arena& A, const DevCfg& c, size_t base, int j, double eta,
                                           double phi) {
    const double thr2 = c.dr_clean * c.dr_clean;
    const float thr2f = float(thr2);
    const float band = A.compact ? 2e-2f : 1e-3f;
    bool sent = false;
    const float2 v = A.compact ? unpack_eta_phi(A.list_q[base + j], sent) : A.list_ef[base + j];
    const float de = v.x - float(eta);
    float dp = v.y - float(phi);
    if (dp > float(kPi)) dp -= float(2 * kPi);
    if (dp <= -float(kPi)) dp += float(2 * kPi);
    const float d2 = de * de + dp * dp;
    if (!sent && d2 < thr2f * (1.0f - band)) return true;
    if (sent || d2 <= thr2f * (1.0f + band)) {
        double e2, p2;
        ref_eta_phi(A, A.list_ref[base + j], e2, p2);
        const double dd = eta - e2, dq = wrap_pi(phi - p2);
        return dd * dd + dq * dq < thr2;
    }
    return false;
}

// Is (eta, phi) within dr_clean of any entry of the event's list? Called by
// all 32 lanes of a warp with the same query. The entries within reach lie in
// at most 2 x 2 eta-phi cells (cell sides >= 2 (dr_clean + 1e-3), the 1e-3
// covering the FP32 rounding of either side): lane (d, s) reads slot s of
// cell d, one round for the whole query; then the lanes stride over the
// list's overflow (entries beyond a cell's slots, or outside the cells'
// eta range).
__device__ __forceinline__ bool dr_close_warp(const Arena& A, const DevCfg& c, int e, int list, double eta,
                                              double phi) {
    static_assert(4 * kCellSlots == 32, "one lane per slot of 2 x 2 cells");
    const int lane = lane_id();
    const size_t L = (size_t)e * 2 + list;
    const size_t base = L * A.list_cap;
    const size_t NC = (size_t)A.cell_ne * A.cell_np;
    const float reach = float(c.dr_clean) + 1e-3f;
    const float ef = float(eta), pf = float(phi);
    const int ie0 = int(floorf((ef - reach + kCellEta) / A.cell_we));
    const int ie1 = int(floorf((ef + reach + kCellEta) / A.cell_we));
    const int jp0 = int(floorf((pf - reach + float(kPi)) / A.cell_wp));
    const int jp1 = int(floorf((pf + reach + float(kPi)) / A.cell_wp));
    const int ip0 = (jp0 % A.cell_np + A.cell_np) % A.cell_np, ip1 = (jp1 % A.cell_np + A.cell_np) % A.cell_np;
    const int d = lane / kCellSlots, s = lane % kCellSlots;
    const int ie = (d & 1) ? ie1 : ie0, ip = (d & 2) ? ip1 : ip0;
    const bool own = !((d & 1) && ie1 == ie0) && !((d & 2) && ip1 == ip0) && ie >= 0 && ie < A.cell_ne;
    bool hit = false;
    if (own) {
        const size_t cell = L * NC + (size_t)ie * A.cell_np + ip;
        if (s < min(A.cell_cnt[cell], kCellSlots)) hit = entry_close(A, c, base, A.cell_idx[cell * kCellSlots + s], eta, phi);
    }
    if (__any_sync(kFull, hit)) return true;
    const int n_ovf = min(A.ovf_cnt[L], A.list_cap);
    for (int k0 = 0; k0 < n_ovf; k0 += 32) {
        const int k = k0 + lane;
        const bool h = k < n_ovf && entry_close(A, c, base, A.ovf_idx[L * A.list_cap + k], eta, phi);
        if (__any_sync(kFull, h)) return true;
    }
    return false;
}

// any of the object's outer-tracker hits carries one of the mark bits
__device__ __forceinline__ bool marked_warp(const Arena& A, const CachedHits& o, int first, int bits) {
    const int j = first + lane_id();
    bool m = j < o.n && (A.mark[o.slots[j]] & bits) != 0;
    return __any_sync(kFull, m);
}

// kept pT5: mark hits and seeds, list for the eta-phi tests, track candidates
__global__ void k_clean_pt5(Arena A) {
    pdl_begin();
    const int n5 = min(A.counters[4], A.pt5_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n5; i += gridDim.x * blockDim.x) {
        if (!A.keep_pt5[i]) continue;
        const CachedHits o = cached_hits(A, i);
        for (int j = 3; j < o.n; ++j) atomicOr(&A.mark[o.slots[j]], 1);
        int g = A.pt5_seed[i];
        atomicOr(&A.seed_link[g], 1);
        const float eta = float(A.pls_eta[g]), phi = float(A.pls_phi[g]);
        list_append(A, o.e, 0, eta, phi, (0 << 28) | i);
        tc_append(A, o.e, 0, g - A.seed_off[o.e], i, o, 3, A.pt5_pt[i], eta, phi);
    }
}

__global__ void k_clean_pt3_cross(Arena A, DevCfg c) {
    pdl_begin();
    const int n5 = min(A.counters[4], A.pt5_cap);
    const int n3 = min(A.counters[5], A.pt3_cap);
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n3; i += warps) {
        if (!A.keep_pt3[i]) continue;
        const CachedHits o = cached_hits(A, n5 + i);
        const int g = A.pt3_seed[i];
        bool drop = (A.seed_link[g] & 1) != 0 || marked_warp(A, o, 3, 1);
        if (!drop) drop = dr_close_warp(A, c, o.e, 0, A.pls_eta[g], A.pls_phi[g]);
        if (lane_id() == 0) A.keep_pt3[i] = !drop;
    }
}

__global__ void k_clean_pt3_mark(Arena A) {
    pdl_begin();
    const int n5 = min(A.counters[4], A.pt5_cap);
    const int n3 = min(A.counters[5], A.pt3_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
        if (!A.keep_pt3[i]) continue;
        const CachedHits o = cached_hits(A, n5 + i);
        for (int j = 3; j < o.n; ++j) atomicOr(&A.mark[o.slots[j]], 2);
        int g = A.pt3_seed[i];
        atomicOr(&A.seed_link[g], 2);
        const float eta = float(A.pls_eta[g]), phi = float(A.pls_phi[g]);
        list_append(A, o.e, 0, eta, phi, (1 << 28) | i);
        tc_append(A, o.e, 1, g - A.seed_off[o.e], i, o, 3, A.pt3_pt[i], eta, phi);
    }
}

__global__ void k_clean_t5(Arena A, DevCfg c) {
    pdl_begin();
    const int n5 = min(A.counters[4], A.pt5_cap);
    const int n3 = min(A.counters[5], A.pt3_cap);
    const int nt = min(A.counters[3], A.t5_cap);
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nt; i += warps) {
        if (!A.keep_t5[i]) continue;
        const CachedHits o = cached_hits(A, n5 + n3 + i);
        bool drop = marked_warp(A, o, 0, 3);
        if (!drop) drop = dr_close_warp(A, c, o.e, 0, A.t5_eta[i], A.t5_phi[i]);
        if (lane_id() == 0) {
            A.keep_t5[i] = !drop;
            if (!drop) {
                const float eta = float(A.t5_eta[i]), phi = float(A.t5_phi[i]);
                list_append(A, o.e, 1, eta, phi, (2 << 28) | i);
                tc_append(A, o.e, 2, -1, i, o, 0, A.t5_pt[i], eta, phi);
            }
        }
    }
}

__global__ void k_clean_pls(Arena A, DevCfg c) {
    pdl_begin();
    const int n_ev = A.bd->n_ev, n_seeds = A.bd->n_seeds;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_seeds; g += warps) {
        if (!A.pls_pass[g] || A.seed_link[g]) continue;
        int e = event_of(A.seed_off, n_ev, g);
        double eta = A.pls_eta[g], phi = A.pls_phi[g];
        if (dr_close_warp(A, c, e, 0, eta, phi) || dr_close_warp(A, c, e, 1, eta, phi)) continue;
        if (lane_id() == 0) tc_append_pls(A, e, g - A.seed_off[e], g, A.pls_pt[g], float(eta), float(phi));
    }
}

// The batch's track candidates, event after event, into the record array of
// the batch's result slot. Blocks take (event, slice) pairs, grid-stride, with
// as many slices per event as the grid has blocks per event (at most 16): for
// one event the copy spreads over 16 blocks, for a batch it stays one or two
// blocks per event. Each block sums the counts of the events before its event
// for the offset and copies its slice; the first slice of an event also
// writes the event's offset and statistics (every other stage has finished).
__global__ void k_tc_pack(Arena A) {
    pdl_begin();
    __shared__ int red[32];
    __shared__ int s_off;
    const int n_ev = A.bd->n_ev;
    TcRec* const out = A.bd->out_rec;
    int* const out_off = A.bd->out_off;
    int* const out_stats = A.bd->out_stats;
    const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5;
    const int slices = max(1, min(16, int(gridDim.x) / max(1, n_ev)));
    for (long long v = blockIdx.x; v < (long long)n_ev * slices; v += gridDim.x) {
        const int e = int(v / slices), j = int(v % slices);
        const int n = min(A.tc_cnt[e], A.tc_cap);
        const int len = (n + slices - 1) / slices;
        const int i0 = j * len;
        if (i0 >= n && j > 0) continue;           // block-uniform: nothing of this event in the slice
        int part = 0;
        for (int k = threadIdx.x; k < e; k += blockDim.x) part += min(A.tc_cnt[k], A.tc_cap);
        for (int d = 16; d; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        if (lane_id() == 0) red[w] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < nw; ++k) t += red[k];
            s_off = t;
        }
        __syncthreads();
        const int off = s_off;
        if (j == 0) {
            if (threadIdx.x == 0) {
                out_off[e] = off;
                if (e == n_ev - 1) out_off[n_ev] = off + n;
            }
            if (threadIdx.x < 16)
                out_stats[kSlotStats * e + threadIdx.x] =
                    threadIdx.x < 8 ? A.ev_counts[8 * e + threadIdx.x] : A.ev_drop[8 * e + threadIdx.x - 8];
            if (threadIdx.x == 16) out_stats[kSlotStats * e + 16] = n;
        }
        const size_t src = (size_t)e * A.tc_cap;
        for (int i = i0 + threadIdx.x; i < min(n, i0 + len); i += blockDim.x) {
            TcRec r;
            r.type = A.tc_type[src + i];
            r.seed = A.tc_seed[src + i];
            const int* h = A.tc_hits + 10 * (src + i);
#pragma unroll
            for (int k = 0; k < 10; ++k) r.hits[k] = h[k];
            r.pt = A.tc_pt[src + i];
            r.eta = A.tc_eta[src + i];
            r.phi = A.tc_phi[src + i];
            r.reserved = 0;
            out[off + i] = r;
        }
        __syncthreads();
    }
}

}  // namespace lst
