// Outer-tracker object kernels: hit binning, mini-doublets (MD), line
// segments (LS), triplets (T3) and quintuplets (T5), in the launch order of
// the paper's Fig. KernelFlow.
//
// Work decomposition: a warp evaluates the candidates of one unit
// lane-parallel, compacts the passing ones in order into a shared-memory stage
// with __ballot_sync, reserves one contiguous segment of the flat arena with a
// single atomicAdd and writes it. The (offset, count) of every unit's segment
// is kept, so the next stage finds "all LS whose inner MD is B" as one
// contiguous range. Units: an inner MD for LS and T3 (one warp each); for MD
// and T5, whose unit costs vary by more than an order of magnitude, work items
// (chunks of a module's lower hits / of an inner MD's T3) taken from a shared
// cursor, heavy items first, whose segments a gather kernel concatenates in
// order. Stage sizes bound the objects one unit may produce (the occupancy
// truncation of Section 3); anything beyond is counted as dropped, never
// written out of bounds (T5 items instead enumerate again and lose nothing).
#include "lst_kernels.cuh"
#include "lst_warp.cuh"

namespace lst {

// ---------------------------------------------------------------------------
// hit binning: counting sort by (event, module, side)
// ---------------------------------------------------------------------------
// Zero the per-batch counters and lists; the key arrays start at all ones.
__global__ void k_reset(Arena A) {
    pdl_begin();
    const BatchDesc B = *A.bd;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    const size_t n_keys = (size_t)B.n_hits + 3 * (size_t)B.n_seeds;
    for (size_t i = t; i < 3 * n_keys; i += stride) A.best[i] = ~0ull;
    for (size_t i = t; i < n_keys; i += stride) A.mark[i] = 0;
    for (size_t i = t; i < (size_t)B.n_ev * 2 * A.n_mod; i += stride) A.bcnt[i] = 0;
    for (size_t i = t; i < (size_t)B.n_seeds; i += stride) A.seed_link[i] = 0;
    for (size_t i = t; i < (size_t)B.n_ev * 8; i += stride) {
        A.ev_counts[i] = 0;
        A.ev_drop[i] = 0;
    }
    const size_t n_cells = (size_t)B.n_ev * 2 * A.cell_ne * A.cell_np;
    for (size_t i = t; i < n_cells; i += stride) A.cell_cnt[i] = 0;
    for (size_t i = t; i < (size_t)B.n_ev; i += stride) {
        A.list_cnt[2 * i] = 0;
        A.list_cnt[2 * i + 1] = 0;
        A.ovf_cnt[2 * i] = 0;
        A.ovf_cnt[2 * i + 1] = 0;
        A.tc_cnt[i] = 0;
        A.t5_evf[i] = 0;
        A.t5_evb[i] = 0;
        A.t5_evc[i] = 0;
    }
    if (t < 32) A.counters[t] = 0;
}

__global__ void k_bin_count(Arena A) {
    pdl_begin();
    const int nb = 2 * A.n_mod;
    const BatchDesc B = *A.bd;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n_hits; i += gridDim.x * blockDim.x) {
        int m = B.hmod[i];
        int s = B.hside[i];
        if (m < 0 || m >= A.n_mod || s > 1) {
            atomicAdd(&A.counters[16], 1);
            continue;
        }
        int e = event_of(A.hit_off, B.n_ev, i);
        atomicAdd(&A.bcnt[(size_t)e * nb + 2 * m + s], 1);
    }
}

// One block per event: exclusive scan of the event's bucket counts into boff;
// the counts are turned into scatter cursors (= offsets). Each warp owns a
// contiguous slice of the buckets: it sums the slice (coalesced), the block
// scans the 32 slice totals, then every warp scans its slice 32 buckets at a
// time with shuffles and writes offsets and cursors.
__global__ void __launch_bounds__(1024) k_bin_scan(Arena A) {
    pdl_begin();
    const int nb = 2 * A.n_mod;
    const int e = blockIdx.x;
    if (e >= A.bd->n_ev) return;
    int* cnt = A.bcnt + (size_t)e * nb;
    int* off = A.boff + (size_t)e * (nb + 1);
    __shared__ int warp_base[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (nb + nw - 1) / nw;
    const int b0 = min(nb, w * per), b1 = min(nb, b0 + per);
    int sum = 0;
    for (int b = b0 + lane; b < b1; b += 32) sum += cnt[b];
#pragma unroll
    for (int d = 16; d; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) warp_base[w] = sum;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? warp_base[lane] : 0, incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        if (lane < nw) warp_base[lane] = incl - v;
        if (lane == nw - 1) off[nb] = incl;
    }
    __syncthreads();
    int run = warp_base[w];
    for (int base = b0; base < b1; base += 32) {
        const int b = base + lane;
        const int c = b < b1 ? cnt[b] : 0;
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        if (b < b1) {
            off[b] = run + incl - c;
            cnt[b] = run + incl - c;      // cursor
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void k_bin_scatter(Arena A) {
    pdl_begin();
    const int nb = 2 * A.n_mod;
    const BatchDesc B = *A.bd;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n_hits; i += gridDim.x * blockDim.x) {
        int m = B.hmod[i];
        int s = B.hside[i];
        if (m < 0 || m >= A.n_mod || s > 1) continue;
        int e = event_of(A.hit_off, B.n_ev, i);
        int h0 = A.hit_off[e];
        int pos = h0 + atomicAdd(&A.bcnt[(size_t)e * nb + 2 * m + s], 1);
        A.sx[pos] = B.hx[i];
        A.sy[pos] = B.hy[i];
        A.sz[pos] = B.hz[i];
        A.sidx[pos] = i - h0;
    }
}

// ---------------------------------------------------------------------------
// MD, one warp per (event, module): the allocation-free entry point's kernel
// (the chain uses the work items below)
// ---------------------------------------------------------------------------
struct MdSmem {
    float lx[kMaxHits], ly[kMaxHits], lz[kMaxHits];
    int li[kMaxHits];
    float ux[kMaxHits], uy[kMaxHits], uz[kMaxHits];
    int ui[kMaxHits];
    int stage[kMdStage];
};

// Stage n sorted-by-bucket hits starting at global position g0 into shared
// memory, ordered by their original index (so MD order does not depend on
// the atomic scatter).
__device__ __forceinline__ void stage_hits(const Arena& A, int g0, int n, float* X, float* Y, float* Z, int* I) {
    const int lane = lane_id();
    float rx[kMaxHits / 32], ry[kMaxHits / 32], rz[kMaxHits / 32];
    int ri[kMaxHits / 32];
#pragma unroll
    for (int k = 0; k < kMaxHits / 32; ++k) {
        int j = lane + 32 * k;
        if (j < n) {
            rx[k] = A.sx[g0 + j];
            ry[k] = A.sy[g0 + j];
            rz[k] = A.sz[g0 + j];
            ri[k] = A.sidx[g0 + j];
            I[j] = ri[k];
        }
    }
    __syncwarp();
    int rank[kMaxHits / 32];
#pragma unroll
    for (int k = 0; k < kMaxHits / 32; ++k) {
        int j = lane + 32 * k;
        rank[k] = 0;
        if (j < n)
            for (int t = 0; t < n; ++t) rank[k] += I[t] < ri[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kMaxHits / 32; ++k) {
        int j = lane + 32 * k;
        if (j < n) {
            X[rank[k]] = rx[k];
            Y[rank[k]] = ry[k];
            Z[rank[k]] = rz[k];
            I[rank[k]] = ri[k];
        }
    }
    __syncwarp();
}

size_t md_smem_bytes() { return kMdWarps * sizeof(MdSmem); }

__global__ void __launch_bounds__(kMdWarps * 32) k_md(Arena A, DevCfg c) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char md_raw[];
    MdSmem& S = reinterpret_cast<MdSmem*>(md_raw)[threadIdx.x >> 5];
    const int lane = lane_id();
    const int n_units = A.bd->n_ev * A.n_mod;
    for (int u = blockIdx.x * kMdWarps + (threadIdx.x >> 5); u < n_units; u += gridDim.x * kMdWarps) {
        const int e = u / A.n_mod, m = u - e * A.n_mod;
        const int* bo = A.boff + (size_t)e * (2 * A.n_mod + 1);
        const int h0 = A.hit_off[e];
        const int ol = bo[2 * m], ou = bo[2 * m + 1];
        int nl = ou - ol, nu = bo[2 * m + 2] - ou;
        int dropped = max(0, nl - kMaxHits) + max(0, nu - kMaxHits);
        nl = min(nl, kMaxHits);
        nu = min(nu, kMaxHits);
        if (nl == 0 || nu == 0) {
            if (lane == 0) {
                A.md_moff[u] = 0;
                A.md_mcnt[u] = 0;
                if (dropped) atomicAdd(&A.ev_drop[e * 8 + 0], dropped);
            }
            continue;
        }
        const float4 mi = A.mod[m];
        stage_hits(A, h0 + ol, nl, S.lx, S.ly, S.lz, S.li);
        stage_hits(A, h0 + ou, nu, S.ux, S.uy, S.uz, S.ui);
        const int total = nl * nu;
        int cnt = 0;
        for (int base = 0; base < total; base += 32) {
            const int p = base + lane;
            bool pass = false;
            int code = 0;
            if (p < total) {
                int l = p / nu, k = p - l * nu;
                code = (l << 16) | k;
                Pt<float> L = hit_pt<float>(S.lx[l], S.ly[l], S.lz[l], mi);
                Pt<float> U = hit_pt<float>(S.ux[k], S.uy[k], S.uz[k], mi);
                float dp, dl;
                int st = md_eval<float>(c, mi, L, U, dp, dl);
                if (st == 2) {
                    Pt<double> Ld = hit_pt<double>(S.lx[l], S.ly[l], S.lz[l], mi);
                    Pt<double> Ud = hit_pt<double>(S.ux[k], S.uy[k], S.uz[k], mi);
                    double dpd, dld;
                    st = md_eval<double>(c, mi, Ld, Ud, dpd, dld);
                }
                pass = st == 1;
            }
            int tot;
            int r = warp_rank(pass, tot);
            if (pass && cnt + r < kMdStage) S.stage[cnt + r] = code;
            cnt += tot;
        }
        __syncwarp();
        int n = min(cnt, kMdStage);
        dropped += cnt - n;
        const int base = reserve(&A.counters[0], A.md_cap, n, dropped);
        for (int i = lane; i < n; i += 32) {
            int code = S.stage[i];
            int l = code >> 16, k = code & 0xffff;
            Pt<float> L = hit_pt<float>(S.lx[l], S.ly[l], S.lz[l], mi);
            Pt<float> U = hit_pt<float>(S.ux[k], S.uy[k], S.uz[k], mi);
            float dp, dl;
            md_eval<float>(c, mi, L, U, dp, dl);
            int o = base + i;
            A.md_lo[o] = S.li[l];
            A.md_up[o] = S.ui[k];
            A.md_gmod[o] = u;
            A.md_p4[o] = make_float4(S.lx[l], S.ly[l], S.lz[l], mi.w < 0.5f ? mi.z : -mi.z);
            A.md_sr[o] = make_float2(mi.y, m_hypot(S.lx[l], S.ly[l]));
            A.md_dx[o] = S.ux[k] - S.lx[l];
            A.md_dy[o] = S.uy[k] - S.ly[l];
            A.md_dphi[o] = dp;
            A.md_dlong[o] = dl;
        }
        if (lane == 0) {
            A.md_moff[u] = base;
            A.md_mcnt[u] = n;
            if (n) atomicAdd(&A.ev_counts[e * 8 + 0], n);
            if (dropped) atomicAdd(&A.ev_drop[e * 8 + 0], dropped);
        }
        __syncwarp();
    }
}

// FP64 re-tests of candidates the FP32 predicates left undecided. Out of line,
// so that no double-precision work is scheduled on the FP32 path (the FP64
// pipe is narrow on this GPU); a warp pays for one only when a lane needs it.
__device__ __noinline__ int md_retest(const DevCfg& c, float4 mi, float lx, float ly, float lz, float ux, float uy,
                                      float uz) {
    Pt<double> L = hit_pt<double>(lx, ly, lz, mi), U = hit_pt<double>(ux, uy, uz, mi);
    double dp, dl;
    return md_eval<double>(c, mi, L, U, dp, dl);
}

__device__ __noinline__ int ls_retest(const Arena& A, const DevCfg& c, int i, int B, float4 miA, float4 miB) {
    double dp;
    return ls_eval<double>(c, md_point<double>(A, i), double(A.md_dx[i]), double(A.md_dy[i]), miA,
                           md_point<double>(A, B), double(A.md_dx[B]), double(A.md_dy[B]), miB, dp);
}

__device__ __noinline__ int t3_retest(const Arena& A, const DevCfg& c, int i, int B, int C) {
    double b, k, r, s;
    return t3_eval<double>(c, md_point<double>(A, i), md_point<double>(A, B), md_point<double>(A, C), b, k, r, s);
}

// ---------------------------------------------------------------------------
// MD as work items (the chain's path; k_md above serves the allocation-free
// entry point). k_bin_sort puts every sensor bucket in original-index order,
// k_md_plan cuts each module's lower hits into chunks so no item holds more
// than about kMdItemPairs pairs, k_md_search writes each chunk's passing
// (lower, upper) positions, k_md_write concatenates the chunks of a module in
// order and writes its MDs.
// ---------------------------------------------------------------------------
constexpr int kMdItemPairs = 1024;
constexpr int kMdCodeStage = 256;

// Warp per sensor bucket: rank by original index; the first kMaxHits (all of
// them in practice) are written back in that order.
__global__ void __launch_bounds__(128) k_bin_sort(Arena A) {
    pdl_begin();
    __shared__ int s_idx[4][kMaxHits];
    __shared__ float s_x[4][kMaxHits], s_y[4][kMaxHits], s_z[4][kMaxHits];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int nb = 2 * A.n_mod;
    const int n_buckets = A.bd->n_ev * nb;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + w; b < n_buckets; b += warps) {
        const int e = b / nb, k = b - e * nb;
        const int* bo = A.boff + (size_t)e * (nb + 1);
        const int g0 = A.hit_off[e] + bo[k], n = bo[k + 1] - bo[k];
        if (n <= 1) continue;
        for (int j = lane; j < n; j += 32) {
            const int ij = A.sidx[g0 + j];
            int rank = 0;
            for (int t = 0; t < n; ++t) rank += A.sidx[g0 + t] < ij;
            if (rank < kMaxHits) {
                s_idx[w][rank] = ij;
                s_x[w][rank] = A.sx[g0 + j];
                s_y[w][rank] = A.sy[g0 + j];
                s_z[w][rank] = A.sz[g0 + j];
            }
        }
        __syncwarp();
        for (int j = lane; j < min(n, kMaxHits); j += 32) {
            A.sidx[g0 + j] = s_idx[w][j];
            A.sx[g0 + j] = s_x[w][j];
            A.sy[g0 + j] = s_y[w][j];
            A.sz[g0 + j] = s_z[w][j];
        }
        __syncwarp();
    }
}

// Lower hits per chunk of module (e, m): at most 32 chunks of about
// kMdItemPairs pairs each.
__device__ __forceinline__ int md_chunk_len(int nl, int nu) {
    int nch = (nl * nu + kMdItemPairs - 1) / kMdItemPairs;
    nch = max(1, min(nch, min(32, nl)));
    return (nl + nch - 1) / nch;
}

__device__ __forceinline__ void md_sizes(const Arena& A, int u, int& e, int& m, int& gl, int& gu, int& nl, int& nu,
                                         int& dropped) {
    e = u / A.n_mod;
    m = u - e * A.n_mod;
    const int* bo = A.boff + (size_t)e * (2 * A.n_mod + 1);
    const int h0 = A.hit_off[e];
    gl = h0 + bo[2 * m];
    gu = h0 + bo[2 * m + 1];
    nl = bo[2 * m + 1] - bo[2 * m];
    nu = bo[2 * m + 2] - bo[2 * m + 1];
    dropped = max(0, nl - kMaxHits) + max(0, nu - kMaxHits);
    nl = min(nl, kMaxHits);
    nu = min(nu, kMaxHits);
}

// Work items {unit, first lower rank | chunk length << 16}: split modules at
// the front of the list, single-chunk modules at the back.
__global__ void k_md_plan(Arena A) {
    pdl_begin();
    const int n_units = A.bd->n_ev * A.n_mod;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += gridDim.x * blockDim.x) {
        int e, m, gl, gu, nl, nu, dropped;
        md_sizes(A, u, e, m, gl, gu, nl, nu, dropped);
        if (nl == 0 || nu == 0) continue;
        const int len = md_chunk_len(nl, nu), nch = (nl + len - 1) / len;
        if (nch > 1) {
            const int k = atomic_add_agg(&A.counters[8], nch);
            for (int j = 0; j < nch; ++j) A.md_items[k + j] = make_int2(u, (j * len) | (len << 16));
        } else {
            const int k = atomic_add_agg(&A.counters[9], 1);
            A.md_items[A.md_item_cap - 1 - k] = make_int2(u, len << 16);
        }
    }
}

struct MdSearchSmem {
    float lx[kMaxHits], ly[kMaxHits], lz[kMaxHits];
    float ux[kMaxHits], uy[kMaxHits], uz[kMaxHits];
    int2 stage[kMdCodeStage];
};

// The pairs of lower ranks [r0, r1) x all upper hits of one module, in order.
template <typename Sink>
__device__ __forceinline__ void md_enumerate(const DevCfg& c, const MdSearchSmem& S, float4 mi, int gl, int gu,
                                             int r0, int r1, int nu, Sink& sink) {
    const int lane = lane_id();
    const int total = (r1 - r0) * nu;
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        bool pass = false;
        int l = 0, k = 0;
        if (p < total) {
            l = p / nu;
            k = p - l * nu;
            Pt<float> L = hit_pt<float>(S.lx[l], S.ly[l], S.lz[l], mi);
            Pt<float> U = hit_pt<float>(S.ux[k], S.uy[k], S.uz[k], mi);
            float dp, dl;
            int st = md_eval<float>(c, mi, L, U, dp, dl);
            if (st == 2) st = md_retest(c, mi, S.lx[l], S.ly[l], S.lz[l], S.ux[k], S.uy[k], S.uz[k]);
            pass = st == 1;
        }
        int tot;
        int r = warp_rank(pass, tot);
        sink(pass, make_int2(gl + r0 + l, gu + k), r, tot);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kMdWarps * 32) k_md_search(Arena A, DevCfg c) {
    pdl_begin();
    __shared__ MdSearchSmem sm[kMdWarps];
    MdSearchSmem& S = sm[threadIdx.x >> 5];
    const int lane = lane_id();
    const int n_front = A.counters[8], n_items = n_front + A.counters[9];
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&A.counters[7], 1);
        k = __shfl_sync(kFull, k, 0);
        if (k >= n_items) break;
        const int2 it = k < n_front ? A.md_items[k] : A.md_items[A.md_item_cap - 1 - (k - n_front)];
        const int u = it.x, r0 = it.y & 0xffff, len = it.y >> 16;
        int e, m, gl, gu, nl, nu, dropped;
        md_sizes(A, u, e, m, gl, gu, nl, nu, dropped);
        const int r1 = min(nl, r0 + len);
        for (int j = lane; j < r1 - r0; j += 32) {
            S.lx[j] = A.sx[gl + r0 + j];
            S.ly[j] = A.sy[gl + r0 + j];
            S.lz[j] = A.sz[gl + r0 + j];
        }
        for (int j = lane; j < nu; j += 32) {
            S.ux[j] = A.sx[gu + j];
            S.uy[j] = A.sy[gu + j];
            S.uz[j] = A.sz[gu + j];
        }
        __syncwarp();
        const float4 mi = A.mod[m];
        int cnt = 0;
        auto stage_sink = [&](bool keep, int2 code, int r, int tot) {
            if (keep && cnt + r < kMdCodeStage) S.stage[cnt + r] = code;
            cnt += tot;
        };
        md_enumerate(c, S, mi, gl, gu, r0, r1, nu, stage_sink);
        int n = cnt, drop = 0;
        const int base = reserve(&A.counters[6], A.md_cap, n, drop);
        if (cnt <= kMdCodeStage) {
            for (int q = lane; q < n; q += 32) A.md_tmp[base + q] = S.stage[q];
        } else {
            int wr = 0;
            auto write_sink = [&](bool keep, int2 code, int r, int tot) {
                if (keep && wr + r < n) A.md_tmp[base + wr + r] = code;
                wr += tot;
            };
            md_enumerate(c, S, mi, gl, gu, r0, r1, nu, write_sink);
        }
        if (lane == 0) {
            A.md_chunk_off[gl + r0] = base;
            A.md_chunk_cnt[gl + r0] = n;
            if (drop) atomicAdd(&A.ev_drop[e * 8 + 0], drop);
        }
        __syncwarp();
    }
}

// Warp per module: its chunks in order become the module's MD segment (at
// most kMdStage MDs, the rest counted as dropped).
__global__ void __launch_bounds__(128) k_md_write(Arena A, DevCfg c) {
    pdl_begin();
    __shared__ int sm_pre[4][32], sm_off[4][32];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int n_units = A.bd->n_ev * A.n_mod;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + w; u < n_units; u += warps) {
        int e, m, gl, gu, nl, nu, dropped;
        md_sizes(A, u, e, m, gl, gu, nl, nu, dropped);
        int off = 0, len = 0;
        if (nl > 0 && nu > 0) {
            const int clen = md_chunk_len(nl, nu), nch = (nl + clen - 1) / clen;
            if (lane < nch) {
                off = A.md_chunk_off[gl + lane * clen];
                len = A.md_chunk_cnt[gl + lane * clen];
            }
        }
        int tot = len;
#pragma unroll
        for (int d = 16; d; d >>= 1) tot += __shfl_xor_sync(kFull, tot, d);
        int n = min(tot, kMdStage);
        dropped += tot - n;
        const int base = reserve(&A.counters[0], A.md_cap, n, dropped);
        const float4 mi = A.mod[m];
        int wr = 0;
        for_each_flat(off, len, sm_pre[w], sm_off[w], [&](bool valid, int, int q) {
            const int o = wr + lane;
            if (valid && o < n) {
                const int2 code = A.md_tmp[q];
                const float lx = A.sx[code.x], ly = A.sy[code.x], lz = A.sz[code.x];
                const float ux = A.sx[code.y], uy = A.sy[code.y], uz = A.sz[code.y];
                Pt<float> L = hit_pt<float>(lx, ly, lz, mi);
                Pt<float> U = hit_pt<float>(ux, uy, uz, mi);
                float dp, dl;
                md_eval<float>(c, mi, L, U, dp, dl);
                const int t = base + o;
                A.md_lo[t] = A.sidx[code.x];
                A.md_up[t] = A.sidx[code.y];
                A.md_gmod[t] = u;
                A.md_p4[t] = make_float4(lx, ly, lz, mi.w < 0.5f ? mi.z : -mi.z);
                A.md_sr[t] = make_float2(mi.y, m_hypot(lx, ly));
                A.md_lsc[t] = ls_terms_f32(c, L, mi.x);
                A.md_dx[t] = ux - lx;
                A.md_dy[t] = uy - ly;
                A.md_dphi[t] = dp;
                A.md_dlong[t] = dl;
            }
            wr += 32;
        });
        if (lane == 0) {
            A.md_moff[u] = base;
            A.md_mcnt[u] = n;
            if (n) atomicAdd(&A.ev_counts[e * 8 + 0], n);
            if (dropped) atomicAdd(&A.ev_drop[e * 8 + 0], dropped);
        }
        __syncwarp();
    }
}

// Inner MDs for the LS and T3 searches are taken kMdChunk at a time from a
// shared cursor (lane 0 claims, all lanes receive): a warp that drew light MDs
// takes more, so the kernel's tail is one chunk's work instead of the heaviest
// warp's share of a fixed stride.
constexpr int kMdChunk = 2;
__device__ __forceinline__ int next_md_chunk(int* cursor) {
    int i = 0;
    if (lane_id() == 0) i = atomicAdd(cursor, kMdChunk);
    return __shfl_sync(kFull, i, 0);
}

// ---------------------------------------------------------------------------
// LS: one warp per inner MD A, candidates = MDs of the connected modules
// ---------------------------------------------------------------------------
struct LsSmem {
    int pre[32], off[32], mod[32];
    int stage[kLsStage];
};


__global__ void __launch_bounds__(kLsWarps * 32, 4) k_ls(Arena A, DevCfg c) {
    pdl_begin();
    __shared__ LsSmem sm[kLsWarps];
    LsSmem& S = sm[threadIdx.x >> 5];
    const int lane = lane_id();
    const int n_md = min(A.counters[0], A.md_cap);
    for (int i0 = next_md_chunk(&A.counters[10]); i0 < n_md; i0 = next_md_chunk(&A.counters[10]))
    for (int i = i0; i < min(i0 + kMdChunk, n_md); ++i) {
        const int gm = A.md_gmod[i];
        const int e = gm / A.n_mod, m1 = gm - e * A.n_mod;
        const float4 miA = A.mod[m1];
        const Pt<float> P = md_point<float>(A, i);
        const float4 tP = A.md_lsc[i];
        const float sAx = A.md_dx[i], sAy = A.md_dy[i];
        const int c0 = A.conn_off[m1], c1 = A.conn_off[m1 + 1];
        int cnt = 0;
        for (int cb = c0; cb < c1; cb += 32) {
            int j = cb + lane;
            int off = 0, len = 0, m2 = 0;
            if (j < c1) {
                m2 = A.conn_tgt[j];
                int u2 = e * A.n_mod + m2;
                off = A.md_moff[u2];
                len = A.md_mcnt[u2];
            }
            S.mod[lane] = m2;
            for_each_flat(off, len, S.pre, S.off, [&](bool valid, int seg, int B) {
                bool pass = false;
                if (valid) {
                    const float4 miB = A.mod[S.mod[seg]];
                    Pt<float> Q = md_point<float>(A, B);
                    float dp;
                    int st = ls_eval_f32(c, P, tP, sAx, sAy, miA, Q, A.md_lsc[B], A.md_dx[B], A.md_dy[B], miB, dp);
                    if (st == 2) st = ls_retest(A, c, i, B, miA, miB);
                    pass = st == 1;
                }
                int tot;
                int r = warp_rank(pass, tot);
                if (pass && cnt + r < kLsStage) S.stage[cnt + r] = B;
                cnt += tot;
            });
        }
        int n = min(cnt, kLsStage);
        int dropped = cnt - n;
        const int base = reserve(&A.counters[1], A.ls_cap, n, dropped);
        for (int k = lane; k < n; k += 32) {
            int B = S.stage[k];
            float4 Bp = A.md_p4[B];
            float Bx = Bp.x, By = Bp.y;
            int o = base + k;
            A.ls_in[o] = i;
            A.ls_out[o] = B;
            A.ls_dphi[o] = atan2f(P.x * By - P.y * Bx, P.x * Bx + P.y * By);
        }
        if (lane == 0) {
            A.ls_off[i] = base;
            A.ls_cnt[i] = n;
            if (n) atomicAdd(&A.ev_counts[e * 8 + 1], n);
            if (dropped) atomicAdd(&A.ev_drop[e * 8 + 1], dropped);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// T3: one warp per inner MD A; candidates = (LS1 from A) x (LS2 from LS1's outer MD)
// ---------------------------------------------------------------------------
struct T3Smem {
    int pre[32], off[32], l1[32], mb[32];
    int2 stage[kT3Stage];
};

__global__ void __launch_bounds__(kT3Warps * 32, 4) k_t3(Arena A, DevCfg c) {
    pdl_begin();
    __shared__ T3Smem sm[kT3Warps];
    T3Smem& S = sm[threadIdx.x >> 5];
    const int lane = lane_id();
    const int n_md = min(A.counters[0], A.md_cap);
    for (int i0 = next_md_chunk(&A.counters[11]); i0 < n_md; i0 = next_md_chunk(&A.counters[11]))
    for (int i = i0; i < min(i0 + kMdChunk, n_md); ++i) {
        const int s0 = A.ls_off[i], s1 = s0 + A.ls_cnt[i];
        if (s1 == s0) {
            if (lane == 0) { A.t3_off[i] = 0; A.t3_cnt[i] = 0; }
            continue;
        }
        const int e = A.md_gmod[i] / A.n_mod;
        const Pt<float> PA = md_point<float>(A, i);
        int cnt = 0;
        for (int cb = s0; cb < s1; cb += 32) {
            int l1 = cb + lane;
            int off = 0, len = 0, B = 0;
            if (l1 < s1) {
                B = A.ls_out[l1];
                off = A.ls_off[B];
                len = A.ls_cnt[B];
            }
            S.l1[lane] = l1;
            S.mb[lane] = B;
            for_each_flat(off, len, S.pre, S.off, [&](bool valid, int seg, int l2) {
                bool pass = false;
                if (valid) {
                    int B_ = S.mb[seg];
                    int C_ = A.ls_out[l2];
                    float beta, kap, rz, sk;
                    int st = t3_eval<float>(c, PA, md_point<float>(A, B_), md_point<float>(A, C_), beta, kap, rz, sk);
                    if (st == 2) st = t3_retest(A, c, i, B_, C_);
                    pass = st == 1;
                }
                int tot;
                int r = warp_rank(pass, tot);
                if (pass && cnt + r < kT3Stage) S.stage[cnt + r] = make_int2(S.l1[seg], l2);
                cnt += tot;
            });
        }
        int n = min(cnt, kT3Stage);
        int dropped = cnt - n;
        const int base = reserve(&A.counters[2], A.t3_cap, n, dropped);
        for (int k = lane; k < n; k += 32) {
            int2 pr = S.stage[k];
            int B_ = A.ls_out[pr.x], C_ = A.ls_out[pr.y];
            // the outputs are the three-point quantities t3_eval decided on
            const Tri<float> t = tri(PA, md_point<float>(A, B_), md_point<float>(A, C_));
            const float beta = t.beta, kap = t.kappa, sk = t.sigk;
            int o = base + k;
            A.t3_lsin[o] = pr.x;
            A.t3_lsout[o] = pr.y;
            A.t3_md[o] = make_int4(i, B_, C_, 0);
            A.t3_beta[o] = beta;
            A.t3_ks[o] = make_float2(kap, sk);
            if (A.compact) {
                const float inv = 1.f / A.two_a;
                A.t3_ksh[o] = __floats2half2_rn(kap * inv, sk * inv);
            }
        }
        if (lane == 0) {
            A.t3_off[i] = base;
            A.t3_cnt[i] = n;
            if (n) atomicAdd(&A.ev_counts[e * 8 + 2], n);
            if (dropped) atomicAdd(&A.ev_drop[e * 8 + 2], dropped);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// T5: candidates = (T3_1 from inner MD A) x (T3_2 from T3_1's outer MD), in
// work items of 8-32 T3_1. FP32 curvature and fit prefilters (conservative),
// then the full test for the survivors (k_t5_refine, float-float fit).
// ---------------------------------------------------------------------------
struct T5Smem {
    int cur[5];                // the warp's item cursor (t5_next_item): event, front count, total, region
    int pre[32], off[32], t1[32];
    float2 ks1[32];            // curvature and sigma of each lane's T3_1
    int2 cand[kT5Pre];
    int2 stage[kT5Stage];      // passing (T3_1, T3_2)
};

__device__ __forceinline__ void t5_mds(const Arena& A, int2 pr, int* m) {
    const int4 a = A.t3_md[pr.x], b = A.t3_md[pr.y];
    m[0] = a.x;
    m[1] = a.y;
    m[2] = a.z;
    m[3] = b.y;
    m[4] = b.z;
}

__device__ __forceinline__ bool t5_prefit_f32(const Arena& A, const DevCfg& c, int2 pr) {
    int m[5];
    t5_mds(A, pr, m);
    Pt<float> P[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) P[j] = md_point<float>(A, m[j]);
    return fit_may_pass_f32<5>(P, c.lim_t5);
}

// Collected candidates: FP32 fit prefilter; the verdicts of each group of 32
// are written to `keep` bits in candidate order (one out-of-line copy of the
// fit keeps the kernel's instruction footprint small).
__device__ __noinline__ unsigned t5_prefit_group(const Arena& A, const DevCfg& c, const int2* cand, int q, int n) {
    bool keep = q < n && t5_prefit_f32(A, c, cand[q]);
    return __ballot_sync(kFull, keep);
}

template <typename Smem, typename Sink>
__device__ __forceinline__ void t5_flush(const Arena& A, const DevCfg& c, Smem& S, int ncand, Sink& sink) {
    const int lane = lane_id();
    for (int base = 0; base < ncand; base += 32) {
        int q = base + lane;
        unsigned m = t5_prefit_group(A, c, S.cand, q, ncand);
        bool keep = (m >> lane) & 1u;
        int tot = __popc(m);
        int r = __popc(m & ((1u << lane) - 1u));
        sink(keep, q < ncand ? S.cand[q] : make_int2(0, 0), r, tot);
    }
    __syncwarp();
}

// Candidates whose T3_1 lies in [t_begin, t_end) (T3 of one inner MD), in a
// fixed order: (T3_1) x (T3_2 from T3_1's outer MD), curvature prefilter,
// FP32 fit prefilter, then the sink.
template <typename Smem, typename Sink>
__device__ __forceinline__ void t5_enumerate(const Arena& A, const DevCfg& c, Smem& S, int t_begin, int t_end,
                                             Sink& sink) {
    const int lane = lane_id();
    const float nk = float(c.n_t5);
    int ncand = 0;
    for (int cb = t_begin; cb < t_end; cb += 32) {
        int t1 = cb + lane;
        int off = 0, len = 0;
        float2 ks = make_float2(0.f, 0.f);
        if (t1 < t_end && (!A.t3_sel || A.t3_ok[t1])) {
            int C_ = A.t3_md[t1].z;
            off = A.t3_off[C_];
            len = A.t3_cnt[C_];
            ks = t3_ks_search(A, t1);
        }
        S.t1[lane] = t1;
        S.ks1[lane] = ks;
        for_each_flat(off, len, S.pre, S.off, [&](bool valid, int seg, int t2) {
            bool pass = false;
            int t1_ = 0;
            if (valid && (!A.t3_sel || A.t3_ok[t2])) {
                t1_ = S.t1[seg];
                const float2 a = S.ks1[seg], b = t3_ks_search(A, t2);
                float k1 = a.x, k2 = b.x;
                float s1_ = a.y, s2_ = b.y;
                float thr = nk * fast_sqrtf(s1_ * s1_ + s2_ * s2_);
                // slack covers the rounding of the stored curvatures (FP32, or FP16 in compact storage)
                pass = fabsf(k1 - k2) <= thr * 1.01f + ks_slack(A) * (fabsf(k1) + fabsf(k2)) + 1e-7f;
            }
            int tot;
            int r = warp_rank(pass, tot);
            if (pass) S.cand[ncand + r] = make_int2(t1_, t2);
            ncand += tot;
            if (ncand > kT5Pre - 32) {
                __syncwarp();
                t5_flush(A, c, S, ncand, sink);
                ncand = 0;
            }
        });
    }
    __syncwarp();
    if (ncand) t5_flush(A, c, S, ncand, sink);
}

// Chunk length of the batch's T5 work items: a small batch splits its heavy
// units finer (their tail sets the kernel's time), a large one keeps the
// per-item overhead low (measured: 8 for one PU200 event, 32 for 64 events).
__device__ __forceinline__ int t5_chunk_len(const Arena& A) {
    const int n_t3 = min(A.counters[2], A.t3_cap);
    return n_t3 < (1 << 21) ? 8 : (n_t3 < (1 << 23) ? 16 : 32);
}

// T5 work items: the T3_1 of each inner MD in chunks of t5_chunk_len, event
// by event. Event e owns the region [base_e, base_e+1) of the item list, as
// long as its T3 count (every item holds at least one T3_1), so no second pass
// is needed: chunks of units with more than one chunk go to the front of the
// region (they are the heavy units and start first), single-chunk units to
// the back. The bases are written for the search (t5_evbase[0..n_ev]).
__global__ void k_t5_plan(Arena A) {
    pdl_begin();
    extern __shared__ int s_base[];
    const int n_ev = A.bd->n_ev;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int e = 0; e < n_ev; ++e) {
            s_base[e] = b;
            b += A.ev_counts[8 * e + 2];
        }
        s_base[n_ev] = b;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e <= n_ev; e += blockDim.x) A.t5_evbase[e] = s_base[e];
    const int n_md = min(A.counters[0], A.md_cap);
    const int clen = t5_chunk_len(A);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_md; i += gridDim.x * blockDim.x) {
        const int n = A.t3_cnt[i];
        if (n == 0) continue;
        const int e = A.md_gmod[i] / A.n_mod;
        const int s0 = A.t3_off[i], nch = (n + clen - 1) / clen;
        if (nch > 1) {
            const int k = atomic_add_agg(&A.t5_evf[e], nch);
            for (int j = 0; j < nch; ++j) A.t5_items[s_base[e] + k + j] = s0 + j * clen;
            atomic_add_agg(&A.counters[22], nch);
        } else {
            const int k = atomic_add_agg(&A.t5_evb[e], 1);
            A.t5_items[s_base[e + 1] - 1 - k] = s0;
            atomic_add_agg(&A.counters[23], 1);
        }
    }
}

size_t t5_plan_smem_bytes(int max_events) { return sizeof(int) * (size_t)(max_events + 1); }

// Next T5 work item of a warp (lane 0 claims, all lanes receive it): the
// events are taken in order, so the warps of the grid work on one or two
// events at a time and the records they gather stay in L2 at batch size.
// counters[24] is the first event whose items may remain. The warp keeps its
// current event's item counts and region in its shared-memory slot (cur: event
// or -1, front count, total, region start and end; registers are scarce in the
// search), so a claim is one atomic and one load; a warp that finds its event's
// cursor past the end moves the pointer on and loads the next event. Every
// pass either claims an item or advances the event, so the loop ends within
// n_ev passes. Returns the item's first T3_1, or -1 when none is left.
__device__ __noinline__ int t5_next_item(const Arena& A, int n_ev, int* cur) {
    int t0 = -1;
    if (lane_id() == 0) {
        for (int pass = 0; pass <= n_ev; ++pass) {
            if (cur[0] < 0) {
                const int e = *reinterpret_cast<volatile const int*>(&A.counters[24]);
                if (e >= n_ev) break;
                cur[0] = e;
                cur[1] = A.t5_evf[e];
                cur[2] = cur[1] + A.t5_evb[e];
                cur[3] = A.t5_evbase[e];
                cur[4] = A.t5_evbase[e + 1];
            }
            const int k = atomicAdd(&A.t5_evc[cur[0]], 1);
            if (k < cur[2]) {
                t0 = k < cur[1] ? A.t5_items[cur[3] + k] : A.t5_items[cur[4] - 1 - (k - cur[1])];
                break;
            }
            atomicMax(&A.counters[24], cur[0] + 1);
            cur[0] = -1;
        }
    }
    return __shfl_sync(kFull, t0, 0);
}

// T5 search (FP32 only): each warp takes work items from a shared cursor
// (split units first). A chunk's survivors are staged in shared memory and
// written as one segment of t5_tmp; a chunk with more survivors than the
// stage holds is enumerated a second time and written straight to its
// reserved segment, in the same order. k_t5_gather orders the segments by
// inner MD and k_t5_refine decides the candidates in FP64.
__global__ void __launch_bounds__(kT5Warps * 32, 6) k_t5(Arena A, DevCfg c) {
    pdl_begin();
    __shared__ T5Smem sm[kT5Warps];
    T5Smem& S = sm[threadIdx.x >> 5];
    const int lane = lane_id();
    const int n_ev = A.bd->n_ev;
    const int stage = min(max(c.t5_stage, 1), kT5Stage);
    const int clen = t5_chunk_len(A);
    if (lane == 0) S.cur[0] = -1;
    __syncwarp();
    for (;;) {
        const int t0 = t5_next_item(A, n_ev, S.cur);
        if (t0 < 0) break;
        const int i = A.t3_md[t0].x;
        const int t_end = min(t0 + clen, A.t3_off[i] + A.t3_cnt[i]);
        int cnt = 0;
        auto stage_sink = [&](bool keep, int2 pr, int r, int tot) {
            if (keep && cnt + r < stage) S.stage[cnt + r] = pr;
            cnt += tot;
        };
        t5_enumerate(A, c, S, t0, t_end, stage_sink);
        int n = cnt, dropped = 0;
        const int base = reserve(&A.counters[21], A.t5_cap, n, dropped);
        if (cnt <= stage) {
            for (int q = lane; q < n; q += 32) A.t5_tmp[base + q] = S.stage[q];
        } else {
            if (lane == 0) atomicAdd(&A.counters[20], 1);
            int wr = 0;
            auto write_sink = [&](bool keep, int2 pr, int r, int tot) {
                if (keep && wr + r < n) A.t5_tmp[base + wr + r] = pr;
                wr += tot;
            };
            t5_enumerate(A, c, S, t0, t_end, write_sink);
        }
        if (lane == 0) {
            A.t5_chunk_off[t0] = base;
            A.t5_chunk_cnt[t0] = n;
            if (dropped) atomicAdd(&A.ev_drop[(A.md_gmod[i] / A.n_mod) * 8 + 3], dropped);
        }
        __syncwarp();
    }
}

// One warp per inner MD: its chunks' survivors, in chunk order, become the
// MD's T5 segment (the order a single pass over the MD's T3_1 would give).
__global__ void __launch_bounds__(128) k_t5_gather(Arena A) {
    pdl_begin();
    __shared__ int sm_pre[4][32], sm_off[4][32];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int n_md = min(A.counters[0], A.md_cap);
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int clen = t5_chunk_len(A);
    for (int i = blockIdx.x * (blockDim.x >> 5) + w; i < n_md; i += warps) {
        const int n1 = A.t3_cnt[i];
        const int nch = (n1 + clen - 1) / clen;      // <= kT3Stage / 8 = 64
        int tot = 0;
        for (int g0 = 0; g0 < nch; g0 += 32) {
            const int j = g0 + lane;
            int len = j < nch ? A.t5_chunk_cnt[A.t3_off[i] + j * clen] : 0;
#pragma unroll
            for (int d = 16; d; d >>= 1) len += __shfl_xor_sync(kFull, len, d);
            tot += len;
        }
        int n = tot, dropped = 0;
        const int base = reserve(&A.counters[3], A.t5_cap, n, dropped);
        int wr = 0;
        for (int g0 = 0; g0 < nch; g0 += 32) {
            const int j = g0 + lane;
            int off = 0, len = 0;
            if (j < nch) {
                const int t0 = A.t3_off[i] + j * clen;
                off = A.t5_chunk_off[t0];
                len = A.t5_chunk_cnt[t0];
            }
            int gsum = len;
#pragma unroll
            for (int d = 16; d; d >>= 1) gsum += __shfl_xor_sync(kFull, gsum, d);
            int pos = wr;
            for_each_flat(off, len, sm_pre[w], sm_off[w], [&](bool valid, int, int q) {
                if (valid && pos + lane < n) {
                    const int2 pr = A.t5_tmp[q];
                    A.t5_in[base + pos + lane] = pr.x;
                    A.t5_out[base + pos + lane] = pr.y;
                }
                pos += 32;
            });
            wr += gsum;
        }
        if (lane == 0) {
            A.t5_off[i] = base;
            A.t5_cnt[i] = n;
            if (dropped) atomicAdd(&A.ev_drop[(A.md_gmod[i] / A.n_mod) * 8 + 3], dropped);
        }
        __syncwarp();
    }
}

// The T5 outputs of candidate i (event e)
__device__ __forceinline__ void t5_store(Arena& A, int i, int e, bool pass, const T5Out& o, bool use_mlp) {
    A.t5_cut[i] = pass;
    A.t5_kappa[i] = o.kappa;
    A.t5_sigk[i] = o.sigk;
    A.t5_ks[i] = make_float2(float(o.kappa), float(o.sigk));
    A.t5_eta[i] = o.eta;
    A.t5_phi[i] = o.phi0;
    A.t5_chi2[i] = float(o.chi2_rphi);
    A.t5_chi2z[i] = float(o.chi2_rz);
    A.t5_score[i] = float(o.score);
    A.t5_pt[i] = float(o.pt);
    if (!use_mlp) {
        A.t5_valid[i] = pass;
        if (pass) atomic_add_agg(&A.ev_counts[e * 8 + 3], 1);
    }
}

// T5 refine, one thread per searched candidate (lane-dense): decides the
// hand-set cuts, writes the T5 outputs and, when enabled, the scoring
// features; without the network the cut decision is the validity. (A group
// of 8 lanes per candidate, as in the pT refines, measured slower here: the
// shuffled float-float sums cost more than the latency they hide.)
__global__ void k_t5_refine(Arena A, DevCfg c) {
    pdl_begin();
    const int n = min(A.counters[3], A.t5_cap);
    const BatchDesc* B = A.bd;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int m[5];
        const int2 pr = make_int2(A.t5_in[i], A.t5_out[i]);
        t5_mds(A, pr, m);
        Pt<float> Pf[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) Pf[j] = md_point<float>(A, m[j]);
        T5Out o;
        const float2 ka = A.t3_ks[pr.x], kb = A.t3_ks[pr.y];
        bool pass = t5_eval(c, Pf, ka.x, ka.y, kb.x, kb.y, c.use_mlp != 0, o);
        const int e = A.md_gmod[m[0]] / A.n_mod;
        t5_store(A, i, e, pass, o, c.use_mlp != 0);
        if (c.features_on) {
            Pt<double> P[5], H[10];
            int code[5];
            const int h0 = A.hit_off[e];
            for (int j = 0; j < 5; ++j) {
                P[j] = pt_f64(Pf[j]);
                H[2 * j] = P[j];
                Pt<double> U = P[j];
                const int hu = h0 + A.md_up[m[j]];
                U.x = B->hx[hu];
                U.y = B->hy[hu];
                U.z = B->hz[hu];
                U.r = hypot(U.x, U.y);
                H[2 * j + 1] = U;
                const int mod = A.md_gmod[m[j]] % A.n_mod;
                code[j] = A.mod_layer[mod] + (A.mod[mod].w > 0.5f ? 6 : 0);
            }
            t5_features(c, P, H, code, A.t5_feat + (size_t)48 * i);
        }
    }
}

// Scoring features of every T3 of the batch, written out (the learned triplet
// selection's training set; k_t3_score computes them in place for the
// network): one thread per T3; the upper hits come from the input arrays.
__global__ void k_t3_features(Arena A, DevCfg c) {
    pdl_begin();
    const int n = min(A.counters[2], A.t3_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Pt<float> P[3], H[6];
        int code[3];
        t3_feature_inputs(A, i, P, H, code);
        float v[48];
        t3_features(c, P, H, code, v);
        float4* f = reinterpret_cast<float4*>(A.t3_feat + (size_t)48 * i);
#pragma unroll
        for (int j = 0; j < 12; ++j) f[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
}

// Validity from the network score (the hand-set cut decision stays in t5_cut).
__global__ void k_t5_mlp_select(Arena A, DevCfg c) {
    pdl_begin();
    const int n = min(A.counters[3], A.t5_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool pass = A.t5_mlp[i] >= c.mlp_threshold && fabs(A.t5_kappa[i]) <= (1.0 + c.tol_r) * 2.0 * c.a;
        A.t5_valid[i] = pass;
        if (pass) {
            int m[5];
            t5_mds(A, make_int2(A.t5_in[i], A.t5_out[i]), m);
            atomicAdd(&A.ev_counts[(A.md_gmod[m[0]] / A.n_mod) * 8 + 3], 1);
        }
    }
}

}  // namespace lst
