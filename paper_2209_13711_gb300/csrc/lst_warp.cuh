// Warp-level building blocks shared by the object kernels: ordered
// compaction of passing candidates and flattened iteration over the
// variable-length segments of up to 32 parent objects.
#pragma once

#include "lst_device.cuh"

namespace lst {

constexpr unsigned kFull = 0xffffffffu;

// Flattened iteration: lane l holds segment (off, len) (len = 0 for none).
// body(valid, seg, item) is called by all 32 lanes for every group of 32
// flattened items, in segment-major order, so that a ballot inside body
// keeps a deterministic order.
template <typename F>
__device__ __forceinline__ void for_each_flat(int off, int len, int* sm_pre, int* sm_off, F&& body) {
    const int lane = lane_id();
    int incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int v = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += v;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    __syncwarp();
    sm_pre[lane] = incl - len;
    sm_off[lane] = off;
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        const bool valid = p < total;
        int seg = 0, item = 0;
        if (valid) {
            int lo = 0, hi = 31;          // largest seg with sm_pre[seg] <= p
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (sm_pre[mid] <= p) lo = mid; else hi = mid - 1;
            }
            seg = lo;
            item = sm_off[seg] + (p - sm_pre[seg]);
        }
        body(valid, seg, item);
    }
    __syncwarp();
}

// atomicAdd(p, v) for the lanes that call it together, one atomic per
// distinct address among them: each lane receives what its own atomicAdd would
// have returned had the lanes of its address gone in lane order. Planning
// kernels add to a handful of per-event or global cursors from every thread;
// unaggregated, those same-address atomics serialise at the L2.
__device__ __forceinline__ int atomic_add_agg(int* p, int v) {
    const unsigned peers = __match_any_sync(__activemask(), reinterpret_cast<unsigned long long>(p));
    const int lane = lane_id(), leader = __ffs(peers) - 1;
    int prefix = 0, total = 0;
    for (unsigned m = peers; m; m &= m - 1) {
        const int l = __ffs(m) - 1;
        const int vl = __shfl_sync(peers, v, l);
        if (l < lane) prefix += vl;
        total += vl;
    }
    int base = 0;
    if (lane == leader) base = atomicAdd(p, total);
    return __shfl_sync(peers, base, leader) + prefix;
}

// Reserve n slots of a flat arena with one atomic per warp; returns the
// base (broadcast) and clips n to the arena capacity (the clipped part is
// added to dropped).
__device__ __forceinline__ int reserve(int* counter, int cap, int& n, int& dropped) {
    int base = 0;
    if (lane_id() == 0 && n > 0) base = atomicAdd(counter, n);
    base = __shfl_sync(kFull, base, 0);
    int fit = n > 0 ? max(0, min(n, cap - base)) : 0;
    dropped += n - fit;
    n = fit;
    return base;
}

}  // namespace lst
