// ksum_tiles.cuh -- source streams of the kernel-sum kernels.
//
// A target node's sources are the points of all partners in its CSR row,
// taken as one concatenated stream.  The stream is consumed in tiles: the
// partner records of up to kPartnerChunk partners are loaded in parallel
// into shared memory together with the prefix sums of their point counts,
// and every slot of a tile finds its partner by binary search in that prefix.
// One tile never spans two chunks.
#pragma once

#include "internal.cuh"

namespace smash {

constexpr int kPartnerChunk = 256;

struct PartnerChunk {
    int64_t off[kPartnerChunk];      // first source index of each partner
    int pre[kPartnerChunk + 1];      // prefix of the partners' point counts
    int n;                           // partners in the chunk
    int warp_tot[32];
};

// Loads partners [e, min(e + kPartnerChunk, e1)) of the row; all threads call it.
template <int NT>
__device__ __forceinline__ void load_partner_chunk(PartnerChunk &pc, int64_t e, int64_t e1,
                                                   const int32_t *__restrict__ col, const int64_t *__restrict__ s_off,
                                                   const int32_t *__restrict__ s_cnt) {
    static_assert(NT == kPartnerChunk, "one partner record per thread");
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t left = e1 - e;
    const int n = left < kPartnerChunk ? (int)left : kPartnerChunk;
    // one partner per thread (NT >= kPartnerChunk is required by the callers)
    int cnt = 0;
    if (tid < n) {
        int j = col[e + tid];
        cnt = s_cnt[j];
        pc.off[tid] = s_off[j];
    }
    // block inclusive scan of cnt over the first kPartnerChunk threads
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) pc.warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = lane < NT / 32 ? pc.warp_tot[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < NT / 32) pc.warp_tot[lane] = ti - t;
    }
    __syncthreads();
    if (tid < kPartnerChunk) pc.pre[tid + 1] = incl + pc.warp_tot[w];
    if (tid == 0) {
        pc.pre[0] = 0;
        pc.n = n;
    }
    __syncthreads();
}

// source index of stream position p (0 <= p < pc.pre[pc.n]) of the chunk
__device__ __forceinline__ int64_t chunk_source(const PartnerChunk &pc, int p) {
    int lo = 0, hi = pc.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pc.pre[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return pc.off[lo] + (p - pc.pre[lo]);
}

}  // namespace smash
