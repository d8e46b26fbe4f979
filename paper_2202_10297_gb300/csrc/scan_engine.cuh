// Block-level scan and single-pass decoupled look-back, shared by the scan
// and batch kernels.
//
// Tile layout ("striped vectors"): a tile is K chunks of BLOCK*V
// contiguous elements; in chunk k thread t owns the V elements at
// k*BLOCK*V + t*V, loaded as one 16-byte vector.  Global loads are fully
// coalesced and need no shared-memory transpose.  The scan order inside a
// tile is (k, t, j) lexicographic for a forward scan and its mirror image
// for a reverse scan.
#pragma once

#include "common.cuh"

namespace adpar {

// Index of (chunk k, warp w) in scan order.
template <bool REV, int K, int NW>
__device__ __forceinline__ int chunk_warp_pos(int k, int w) {
    return REV ? (K - 1 - k) * NW + (NW - 1 - w) : k * NW + w;
}

// Part 1 of a block scan.  agg[k] is the thread's aggregate of its V
// elements of chunk k (in scan order).  On return:
//   wex[k]        the warp-exclusive prefix of the thread for chunk k,
//   s_tot[q]      the block-exclusive prefix of (chunk, warp) q,
//   return value  (in warp 0) the aggregate of the whole tile.
// Requires K * NW <= 32.  Warp 0 writes s_tot after the internal barrier,
// so callers must __syncthreads() before block_scan_excl reads it.
template <class S, bool REV, int K, int NW, class Comb>
__device__ __forceinline__ S block_scan_part1(const S (&agg)[K], S (&wex)[K], S* s_tot,
                                              const S& ident, Comb comb) {
    static_assert(K * NW <= 32, "one warp scans the per-warp totals");
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        S inc = agg[k];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            S o = REV ? shfl_down_s(inc, off) : shfl_up_s(inc, off);
            bool ok = REV ? (lane + off < 32) : (lane >= off);
            if (ok) inc = comb(o, inc);
        }
        S ex = REV ? shfl_down_s(inc, 1) : shfl_up_s(inc, 1);
        if (REV ? lane == 31 : lane == 0) ex = ident;
        wex[k] = ex;
        if (REV ? lane == 0 : lane == 31) s_tot[chunk_warp_pos<REV, K, NW>(k, warp)] = inc;
    }
    __syncthreads();
    S total = ident;
    if (warp == 0) {
        constexpr int Q = K * NW;
        S v = lane < Q ? s_tot[lane] : ident;
        S inc = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            S o = shfl_up_s(inc, off);
            if (lane >= off) inc = comb(o, inc);
        }
        S ex = shfl_up_s(inc, 1);
        if (lane == 0) ex = ident;
        __syncwarp();
        if (lane < Q) s_tot[lane] = ex;
        total = shfl_idx_s(inc, Q - 1);
    }
    return total;
}

// Part 2: the thread's exclusive prefix for chunk k, given the exclusive
// prefix of the whole tile (visible in shared memory after a sync).
template <class S, bool REV, int K, int NW, class Comb>
__device__ __forceinline__ S block_scan_excl(int k, const S (&wex)[K], const S* s_tot,
                                             const S& tile_prefix, Comb comb) {
    const int warp = threadIdx.x >> 5;
    return comb(tile_prefix, comb(s_tot[chunk_warp_pos<REV, K, NW>(k, warp)], wex[k]));
}

// Tile status arrays of one single-pass scan.
template <class S>
struct LookbackState {
    uint32_t* flag;  // 0: nothing yet, 1: aggregate published, 2: inclusive prefix published
    S* agg;
    S* incl;
};

// Decoupled look-back, run by one whole warp for logical tile t.
// Publishes the tile's aggregate, walks back over the predecessors in
// windows of 32 (each lane polls one tile, bounded), stops at the first
// tile whose inclusive prefix is out, publishes this tile's inclusive
// prefix and returns the exclusive prefix (in every lane).
template <class S, class Comb>
__device__ __forceinline__ S lookback(int64_t t, LookbackState<S> st, const S& tile_total,
                                      const S& ident, Comb comb, WsHeader* hdr) {
    const int lane = threadIdx.x & 31;
    if (t == 0) {
        if (lane == 0) {
            st.incl[0] = tile_total;
            st_release_u32(&st.flag[0], 2u);
        }
        return ident;
    }
    if (lane == 0) {
        st.agg[t] = tile_total;
        st_release_u32(&st.flag[t], 1u);
    }
    S prefix = ident;
    int64_t base = t - 1;
    while (true) {
        const int64_t idx = base - lane;
        uint32_t f = 2u;  // before tile 0: a virtual inclusive identity
        if (idx >= 0) f = wait_flag(&st.flag[idx], hdr);  // 0 only after a timeout
        const uint32_t stop_mask = __ballot_sync(0xffffffffu, f != 1u);
        const int stop = stop_mask ? __ffs(stop_mask) - 1 : 31;
        S v = ident;
        if (lane <= stop && idx >= 0) {
            if (f == 2u) v = ld_cg(&st.incl[idx]);
            else if (f == 1u) v = ld_cg(&st.agg[idx]);
        }
        // lanes hold tiles in decreasing order: higher lane = earlier tile
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            S o = shfl_down_s(v, off);
            if (lane + off < 32) v = comb(o, v);
        }
        prefix = comb(v, prefix);
        if (stop_mask) break;
        base -= 32;
    }
    prefix = shfl_idx_s(prefix, 0);
    if (lane == 0) {
        st.incl[t] = comb(prefix, tile_total);
        st_release_u32(&st.flag[t], 2u);
    }
    return prefix;
}

}  // namespace adpar
