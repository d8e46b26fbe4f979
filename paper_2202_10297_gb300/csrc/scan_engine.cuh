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

// The barrier of a block scan: the whole block (BAR = 0) or, in a kernel
// with warps outside the scan, named barrier BAR over the NW scanning warps.
template <int BAR, int NW>
__device__ __forceinline__ void scan_bar() {
    if constexpr (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NW * 32) : "memory");
}

// Part 1 of a block scan.  agg[k] is the thread's aggregate of its V
// elements of chunk k (in scan order).  On return:
//   wex[k]        the warp-exclusive prefix of the thread for chunk k,
//   s_tot[q]      the block-exclusive prefix of (chunk, warp) q,
//   return value  (in warp 0) the aggregate of the whole tile.
// Warp 0 scans the K*NW per-warp totals with R = ceil(K*NW/32) of them per
// lane.  Warp 0 writes s_tot after the internal barrier, so callers must
// pass the same barrier again before block_scan_excl reads it.
template <class S, bool REV, int K, int NW, int BAR = 0, class Comb>
__device__ __forceinline__ S block_scan_part1(const S (&agg)[K], S (&wex)[K], S* s_tot,
                                              const S& ident, Comb comb) {
    constexpr int Q = K * NW;
    constexpr int R = (Q + 31) / 32;
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
    scan_bar<BAR, NW>();
    S total = ident;
    if (warp == 0) {
        // with one total per lane (Q <= 32) the scan needs only the steps
        // that span lanes 0..Q-1, and the tile total is lane Q-1's
        constexpr int SPAN = R == 1 ? Q : 32;
        S v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = lane * R + r;
            v[r] = q < Q ? s_tot[q] : ident;
        }
        S run = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) run = comb(run, v[r]);
        S inc = run;
#pragma unroll
        for (int off = 1; off < SPAN; off <<= 1) {
            S o = shfl_up_s(inc, off);
            if (lane >= off) inc = comb(o, inc);
        }
        S ex = shfl_up_s(inc, 1);
        if (lane == 0) ex = ident;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = lane * R + r;
            if (q < Q) s_tot[q] = ex;
            ex = comb(ex, v[r]);
        }
        total = shfl_idx_s(inc, SPAN - 1);
    }
    return total;
}

// Part 2 when the tile's exclusive prefix is already folded into s_tot
// (block_fold_prefix) or is the identity: one combine per thread.
template <class S, bool REV, int K, int NW, class Comb>
__device__ __forceinline__ S block_scan_excl_folded(int k, const S (&wex)[K], const S* s_tot, Comb comb) {
    const int warp = threadIdx.x >> 5;
    return comb(s_tot[chunk_warp_pos<REV, K, NW>(k, warp)], wex[k]);
}

// Called by warp 0 (every lane holding the tile's exclusive prefix `pre`)
// after block_scan_part1 and before the barrier that precedes
// block_scan_excl_folded: folds pre into the K*NW per-warp prefixes once,
// instead of once per thread.
template <class S, int K, int NW, class Comb>
__device__ __forceinline__ void block_fold_prefix(S* s_tot, const S& pre, Comb comb) {
    constexpr int Q = K * NW;
    const int lane = threadIdx.x & 31;
    for (int q = lane; q < Q; q += 32) s_tot[q] = comb(pre, s_tot[q]);
}

// Part 2: the thread's exclusive prefix for chunk k, given the exclusive
// prefix of the whole tile (visible in shared memory after a sync).
template <class S, bool REV, int K, int NW, class Comb>
__device__ __forceinline__ S block_scan_excl(int k, const S (&wex)[K], const S* s_tot,
                                             const S& tile_prefix, Comb comb) {
    const int warp = threadIdx.x >> 5;
    return comb(tile_prefix, comb(s_tot[chunk_warp_pos<REV, K, NW>(k, warp)], wex[k]));
}

// Look-back slots of one single-pass scan.  Every tile has an aggregate
// slot and an inclusive-prefix slot; a slot holds the state S as 64-bit
// words whose high half is a status tag (1 = aggregate, 2 = inclusive)
// and whose low half is 32 bits of S.  Each word is written and read as
// one single-copy-atomic 64-bit access, so a reader that sees the tag in
// every word of a slot has the whole value: no fence on either side and
// one memory round trip per look-back window.  Slots start zeroed.
template <class S>
struct LookbackState {
    unsigned long long* agg;   // [tiles * words]
    unsigned long long* incl;  // [tiles * words]
};

template <class S>
constexpr int lb_words() {
    static_assert(sizeof(S) % 4 == 0, "4-byte granules");
    return (int)(sizeof(S) / 4);
}

template <class S>
__device__ __forceinline__ void lb_publish(unsigned long long* slot, const S& v, uint32_t tag) {
    constexpr int W = lb_words<S>();
    union { S s; uint32_t w[W]; } u;
    u.s = v;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const unsigned long long word = ((unsigned long long)tag << 32) | u.w[i];
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(slot + i), "l"(word) : "memory");
    }
}

// Reads a slot; returns true (and the value) if every word carries `tag`.
template <class S>
__device__ __forceinline__ bool lb_read(const unsigned long long* slot, uint32_t tag, S& out) {
    constexpr int W = lb_words<S>();
    union { S s; uint32_t w[W]; } u;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        unsigned long long word;
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(word) : "l"(slot + i) : "memory");
        ok = ok && (uint32_t)(word >> 32) == tag;
        u.w[i] = (uint32_t)word;
    }
    out = u.s;
    return ok;
}

// Polls tile idx until its inclusive prefix (returns 2) or aggregate
// (returns 1) is out; returns 0 after a timeout (status recorded).
template <class S>
__device__ __forceinline__ uint32_t lb_wait(const LookbackState<S>& st, int64_t idx, S& out,
                                            WsHeader* hdr) {
    constexpr int W = lb_words<S>();
    uint32_t it = 0;
    while (true) {
        S vi, va;
        const bool inc = lb_read(st.incl + idx * W, 2u, vi);
        const bool ag = lb_read(st.agg + idx * W, 1u, va);
        if (inc) { out = vi; return 2u; }
        if (ag) { out = va; return 1u; }
        ++it;
        if (it > kSpinLimit || ((it & 255u) == 0 && gave_up(hdr))) {
            record_status(hdr, ADPAR_ERR_TIMEOUT);
            return 0u;
        }
        __nanosleep(it < 32 ? 0 : 100);
    }
}

// Decoupled look-back, run by one whole warp for logical tile t.
// Publishes the tile's aggregate, walks back over the predecessors in
// windows of 32 (each lane polls one tile, bounded), stops at the first
// tile whose inclusive prefix is out, publishes this tile's inclusive
// prefix and returns the exclusive prefix (in every lane).
template <class S, class Comb>
__device__ __forceinline__ S lookback(int64_t t, LookbackState<S> st, const S& tile_total,
                                      const S& ident, Comb comb, WsHeader* hdr) {
    constexpr int W = lb_words<S>();
    const int lane = threadIdx.x & 31;
    if (t == 0) {
        if (lane == 0) lb_publish(st.incl, tile_total, 2u);
        return ident;
    }
    if (lane == 0) lb_publish(st.agg + t * W, tile_total, 1u);
    S prefix = ident;
    int64_t base = t - 1;
    while (true) {
        const int64_t idx = base - lane;
        uint32_t f = 2u;  // before tile 0: a virtual inclusive identity
        S v = ident;
        if (idx >= 0) f = lb_wait(st, idx, v, hdr);  // 0 only after a timeout
        const uint32_t stop_mask = __ballot_sync(0xffffffffu, f != 1u);
        const int stop = stop_mask ? __ffs(stop_mask) - 1 : 31;
        if (lane > stop || idx < 0 || f == 0u) v = ident;
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
    if (lane == 0) lb_publish(st.incl + t * W, comb(prefix, tile_total), 2u);
    return prefix;
}

}  // namespace adpar
