// Linear-recurrence scan VJP tiles of the batched launch, on per-thread
// runs (the rule and the two passes of scan_runs.cuh, Sec. 5.2), for
// segments of any length inside one persistent kernel of 256 threads.
//
// A tile is kBNT = 256 runs (one per thread) of one 128-byte row each.
//   forward tile t: folds its runs, scans them, looks back over the
//     segment's earlier tiles for its exclusive prefix, and stores every
//     run's exclusive carry (from the segment's start) and product of a;
//     then raises done[t].
//   reverse tile (tiles right to left): waits for done[t], re-forms the
//     primal from the run's carry, scans the runs' reverse transfers with a
//     look-back over the segment's later tiles, and writes the adjoints.
// Tiles move through shared memory by cooperative 16-byte loads and stores
// (segments have arbitrary addresses: no tensor maps), in the 128-byte
// swizzled layout of scan_runs.cuh; b goes straight into registers in the
// reverse tile.
#pragma once

#include "scan_runs.cuh"

namespace adpar {

constexpr int kBNT = 256;              // runs (threads) per batch tile
constexpr int kBArr = kBNT * 128;      // one array's tile in bytes (32 KB)
constexpr int kBRunSmem = 3 * kBArr;   // shared memory of a reverse tile

template <class T>
constexpr int brun_tile() {
    return kBNT * RunCfg<T>::V;  // elements per tile: 4096 FP64, 8192 FP32
}

// Thread 0 asks L2 for elements [lo, hi) of p (the whole 16-byte units):
// L2 fetches the whole range at once, so the block's own loads that follow
// wait for about one memory latency instead of one per batch of loads in
// flight.  p + lo must be 16-byte aligned.
template <class T>
__device__ __forceinline__ void range_prefetch_l2(const T* p, int64_t lo, int64_t hi) {
    const uint32_t bytes = (uint32_t)(((hi - lo) * (int64_t)sizeof(T)) & ~(int64_t)15);
    if (threadIdx.x == 0 && hi > lo && bytes > 0) tc::prefetch_l2(p + lo, bytes);
}

// a segment's runs state in the workspace
struct BRunState {
    unsigned long long* p_agg;   // forward look-back slots (RunP)
    unsigned long long* p_incl;
    unsigned long long* r_agg;   // reverse look-back slots (RunL)
    unsigned long long* r_incl;
    uint32_t* done;              // [tiles] a forward tile's carries are stored
    void* carA;                  // [tiles * kBNT] A before the run (from the segment's start)
    void* carB;                  // [tiles * kBNT] B before the run
    void* prod;                  // [tiles * kBNT] product of a over the run
};

// one array's tile into the swizzled layout: 16-byte chunk i of the tile is
// chunk i % 8 of run i / 8; past the end of the data, pad
template <class T>
__device__ __forceinline__ void brun_load(unsigned char* dst, const T* src, int64_t e0, int64_t n, T pad) {
    constexpr int EPC = RunCfg<T>::EPC;
    const bool whole = e0 + (int64_t)brun_tile<T>() <= n;
#pragma unroll 4
    for (int i = threadIdx.x; i < kBNT * kRunChunks; i += kBNT) {
        const int64_t e = e0 + (int64_t)i * EPC;
        RunVec<T> v;
        if (whole) {
            v = *reinterpret_cast<const RunVec<T>*>(src + e);
        } else {
#pragma unroll
            for (int j = 0; j < EPC; ++j) v.v[j] = e + j < n ? src[e + j] : pad;
        }
        run_st<T>(dst, run_chunk_off(i / kRunChunks, i % kRunChunks), v);
    }
}

// the inverse: a tile of outputs from the swizzled layout to global memory
template <class T>
__device__ __forceinline__ void brun_store(T* dst, const unsigned char* src, int64_t e0, int64_t n) {
    constexpr int EPC = RunCfg<T>::EPC;
    const bool whole = e0 + (int64_t)brun_tile<T>() <= n;
#pragma unroll 4
    for (int i = threadIdx.x; i < kBNT * kRunChunks; i += kBNT) {
        const int64_t e = e0 + (int64_t)i * EPC;
        const RunVec<T> v = run_ld<T>(src, run_chunk_off(i / kRunChunks, i % kRunChunks));
        if (whole) {
            *reinterpret_cast<RunVec<T>*>(dst + e) = v;
        } else {
#pragma unroll
            for (int j = 0; j < EPC; ++j)
                if (e + j < n) dst[e + j] = v.v[j];
        }
    }
}

template <class T>
__device__ void brun_fwd_tile(const T* a, const T* b, int64_t n, const BRunState& S, int64_t tile,
                              unsigned char* smem, WsHeader* hdr) {
    using P = RunP<T>;
    constexpr int NW = kBNT / 32;
    __shared__ P s_totP[NW];
    unsigned char* sA = smem;
    unsigned char* sB = smem + kBArr;
    const int64_t e0 = tile * brun_tile<T>();
    const int64_t e1 = min(n, e0 + (int64_t)brun_tile<T>());
    range_prefetch_l2(a, e0, e1);
    range_prefetch_l2(b, e0, e1);
    brun_load<T>(sA, a, e0, n, T(1));  // (1, 0) is the neutral element
    brun_load<T>(sB, b, e0, n, T(0));
    __syncthreads();
    const int t = threadIdx.x;
    T A = T(1), B = T(0);
#pragma unroll
    for (int p = 0; p < kRunChunks; ++p) {
        const RunVec<T> x = run_ld<T>(sA, run_chunk_off(t, p));
        const RunVec<T> y = run_ld<T>(sB, run_chunk_off(t, p));
#pragma unroll
        for (int j = 0; j < RunCfg<T>::EPC; ++j) {
            B = run_fma(x.v[j], B, y.v[j]);
            A *= x.v[j];
        }
    }
    const P agg[1] = {P{A, B}};
    auto comb = [](const P& l, const P& r) { return P{l.A * r.A, run_fma(r.A, l.B, r.B)}; };
    const P ident{T(1), T(0)};
    P wex[1];
    const P total = block_scan_part1<P, false, 1, NW>(agg, wex, s_totP, ident, comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<P> st{S.p_agg, S.p_incl};
        const P pre = lookback(tile, st, total, ident, comb, hdr);
        block_fold_prefix<P, 1, NW>(s_totP, pre, comb);
    }
    __syncthreads();
    const P ex = block_scan_excl_folded<P, false, 1, NW>(0, wex, s_totP, comb);
    const int64_t run = tile * kBNT + t;
    static_cast<T*>(S.carA)[run] = ex.A;
    static_cast<T*>(S.carB)[run] = ex.B;
    static_cast<T*>(S.prod)[run] = A;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release_u32(S.done + tile, 1u);
}

template <class T>
__device__ void brun_rev_tile(const T* a, const T* b, const T* ya, const T* yb, T* abar, T* bbar, int64_t n,
                              const BRunState& S, int64_t tiles, int64_t t_log, unsigned char* smem,
                              WsHeader* hdr) {
    using L = RunL<T>;
    constexpr int V = RunCfg<T>::V, EPC = RunCfg<T>::EPC, NW = kBNT / 32;
    __shared__ L s_totL[NW];
    __shared__ int s_ok;
    unsigned char* sA = smem;
    unsigned char* sYA = smem + kBArr;      // ybar_A, then abar
    unsigned char* sYB = smem + 2 * kBArr;  // ybar_B, then bbar
    const int64_t tile = tiles - 1 - t_log;  // right to left
    const int64_t e0 = tile * brun_tile<T>();
    const int t = threadIdx.x;
    const int64_t e1 = min(n, e0 + (int64_t)brun_tile<T>());
    range_prefetch_l2(a, e0, e1);
    range_prefetch_l2(ya, e0, e1);
    range_prefetch_l2(yb, e0, e1);
    range_prefetch_l2(b, e0, e1);
    // the cotangents and a need no carry: their tiles load first
    brun_load<T>(sA, a, e0, n, T(1));
    brun_load<T>(sYA, ya, e0, n, T(0));
    brun_load<T>(sYB, yb, e0, n, T(0));
    if (threadIdx.x == 0) s_ok = wait_flag(S.done + tile, hdr) != 0u;
    __syncthreads();
    const int64_t run = tile * kBNT + t;
    T PA = T(1), PB = T(0), cprod = T(1);
    if (s_ok) {  // else a timeout is recorded: finish without the carries
        PA = ld_cg(static_cast<const T*>(S.carA) + run);
        PB = ld_cg(static_cast<const T*>(S.carB) + run);
        cprod = ld_cg(static_cast<const T*>(S.prod) + run);
    }
    T Bp[V];  // b_j, then B_{j-1}
    {
        const int64_t r0 = e0 + (int64_t)t * V;
        if (r0 + V <= n) {
#pragma unroll
            for (int p = 0; p < kRunChunks; ++p) {
                const RunVec<T> v = *reinterpret_cast<const RunVec<T>*>(b + r0 + EPC * p);
#pragma unroll
                for (int j = 0; j < EPC; ++j) Bp[EPC * p + j] = v.v[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) Bp[j] = r0 + j < n ? b[r0 + j] : T(0);
        }
    }
    // the primal from the carry: A_{j-1} and B_{j-1} in registers
    T Aprev[V];
    {
        T A = PA, B = PB;
#pragma unroll
        for (int p = 0; p < kRunChunks; ++p) {
            const RunVec<T> x = run_ld<T>(sA, run_chunk_off(t, p));
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const T bj = Bp[EPC * p + j];
                Aprev[EPC * p + j] = A;
                Bp[EPC * p + j] = B;
                B = run_fma(x.v[j], B, bj);
                A *= x.v[j];
            }
        }
    }
    // the run's reverse transfer: R_j = ybar_j + a_{j+1} R_{j+1}
    T RA = T(0), RB = T(0), a_next = T(0);
#pragma unroll
    for (int p = kRunChunks - 1; p >= 0; --p) {
        const int off = run_chunk_off(t, p);
        const RunVec<T> y1 = run_ld<T>(sYA, off);
        const RunVec<T> y2 = run_ld<T>(sYB, off);
        const RunVec<T> aa = run_ld<T>(sA, off);
#pragma unroll
        for (int j = EPC - 1; j >= 0; --j) {
            if (p == kRunChunks - 1 && j == EPC - 1) {  // R_e = ybar_e (no FMA)
                RA = y1.v[j];
                RB = y2.v[j];
            } else {
                RA = run_fma(a_next, RA, y1.v[j]);
                RB = run_fma(a_next, RB, y2.v[j]);
            }
            a_next = aa.v[j];
        }
    }
    const L agg[1] = {L{cprod, a_next * RA, a_next * RB}};
    auto comb = [](const L& x, const L& y) {
        return L{y.c * x.c, run_fma(y.c, x.dA, y.dA), run_fma(y.c, x.dB, y.dB)};
    };
    const L ident{T(1), T(0), T(0)};
    L wex[1];
    const L total = block_scan_part1<L, true, 1, NW>(agg, wex, s_totL, ident, comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<L> st{S.r_agg, S.r_incl};
        const L pre = lookback(t_log, st, total, ident, comb, hdr);
        block_fold_prefix<L, 1, NW>(s_totL, pre, comb);
    }
    __syncthreads();
    const L ex = block_scan_excl_folded<L, true, 1, NW>(0, wex, s_totL, comb);
    // rs_bar right to left and the outputs, over the cotangents' tiles
    {
        T rA = ex.dA, rB = ex.dB;
        T a_up = T(1);
#pragma unroll
        for (int p = kRunChunks - 1; p >= 0; --p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> y1 = run_ld<T>(sYA, off);
            const RunVec<T> y2 = run_ld<T>(sYB, off);
            const RunVec<T> aa = run_ld<T>(sA, off);
            RunVec<T> oa, ob;
#pragma unroll
            for (int j = EPC - 1; j >= 0; --j) {
                rA = run_fma(a_up, rA, y1.v[j]);
                rB = run_fma(a_up, rB, y2.v[j]);
                oa.v[j] = run_fma(Aprev[EPC * p + j], rA, Bp[EPC * p + j] * rB);
                ob.v[j] = rB;
                a_up = aa.v[j];
            }
            run_st<T>(sYA, off, oa);
            run_st<T>(sYB, off, ob);
        }
    }
    __syncthreads();
    brun_store<T>(abar, sYA, e0, n);
    brun_store<T>(bbar, sYB, e0, n);
}

}  // namespace adpar
