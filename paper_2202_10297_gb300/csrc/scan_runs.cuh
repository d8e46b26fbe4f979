// The linear-recurrence scan VJP with per-thread runs (Sec. 5.2's rule for
// (a1,b1) (.) (a2,b2) = (a2 a1, a2 b1 + b2)), in FP64 and FP32.  In FP64 the
// GB300's FP64 rate (2 lanes per SM per clock) rather than HBM bounds this
// operator; in FP32 HBM does.
//
// Every thread owns a run of V consecutive elements (one 128-byte row: 16
// doubles or 32 floats), so the per-element work is plain sequential
// recurrences and the block-level scans (a few operations per combine) run
// once per run instead of once per element:
//
//  pass C (forward): fold each run into its primal aggregate (prod of a, B
//     over the run: 2 operations per element), scan the runs of a tile, and
//     store per run the exclusive carry from the tile's start and the run's
//     product of a, and per tile its aggregate; one block then scans the
//     tile aggregates into the state before each tile (no look-back: a pass
//     that writes little per element has nothing to hide one behind).
//  pass R (reverse, tiles right to left), per run, with U_j = a_j rs_bar_j
//     (the adjoint flowing left out of element j):
//     1. the primal from the run's carry: A_{j-1}, B_{j-1} (2 per element);
//     2. the run's transfer U_{e+1} -> U_s = d + c U_{e+1}: c = the product
//        of a over the run (from pass C), d = a_s * the local reverse fold
//        R_j = ybar_j + a_{j+1} R_{j+1} (2 per element);
//     3. the reverse scan of the transfers over the tile's runs and the
//        look-back across tiles give each run its incoming U_{e+1};
//     4. rs_bar_j = ybar_j + a_{j+1} rs_bar_{j+1} (rs_bar_e = ybar_e + U_{e+1})
//        and the outputs abar_j = A_{j-1} rsA_j + B_{j-1} rsB_j,
//        bbar_j = rsB_j (4 per element).
//  That is 10 operations per element plus a share of the run scans, and
//  (2 + 4 + 2) element sizes of HBM traffic per element plus 3 per run.
//
// A tile is NT runs; each input array's tile (NT runs of 128 bytes)
// comes into shared memory by one 3-D TMA copy with the 128-byte swizzle
// (in the reverse pass b instead goes straight into registers)
// (16-byte chunk c of 128-byte row r stored at chunk c ^ (r & 7)), so that a
// thread reading its own run with 16-byte loads meets few bank conflicts.
// The outputs are written back into the cotangents' tiles and stored by TMA.
// A tile that is not whole (the last one) is loaded and stored element by
// element with bounds checks, in the same layout.
#pragma once

#include <cuda.h>

#include "scan_engine.cuh"
#include "tc.cuh"

namespace adpar {

constexpr int kRunChunks = 8;  // 16-byte chunks per run
// L2 prefetch distances in tiles: a block asks L2 for the inputs of the
// tile this many tiles further on in its pass's order, so that HBM reads run
// ahead of the tiles that hold shared memory (passes reading two arrays per
// tile use C, four arrays R; FP32 at 2^26 pairs, carry + reverse pass: no
// prefetch 0.440 ms, C/R = 608/304 0.433, 304/152 0.417, 152/76 0.413)
constexpr int kRunAheadC = 152;
constexpr int kRunAheadR = 76;

template <class T>
struct RunCfg {
    static constexpr int V = 128 / (int)sizeof(T);   // elements per run
    static constexpr int EPC = 16 / (int)sizeof(T);  // elements per 16-byte chunk
    // runs (threads) per tile (tiles of 64 runs were slower at 2^26: FP32
    // 0.52 -> 0.59 ms, FP64 1.94 -> 2.23 ms)
    static constexpr int NT = 128;
    static constexpr int NW = NT / 32;               // warps per tile
    static constexpr int TILE = V * NT;              // elements per tile
    static constexpr int ARR = NT * 128;             // one array's tile in bytes
};

template <class T>
struct alignas(16) RunVec {
    T v[16 / sizeof(T)];
};

template <class T>
struct RunP {  // primal state (A, B)
    T A, B;
};
template <class T>
struct RunL {  // reverse transfer U -> d + c U, for both components
    T c, dA, dB;
};

__device__ __forceinline__ double run_fma(double x, double y, double z) { return fma(x, y, z); }
__device__ __forceinline__ float run_fma(float x, float y, float z) { return fmaf(x, y, z); }

// the primal operator on RunP, in the shape the carry scan takes
template <class T>
struct RunPOp {
    using P = RunP<T>;
    __device__ static P pid() { return P{T(1), T(0)}; }
    __device__ static P pcomb(const P& l, const P& r) { return P{l.A * r.A, run_fma(r.A, l.B, r.B)}; }
};

template <class T>
struct RunArgs {
    int64_t n;
    int64_t tiles;
    const T* a;
    const T* b;
    const T* ya;
    const T* yb;
    T* abar;
    T* bbar;
    int accumulate;
    WsHeader* hdr;
    unsigned long long* lbR_agg;
    unsigned long long* lbR_incl;
    T* carA;        // [tiles * NT] A before the run, from the tile's start
    T* carB;        // [tiles * NT] B before the run, from the tile's start
    T* prod;        // [tiles * NT] product of a over the run
    RunP<T>* tagg;  // [tiles] the tile's primal aggregate
    RunP<T>* tcar;  // [tiles] the primal state before the tile
};

// byte offset of 16-byte chunk p of run t in a swizzled array tile
__device__ __forceinline__ int run_chunk_off(int t, int p) { return t * 128 + (((p & 7) ^ (t & 7)) << 4); }

template <class T>
__device__ __forceinline__ RunVec<T> run_ld(const unsigned char* base, int off) {
    return *reinterpret_cast<const RunVec<T>*>(base + off);
}
template <class T>
__device__ __forceinline__ void run_st(unsigned char* base, int off, const RunVec<T>& v) {
    *reinterpret_cast<RunVec<T>*>(base + off) = v;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            tc::smem_u32(dst)),
        "l"(tm), "r"(0), "r"(0), "r"(z), "r"(tc::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tm), "r"(0),
                 "r"(0), "r"(z), "r"(tc::smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait_read() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// One tile's arrays into shared memory: TMA when the tile is whole, else
// element by element (pad past the end of the data).  All threads call it;
// on return the data is visible to the block.
template <class T, int NA>
__device__ __forceinline__ void run_tile_load(unsigned char* const (&dst)[NA], const CUtensorMap* const (&tm)[NA],
                                              const T* const (&src)[NA], const T (&pad)[NA], bool whole,
                                              int64_t tile, int64_t n, uint64_t* bar, WsHeader* hdr) {
    using Cf = RunCfg<T>;
    if (whole) {
        if (threadIdx.x == 0) {
            tc::mbar_init(bar, 1);
            tc::fence_mbar_init();
            tc::mbar_arrive_expect_tx(bar, (uint32_t)(NA * Cf::ARR));
#pragma unroll
            for (int q = 0; q < NA; ++q) tma_load_3d(dst[q], tm[q], (int)(tile * Cf::NT), bar);
        }
        __syncthreads();
        bool ok = false;
        for (uint32_t w = 0; w < (1u << 20) && !ok; ++w) ok = tc::mbar_try_wait(bar, 0u);
        if (!ok) record_status(hdr, ADPAR_ERR_TIMEOUT);
    } else {
        const int64_t e0 = tile * Cf::TILE;
        for (int i = threadIdx.x; i < Cf::NT * kRunChunks; i += Cf::NT) {
            const int t = i / kRunChunks, p = i % kRunChunks;
            const int64_t e = e0 + (int64_t)t * Cf::V + Cf::EPC * p;
            const int off = run_chunk_off(t, p);
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                RunVec<T> v;
#pragma unroll
                for (int j = 0; j < Cf::EPC; ++j) v.v[j] = e + j < n ? src[q][e + j] : pad[q];
                run_st<T>(dst[q], off, v);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- pass C
template <class T>
__global__ void __launch_bounds__(RunCfg<T>::NT) linrec_runs_carry_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB,
                                                                   RunArgs<T> R) {
    using Cf = RunCfg<T>;
    using P = RunP<T>;
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    unsigned char* sA = s_dyn;
    unsigned char* sB = s_dyn + Cf::ARR;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ P s_tot[Cf::NW];
    const int64_t tile = blockIdx.x;
    const bool whole = (tile + 1) * Cf::TILE <= R.n;
    if (threadIdx.x == 0 && (tile + kRunAheadC + 1) * Cf::TILE <= R.n) {
        tc::prefetch_l2(R.a + (tile + kRunAheadC) * Cf::TILE, Cf::ARR);
        tc::prefetch_l2(R.b + (tile + kRunAheadC) * Cf::TILE, Cf::ARR);
    }
    {
        unsigned char* const dst[2] = {sA, sB};
        const CUtensorMap* const tm[2] = {&tmA, &tmB};
        const T* const src[2] = {R.a, R.b};
        const T pad[2] = {T(1), T(0)};  // (1, 0) is the neutral element
        run_tile_load<T, 2>(dst, tm, src, pad, whole, tile, R.n, &s_bar, R.hdr);
    }
    const int t = threadIdx.x;
    T A = T(1), B = T(0);
#pragma unroll
    for (int p = 0; p < kRunChunks; ++p) {
        const RunVec<T> x = run_ld<T>(sA, run_chunk_off(t, p));
        const RunVec<T> y = run_ld<T>(sB, run_chunk_off(t, p));
#pragma unroll
        for (int j = 0; j < Cf::EPC; ++j) {
            B = run_fma(x.v[j], B, y.v[j]);
            A *= x.v[j];
        }
    }
    const P agg[1] = {P{A, B}};
    auto comb = [](const P& l, const P& r) { return P{l.A * r.A, run_fma(r.A, l.B, r.B)}; };
    P wex[1];
    const P ident{T(1), T(0)};
    const P total = block_scan_part1<P, false, 1, Cf::NW>(agg, wex, s_tot, ident, comb);
    if (threadIdx.x == 0) R.tagg[tile] = total;
    __syncthreads();
    const P ex = block_scan_excl_folded<P, false, 1, Cf::NW>(0, wex, s_tot, comb);  // from the tile's start
    const int64_t run = tile * Cf::NT + t;
    R.carA[run] = ex.A;
    R.carB[run] = ex.B;
    R.prod[run] = A;
}

// ---------------------------------------------------------------- pass R
// four blocks per SM (FP64 spills a few registers at that bound; three
// blocks without spills measured 1.88 against 1.76 ms at 2^26)
template <class T>
__global__ void __launch_bounds__(RunCfg<T>::NT, 4) linrec_runs_vjp_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmYA,
    const __grid_constant__ CUtensorMap tmYB, const __grid_constant__ CUtensorMap tmOA,
    const __grid_constant__ CUtensorMap tmOB, RunArgs<T> R) {
    using Cf = RunCfg<T>;
    using L = RunL<T>;
    constexpr int V = Cf::V, EPC = Cf::EPC;
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    unsigned char* sA = s_dyn;
    unsigned char* sYA = s_dyn + Cf::ARR;      // ybar_A, then abar
    unsigned char* sYB = s_dyn + 2 * Cf::ARR;  // ybar_B, then bbar
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tile;
    __shared__ L s_tot[Cf::NW];
    if (threadIdx.x == 0) s_tile = atomicAdd(&R.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;
    const int64_t tile = R.tiles - 1 - t_log;  // tiles are taken right to left
    const bool whole = (tile + 1) * Cf::TILE <= R.n;
    const int t = threadIdx.x;
    if (t == 0 && tile >= kRunAheadR) {  // a tile left of another is whole
        const int64_t e = (tile - kRunAheadR) * Cf::TILE;
        tc::prefetch_l2(R.a + e, Cf::ARR);
        tc::prefetch_l2(R.b + e, Cf::ARR);
        tc::prefetch_l2(R.ya + e, Cf::ARR);
        tc::prefetch_l2(R.yb + e, Cf::ARR);
    }
    const int64_t run = tile * Cf::NT + t;
    // the run's carry (the state before the tile, then the run's local
    // carry within it) and product (pass C) load while the tile arrives
    const RunP<T> tc0 = R.tcar[tile];
    const T lA = R.carA[run], lB = R.carB[run], cprod = R.prod[run];
    const T PA = tc0.A * lA, PB = run_fma(lA, tc0.B, lB);
    // b is read once, by its own thread: straight from global memory into
    // registers (its 128-byte row in eight 16-byte loads), so that the tile
    // holds three arrays in shared memory and four tiles fit on an SM
    T Bp[V];  // b_j, then B_{j-1}
    {
        const int64_t e0 = tile * Cf::TILE + (int64_t)t * V;
        if (whole) {
#pragma unroll
            for (int p = 0; p < kRunChunks; ++p) {
                const RunVec<T> v = *reinterpret_cast<const RunVec<T>*>(R.b + e0 + EPC * p);
#pragma unroll
                for (int j = 0; j < EPC; ++j) Bp[EPC * p + j] = v.v[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) Bp[j] = e0 + j < R.n ? R.b[e0 + j] : T(0);
        }
    }
    {
        unsigned char* const dst[3] = {sA, sYA, sYB};
        const CUtensorMap* const tm[3] = {&tmA, &tmYA, &tmYB};
        const T* const src[3] = {R.a, R.ya, R.yb};
        const T pad[3] = {T(1), T(0), T(0)};
        run_tile_load<T, 3>(dst, tm, src, pad, whole, tile, R.n, &s_bar, R.hdr);
    }

    // 1. the primal from the carry: A_{j-1} and B_{j-1} in registers
    T Aprev[V];
    {
        T A = PA, B = PB;
#pragma unroll
        for (int p = 0; p < kRunChunks; ++p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> x = run_ld<T>(sA, off);
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
    // 2. the run's reverse transfer: R_j = ybar_j + a_{j+1} R_{j+1}, from
    //    R_e = ybar_e; a_next ends as a_s, the run's first a
    T RA = T(0), RB = T(0), a_next = T(0);
#pragma unroll
    for (int p = kRunChunks - 1; p >= 0; --p) {
        const int off = run_chunk_off(t, p);
        const RunVec<T> ya = run_ld<T>(sYA, off);
        const RunVec<T> yb = run_ld<T>(sYB, off);
        const RunVec<T> aa = run_ld<T>(sA, off);
#pragma unroll
        for (int j = EPC - 1; j >= 0; --j) {
            if (p == kRunChunks - 1 && j == EPC - 1) {  // R_e = ybar_e (no FMA)
                RA = ya.v[j];
                RB = yb.v[j];
            } else {
                RA = run_fma(a_next, RA, ya.v[j]);
                RB = run_fma(a_next, RB, yb.v[j]);
            }
            a_next = aa.v[j];
        }
    }
    const L agg[1] = {L{cprod, a_next * RA, a_next * RB}};
    // 3. scan of the transfers, right to left: comb(x, y) with x to the
    //    right of y is "x, then y"
    auto comb = [](const L& x, const L& y) {
        return L{y.c * x.c, run_fma(y.c, x.dA, y.dA), run_fma(y.c, x.dB, y.dB)};
    };
    const L ident{T(1), T(0), T(0)};
    L wex[1];
    const L total = block_scan_part1<L, true, 1, Cf::NW>(agg, wex, s_tot, ident, comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<L> st{R.lbR_agg, R.lbR_incl};
        const L pre = lookback(t_log, st, total, ident, comb, R.hdr);
        block_fold_prefix<L, 1, Cf::NW>(s_tot, pre, comb);
    }
    __syncthreads();
    const L ex = block_scan_excl_folded<L, true, 1, Cf::NW>(0, wex, s_tot, comb);

    // 4. rs_bar right to left and the outputs, written over the cotangents;
    //    rs_bar_e = ybar_e + U_{e+1} with U_{e+1} = ex.d (a_up starts at 1)
    {
        T rA = ex.dA, rB = ex.dB;  // U entering the run's last element
        T a_up = T(1);             // a_{j+1} (the factor carried into U)
#pragma unroll
        for (int p = kRunChunks - 1; p >= 0; --p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> ya = run_ld<T>(sYA, off);
            const RunVec<T> yb = run_ld<T>(sYB, off);
            const RunVec<T> aa = run_ld<T>(sA, off);
            RunVec<T> oa, ob;
#pragma unroll
            for (int j = EPC - 1; j >= 0; --j) {
                rA = run_fma(a_up, rA, ya.v[j]);
                rB = run_fma(a_up, rB, yb.v[j]);
                oa.v[j] = run_fma(Aprev[EPC * p + j], rA, Bp[EPC * p + j] * rB);
                ob.v[j] = rB;
                a_up = aa.v[j];
            }
            run_st<T>(sYA, off, oa);
            run_st<T>(sYB, off, ob);
        }
    }

    if (whole && !R.accumulate) {
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_3d(&tmOA, (int)(tile * Cf::NT), sYA);
            tma_store_3d(&tmOB, (int)(tile * Cf::NT), sYB);
            bulk_commit_and_wait_read();
        }
        __syncthreads();
    } else {
        const int64_t e0 = tile * Cf::TILE + (int64_t)t * V;
#pragma unroll 2
        for (int p = 0; p < kRunChunks; ++p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> oa = run_ld<T>(sYA, off);
            const RunVec<T> ob = run_ld<T>(sYB, off);
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const int64_t e = e0 + EPC * p + j;
                if (e < R.n) {
                    R.abar[e] = R.accumulate ? R.abar[e] + oa.v[j] : oa.v[j];
                    R.bbar[e] = R.accumulate ? R.bbar[e] + ob.v[j] : ob.v[j];
                }
            }
        }
    }
}

}  // namespace adpar

// ------------------------------------------------- forward mode (JVP)
// The tangent of the linear-recurrence scan (Sec. 3's dual numbers through
// the operator): one single-pass scan of dual states (A, B, dA, dB) on
// per-thread runs.  A tile folds each run from the identity (6 operations
// per element), scans the runs, looks back over the earlier tiles for its
// exclusive prefix, then re-folds every run from its exclusive carry and
// writes the inclusive tangents (and, when asked, the primal) over the
// input tiles, which leave by TMA.
namespace adpar {

template <class T>
struct RunD {  // dual primal state
    T A, B, dA, dB;
};

// one element (x = a_j, y = b_j, dx, dy) folded into a dual state
template <class T>
__device__ __forceinline__ void rund_push(RunD<T>& s, T x, T y, T dx, T dy) {
    s.dB = run_fma(dx, s.B, run_fma(x, s.dB, dy));  // d(x B + y)
    s.B = run_fma(x, s.B, y);
    s.dA = run_fma(dx, s.A, x * s.dA);  // d(x A)
    s.A = x * s.A;
}

template <class T>
struct RunJvpArgs {
    int64_t n;
    int64_t tiles;
    const T* a;
    const T* b;
    const T* ad;
    const T* bd;
    T* ys_a;  // nullable
    T* ys_b;
    T* yd_a;
    T* yd_b;
    WsHeader* hdr;
    unsigned long long* lb_agg;
    unsigned long long* lb_incl;
};

template <class T>
__global__ void __launch_bounds__(RunCfg<T>::NT) linrec_runs_jvp_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmAD, const __grid_constant__ CUtensorMap tmBD,
    const __grid_constant__ CUtensorMap tmYA, const __grid_constant__ CUtensorMap tmYB,
    const __grid_constant__ CUtensorMap tmDA, const __grid_constant__ CUtensorMap tmDB, RunJvpArgs<T> R) {
    using Cf = RunCfg<T>;
    using D = RunD<T>;
    constexpr int EPC = Cf::EPC;
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    unsigned char* sA = s_dyn;                 // a, then ys_a
    unsigned char* sB = s_dyn + Cf::ARR;       // b, then ys_b
    unsigned char* sAD = s_dyn + 2 * Cf::ARR;  // adot, then ysdot_a
    unsigned char* sBD = s_dyn + 3 * Cf::ARR;  // bdot, then ysdot_b
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tile;
    __shared__ D s_tot[Cf::NW];
    if (threadIdx.x == 0) s_tile = atomicAdd(&R.hdr->ticket[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const bool whole = (tile + 1) * Cf::TILE <= R.n;
    const int t = threadIdx.x;
    if (t == 0 && (tile + kRunAheadR + 1) * Cf::TILE <= R.n) {
        const int64_t e = (tile + kRunAheadR) * Cf::TILE;
        tc::prefetch_l2(R.a + e, Cf::ARR);
        tc::prefetch_l2(R.b + e, Cf::ARR);
        tc::prefetch_l2(R.ad + e, Cf::ARR);
        tc::prefetch_l2(R.bd + e, Cf::ARR);
    }
    {
        unsigned char* const dst[4] = {sA, sB, sAD, sBD};
        const CUtensorMap* const tm[4] = {&tmA, &tmB, &tmAD, &tmBD};
        const T* const src[4] = {R.a, R.b, R.ad, R.bd};
        const T pad[4] = {T(1), T(0), T(0), T(0)};  // the identity element with a zero tangent
        run_tile_load<T, 4>(dst, tm, src, pad, whole, tile, R.n, &s_bar, R.hdr);
    }
    const D ident{T(1), T(0), T(0), T(0)};
    D run = ident;
#pragma unroll
    for (int p = 0; p < kRunChunks; ++p) {
        const int off = run_chunk_off(t, p);
        const RunVec<T> x = run_ld<T>(sA, off), y = run_ld<T>(sB, off);
        const RunVec<T> dx = run_ld<T>(sAD, off), dy = run_ld<T>(sBD, off);
#pragma unroll
        for (int j = 0; j < EPC; ++j) rund_push(run, x.v[j], y.v[j], dx.v[j], dy.v[j]);
    }
    // l then r
    auto comb = [](const D& l, const D& r) {
        return D{r.A * l.A, run_fma(r.A, l.B, r.B), run_fma(r.dA, l.A, r.A * l.dA),
                 run_fma(r.dA, l.B, run_fma(r.A, l.dB, r.dB))};
    };
    const D agg[1] = {run};
    D wex[1];
    const D total = block_scan_part1<D, false, 1, Cf::NW>(agg, wex, s_tot, ident, comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<D> st{R.lb_agg, R.lb_incl};
        const D pre = lookback(tile, st, total, ident, comb, R.hdr);
        block_fold_prefix<D, 1, Cf::NW>(s_tot, pre, comb);
    }
    __syncthreads();
    D s = block_scan_excl_folded<D, false, 1, Cf::NW>(0, wex, s_tot, comb);
    const bool want_ys = R.ys_a != nullptr;
    // re-fold from the exclusive carry: the inclusive outputs over the inputs
#pragma unroll
    for (int p = 0; p < kRunChunks; ++p) {
        const int off = run_chunk_off(t, p);
        const RunVec<T> x = run_ld<T>(sA, off), y = run_ld<T>(sB, off);
        const RunVec<T> dx = run_ld<T>(sAD, off), dy = run_ld<T>(sBD, off);
        RunVec<T> oA, oB, oDA, oDB;
#pragma unroll
        for (int j = 0; j < EPC; ++j) {
            rund_push(s, x.v[j], y.v[j], dx.v[j], dy.v[j]);
            oA.v[j] = s.A;
            oB.v[j] = s.B;
            oDA.v[j] = s.dA;
            oDB.v[j] = s.dB;
        }
        if (want_ys) {
            run_st<T>(sA, off, oA);
            run_st<T>(sB, off, oB);
        }
        run_st<T>(sAD, off, oDA);
        run_st<T>(sBD, off, oDB);
    }
    if (whole) {
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_3d(&tmDA, (int)(tile * Cf::NT), sAD);
            tma_store_3d(&tmDB, (int)(tile * Cf::NT), sBD);
            if (want_ys) {
                tma_store_3d(&tmYA, (int)(tile * Cf::NT), sA);
                tma_store_3d(&tmYB, (int)(tile * Cf::NT), sB);
            }
            bulk_commit_and_wait_read();
        }
        __syncthreads();
    } else {
        const int64_t e0 = tile * Cf::TILE + (int64_t)t * Cf::V;
#pragma unroll 2
        for (int p = 0; p < kRunChunks; ++p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> oA = run_ld<T>(sA, off), oB = run_ld<T>(sB, off);
            const RunVec<T> oDA = run_ld<T>(sAD, off), oDB = run_ld<T>(sBD, off);
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const int64_t e = e0 + EPC * p + j;
                if (e < R.n) {
                    R.yd_a[e] = oDA.v[j];
                    R.yd_b[e] = oDB.v[j];
                    if (want_ys) {
                        R.ys_a[e] = oA.v[j];
                        R.ys_b[e] = oB.v[j];
                    }
                }
            }
        }
    }
}

}  // namespace adpar

// --------------------------------------- reduce VJP, general rule (LINREC)
// The VJP of y = reduce (.) as for the linear recurrence by the general rule
// of Sec. 5.1: with l_i the composite of the elements before i and r_i of
// those after it, y = l_i (.) as_i (.) r_i, so abar_i = A(r_i) (ybar_A A(l_i)
// + ybar_B B(l_i)) and bbar_i = A(r_i) ybar_B, where A(r_i) is the product of
// the a after i.  After the carry pass (run carries and products, tile
// carries), a reverse pass per tile re-forms l from the run's carry (2
// operations per element, plus 2 for ybar_A A + ybar_B B), scans the runs'
// products of a right to left with a look-back over the later tiles for
// A(r), and forms the outputs (3 per element): 7 per element here and 2 in
// the carry pass.
namespace adpar {

template <class T>
struct RunS {  // a product of a (scalar look-back state)
    T c;
};

template <class T>
__global__ void __launch_bounds__(RunCfg<T>::NT, 4) linrec_runs_reduce_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmOA, const __grid_constant__ CUtensorMap tmOB, RunArgs<T> R,
    const T* ybar_a, const T* ybar_b, T* y_a, T* y_b) {
    using Cf = RunCfg<T>;
    using S = RunS<T>;
    constexpr int V = Cf::V, EPC = Cf::EPC;
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    unsigned char* sA = s_dyn;            // a, then abar
    unsigned char* sB = s_dyn + Cf::ARR;  // b, then bbar
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tile;
    __shared__ S s_tot[Cf::NW];
    if (threadIdx.x == 0) s_tile = atomicAdd(&R.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;
    const int64_t tile = R.tiles - 1 - t_log;  // tiles are taken right to left
    const bool whole = (tile + 1) * Cf::TILE <= R.n;
    const int t = threadIdx.x;
    if (t == 0 && tile >= kRunAheadC) {  // a tile left of another is whole
        tc::prefetch_l2(R.a + (tile - kRunAheadC) * Cf::TILE, Cf::ARR);
        tc::prefetch_l2(R.b + (tile - kRunAheadC) * Cf::TILE, Cf::ARR);
    }
    const int64_t run = tile * Cf::NT + t;
    const RunP<T> tc0 = R.tcar[tile];
    const T lA = R.carA[run], lB = R.carB[run], cprod = R.prod[run];
    const T PA = tc0.A * lA, PB = run_fma(lA, tc0.B, lB);
    const T yA = *ybar_a, yB = *ybar_b;
    if (y_a && t_log == 0 && threadIdx.x == 0) {  // y: the state before the last tile, then the tile
        const RunP<T> ag = R.tagg[tile];
        *y_a = tc0.A * ag.A;
        *y_b = run_fma(ag.A, tc0.B, ag.B);
    }
    {
        unsigned char* const dst[2] = {sA, sB};
        const CUtensorMap* const tm[2] = {&tmA, &tmB};
        const T* const src[2] = {R.a, R.b};
        const T pad[2] = {T(1), T(0)};
        run_tile_load<T, 2>(dst, tm, src, pad, whole, tile, R.n, &s_bar, R.hdr);
    }
    // the product of a after each run: reverse scan of the runs' products,
    // look-back over the later tiles
    auto mul = [](const S& x, const S& y) { return S{x.c * y.c}; };
    const S ident{T(1)};
    const S agg[1] = {S{cprod}};
    S wex[1];
    const S total = block_scan_part1<S, true, 1, Cf::NW>(agg, wex, s_tot, ident, mul);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<S> st{R.lbR_agg, R.lbR_incl};
        const S pre = lookback(t_log, st, total, ident, mul, R.hdr);
        block_fold_prefix<S, 1, Cf::NW>(s_tot, pre, mul);
    }
    // l re-formed from the run's carry: t_j = ybar_A A_{j-1} + ybar_B B_{j-1}
    T tj[V];
    {
        T A = PA, B = PB;
#pragma unroll
        for (int p = 0; p < kRunChunks; ++p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> x = run_ld<T>(sA, off), y = run_ld<T>(sB, off);
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                tj[EPC * p + j] = run_fma(A, yA, B * yB);
                B = run_fma(x.v[j], B, y.v[j]);
                A *= x.v[j];
            }
        }
    }
    __syncthreads();
    T rA = block_scan_excl_folded<S, true, 1, Cf::NW>(0, wex, s_tot, mul).c;  // product of a after the run
    // right to left: the outputs, then fold a_j into the product
#pragma unroll
    for (int p = kRunChunks - 1; p >= 0; --p) {
        const int off = run_chunk_off(t, p);
        const RunVec<T> x = run_ld<T>(sA, off);
        RunVec<T> oa, ob;
#pragma unroll
        for (int j = EPC - 1; j >= 0; --j) {
            oa.v[j] = rA * tj[EPC * p + j];
            ob.v[j] = rA * yB;
            rA *= x.v[j];
        }
        run_st<T>(sA, off, oa);
        run_st<T>(sB, off, ob);
    }
    if (whole && !R.accumulate) {
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_3d(&tmOA, (int)(tile * Cf::NT), sA);
            tma_store_3d(&tmOB, (int)(tile * Cf::NT), sB);
            bulk_commit_and_wait_read();
        }
        __syncthreads();
    } else {
        const int64_t e0 = tile * Cf::TILE + (int64_t)t * V;
#pragma unroll 2
        for (int p = 0; p < kRunChunks; ++p) {
            const int off = run_chunk_off(t, p);
            const RunVec<T> oa = run_ld<T>(sA, off), ob = run_ld<T>(sB, off);
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const int64_t e = e0 + EPC * p + j;
                if (e < R.n) {
                    R.abar[e] = R.accumulate ? R.abar[e] + oa.v[j] : oa.v[j];
                    R.bbar[e] = R.accumulate ? R.bbar[e] + ob.v[j] : ob.v[j];
                }
            }
        }
    }
}

}  // namespace adpar
