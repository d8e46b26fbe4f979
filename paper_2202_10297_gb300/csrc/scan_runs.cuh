// The linear-recurrence scan VJP in FP64 with per-thread runs (Sec. 5.2's
// rule for (a1,b1) (.) (a2,b2) = (a2 a1, a2 b1 + b2)), for GB300, whose FP64
// rate (2 lanes per SM per clock) rather than HBM bounds this operator.
//
// Every thread owns a run of kRunV consecutive elements, so the per-element
// work is plain sequential recurrences and the block-level scans (a few FP64
// operations per combine) run once per run instead of once per element:
//
//  pass C (forward): fold each run into its primal aggregate (prod of a, B
//     over the run: 2 FP64 operations per element), scan the runs of a tile,
//     and store per run the exclusive carry from the tile's start and the
//     run's product of a, and per tile its aggregate; one block then scans
//     the tile aggregates into the state before each tile (no look-back:
//     a pass that writes little per element has nothing to hide one behind).
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
//  That is 10 FP64 operations per element plus a share of the run scans,
//  and 16 + 32 + 16 bytes of HBM traffic per element plus 48 bytes per run.
//
// A tile is kRunNT runs; each input array's tile (kRunNT runs of kRunV
// doubles) comes into shared memory by one 3-D TMA copy with the 128-byte swizzle
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

constexpr int kRunV = 16;                   // elements per run (a multiple of 16)
constexpr int kRunRows = kRunV / 16;        // 128-byte rows per run
constexpr int kRunNT = 128;                 // runs (threads) per tile
constexpr int kRunNW = kRunNT / 32;         // warps per tile
constexpr int kRunTile = kRunV * kRunNT;    // elements per tile
constexpr int kRunArrBytes = kRunTile * 8;  // one array's tile

struct RunP {  // primal state (A, B)
    double A, B;
};
struct RunL {  // reverse transfer U -> d + c U, for both components
    double c, dA, dB;
};
// the primal operator on RunP, in the shape the carry scan takes
struct RunPOp {
    using P = RunP;
    __device__ static P pid() { return P{1.0, 0.0}; }
    __device__ static P pcomb(const P& l, const P& r) { return P{l.A * r.A, fma(r.A, l.B, r.B)}; }
};

struct RunArgs {
    int64_t n;
    int64_t tiles;
    const double* a;
    const double* b;
    const double* ya;
    const double* yb;
    double* abar;
    double* bbar;
    int accumulate;
    WsHeader* hdr;
    unsigned long long* lbP_agg;
    unsigned long long* lbP_incl;
    unsigned long long* lbR_agg;
    unsigned long long* lbR_incl;
    double* carA;  // [tiles * kRunNT] A before the run, from the tile's start
    double* carB;  // [tiles * kRunNT] B before the run, from the tile's start
    double* prod;  // [tiles * kRunNT] product of a over the run
    RunP* tagg;    // [tiles] the tile's primal aggregate
    RunP* tcar;    // [tiles] the primal state before the tile
};

// byte offset of the 16-byte pair p (elements 2p, 2p+1) of run t in a
// swizzled array tile
__device__ __forceinline__ int run_pair_off(int t, int p) {
    const int r = kRunRows * t + (p >> 3);
    return r * 128 + (((p & 7) ^ (r & 7)) << 4);
}

__device__ __forceinline__ double2 lds2(const unsigned char* base, int off) {
    return *reinterpret_cast<const double2*>(base + off);
}
__device__ __forceinline__ void sts2(unsigned char* base, int off, double x, double y) {
    *reinterpret_cast<double2*>(base + off) = make_double2(x, y);
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
template <int NA>
__device__ __forceinline__ void run_tile_load(unsigned char* const (&dst)[NA], const CUtensorMap* const (&tm)[NA],
                                              const double* const (&src)[NA], const double (&pad)[NA], bool whole,
                                              int64_t tile, int64_t n, uint64_t* bar, WsHeader* hdr) {
    if (whole) {
        if (threadIdx.x == 0) {
            tc::mbar_init(bar, 1);
            tc::fence_mbar_init();
            tc::mbar_arrive_expect_tx(bar, (uint32_t)(NA * kRunArrBytes));
#pragma unroll
            for (int q = 0; q < NA; ++q) tma_load_3d(dst[q], tm[q], (int)(tile * kRunNT), bar);
        }
        __syncthreads();
        bool ok = false;
        for (uint32_t w = 0; w < (1u << 20) && !ok; ++w) ok = tc::mbar_try_wait(bar, 0u);
        if (!ok) record_status(hdr, ADPAR_ERR_TIMEOUT);
    } else {
        const int64_t e0 = tile * kRunTile;
        for (int i = threadIdx.x; i < kRunTile / 2; i += kRunNT) {
            const int t = i / (kRunV / 2), p = i % (kRunV / 2);
            const int64_t e = e0 + (int64_t)t * kRunV + 2 * p;
            const int off = run_pair_off(t, p);
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                const double x = e < n ? src[q][e] : pad[q];
                const double y = e + 1 < n ? src[q][e + 1] : pad[q];
                sts2(dst[q], off, x, y);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- pass C
__global__ void __launch_bounds__(kRunNT) linrec_runs_carry_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB,
                                                                   RunArgs R) {
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    unsigned char* sA = s_dyn;
    unsigned char* sB = s_dyn + kRunArrBytes;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ RunP s_tot[kRunNW];
    const int64_t tile = blockIdx.x;
    const bool whole = (tile + 1) * kRunTile <= R.n;
    {
        unsigned char* const dst[2] = {sA, sB};
        const CUtensorMap* const tm[2] = {&tmA, &tmB};
        const double* const src[2] = {R.a, R.b};
        const double pad[2] = {1.0, 0.0};  // (1, 0) is the neutral element
        run_tile_load<2>(dst, tm, src, pad, whole, tile, R.n, &s_bar, R.hdr);
    }
    const int t = threadIdx.x;
    double A = 1.0, B = 0.0;
#pragma unroll
    for (int p = 0; p < kRunV / 2; ++p) {
        const double2 x = lds2(sA, run_pair_off(t, p));
        const double2 y = lds2(sB, run_pair_off(t, p));
        B = fma(x.x, B, y.x);
        A *= x.x;
        B = fma(x.y, B, y.y);
        A *= x.y;
    }
    const RunP agg[1] = {RunP{A, B}};
    auto comb = [](const RunP& l, const RunP& r) { return RunP{l.A * r.A, fma(r.A, l.B, r.B)}; };
    RunP wex[1];
    const RunP ident{1.0, 0.0};
    const RunP total = block_scan_part1<RunP, false, 1, kRunNW>(agg, wex, s_tot, ident, comb);
    if (threadIdx.x == 0) R.tagg[tile] = total;
    __syncthreads();
    const RunP ex = block_scan_excl<RunP, false, 1, kRunNW>(0, wex, s_tot, ident, comb);
    const int64_t run = tile * kRunNT + t;
    R.carA[run] = ex.A;
    R.carB[run] = ex.B;
    R.prod[run] = A;
}

// ---------------------------------------------------------------- pass R
__global__ void __launch_bounds__(kRunNT) linrec_runs_vjp_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmYA, const __grid_constant__ CUtensorMap tmYB,
    const __grid_constant__ CUtensorMap tmOA, const __grid_constant__ CUtensorMap tmOB, RunArgs R) {
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    unsigned char* sA = s_dyn;
    unsigned char* sB = s_dyn + kRunArrBytes;      // b, then B_{j-1}
    unsigned char* sYA = s_dyn + 2 * kRunArrBytes;  // ybar_A, then abar
    unsigned char* sYB = s_dyn + 3 * kRunArrBytes;  // ybar_B, then bbar
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tile;
    __shared__ RunL s_tot[kRunNW];
    __shared__ RunL s_pre;
    if (threadIdx.x == 0) s_tile = atomicAdd(&R.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;
    const int64_t tile = R.tiles - 1 - t_log;  // tiles are taken right to left
    const bool whole = (tile + 1) * kRunTile <= R.n;
    const int t = threadIdx.x;
    const int64_t run = tile * kRunNT + t;
    // the run's carry (the state before the tile, then the run's local
    // carry within it) and product (pass C) load while the tile arrives
    const RunP tc0 = R.tcar[tile];
    const double lA = R.carA[run], lB = R.carB[run], cprod = R.prod[run];
    const double PA = tc0.A * lA, PB = fma(lA, tc0.B, lB);
    {
        unsigned char* const dst[4] = {sA, sB, sYA, sYB};
        const CUtensorMap* const tm[4] = {&tmA, &tmB, &tmYA, &tmYB};
        const double* const src[4] = {R.a, R.b, R.ya, R.yb};
        const double pad[4] = {1.0, 0.0, 0.0, 0.0};
        run_tile_load<4>(dst, tm, src, pad, whole, tile, R.n, &s_bar, R.hdr);
    }

    // 1. the primal from the carry: A_{j-1} in registers, B_{j-1} over b
    double Aprev[kRunV];
    {
        double A = PA, B = PB;
#pragma unroll
        for (int p = 0; p < kRunV / 2; ++p) {
            const int off = run_pair_off(t, p);
            const double2 x = lds2(sA, off);
            const double2 y = lds2(sB, off);
            const double B0 = B;
            Aprev[2 * p] = A;
            B = fma(x.x, B, y.x);
            A *= x.x;
            Aprev[2 * p + 1] = A;
            sts2(sB, off, B0, B);
            B = fma(x.y, B, y.y);
            A *= x.y;
        }
    }
    // 2. the run's reverse transfer: R_j = ybar_j + a_{j+1} R_{j+1}
    double RA, RB, a_next;
    {
        const double2 y1 = lds2(sYA, run_pair_off(t, kRunV / 2 - 1));
        const double2 y2 = lds2(sYB, run_pair_off(t, kRunV / 2 - 1));
        const double2 x = lds2(sA, run_pair_off(t, kRunV / 2 - 1));
        RA = fma(x.y, y1.y, y1.x);
        RB = fma(x.y, y2.y, y2.x);
        a_next = x.x;
#pragma unroll
        for (int p = kRunV / 2 - 2; p >= 0; --p) {
            const int off = run_pair_off(t, p);
            const double2 ya = lds2(sYA, off);
            const double2 yb = lds2(sYB, off);
            const double2 aa = lds2(sA, off);
            RA = fma(a_next, RA, ya.y);
            RB = fma(a_next, RB, yb.y);
            RA = fma(aa.y, RA, ya.x);
            RB = fma(aa.y, RB, yb.x);
            a_next = aa.x;
        }
    }
    // a_next is now a_s, the run's first a
    const RunL agg[1] = {RunL{cprod, a_next * RA, a_next * RB}};
    // 3. scan of the transfers, right to left: comb(x, y) with x to the
    //    right of y is "x, then y"
    auto comb = [](const RunL& x, const RunL& y) {
        return RunL{y.c * x.c, fma(y.c, x.dA, y.dA), fma(y.c, x.dB, y.dB)};
    };
    const RunL ident{1.0, 0.0, 0.0};
    RunL wex[1];
    const RunL total = block_scan_part1<RunL, true, 1, kRunNW>(agg, wex, s_tot, ident, comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<RunL> st{R.lbR_agg, R.lbR_incl};
        const RunL pre = lookback(t_log, st, total, ident, comb, R.hdr);
        if ((threadIdx.x & 31) == 0) s_pre = pre;
    }
    __syncthreads();
    const RunL ex = block_scan_excl<RunL, true, 1, kRunNW>(0, wex, s_tot, s_pre, comb);

    // 4. rs_bar right to left and the outputs, written over the cotangents
    {
        double rA = ex.dA, rB = ex.dB;  // U entering the run's last element
        double a_up = 1.0;              // a_{j+1} (the factor carried into U)
#pragma unroll
        for (int p = kRunV / 2 - 1; p >= 0; --p) {
            const int off = run_pair_off(t, p);
            const double2 ya = lds2(sYA, off);
            const double2 yb = lds2(sYB, off);
            const double2 aa = lds2(sA, off);
            const double2 bp = lds2(sB, off);  // B_{j-1}
            // element 2p+1
            const double rA1 = fma(a_up, rA, ya.y);
            const double rB1 = fma(a_up, rB, yb.y);
            const double o1 = fma(Aprev[2 * p + 1], rA1, bp.y * rB1);
            // element 2p
            const double rA0 = fma(aa.y, rA1, ya.x);
            const double rB0 = fma(aa.y, rB1, yb.x);
            const double o0 = fma(Aprev[2 * p], rA0, bp.x * rB0);
            sts2(sYA, off, o0, o1);
            sts2(sYB, off, rB0, rB1);
            rA = rA0;
            rB = rB0;
            a_up = aa.x;
        }
    }
    // the first element's factor a_{j+1} for j = e is applied through U:
    // rs_bar_e = ybar_e + U_{e+1} with U_{e+1} = ex.d (a_up starts at 1)

    if (whole && !R.accumulate) {
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_3d(&tmOA, (int)(tile * kRunNT), sYA);
            tma_store_3d(&tmOB, (int)(tile * kRunNT), sYB);
            bulk_commit_and_wait_read();
        }
        __syncthreads();
    } else {
        const int64_t e0 = tile * kRunTile + (int64_t)t * kRunV;
#pragma unroll 4
        for (int p = 0; p < kRunV / 2; ++p) {
            const int off = run_pair_off(t, p);
            const double2 oa = lds2(sYA, off);
            const double2 ob = lds2(sYB, off);
            const int64_t e = e0 + 2 * p;
            if (e < R.n) {
                R.abar[e] = R.accumulate ? R.abar[e] + oa.x : oa.x;
                R.bbar[e] = R.accumulate ? R.bbar[e] + ob.x : ob.x;
            }
            if (e + 1 < R.n) {
                R.abar[e + 1] = R.accumulate ? R.abar[e + 1] + oa.y : oa.y;
                R.bbar[e + 1] = R.accumulate ? R.bbar[e + 1] + ob.y : ob.y;
            }
        }
    }
}

}  // namespace adpar
