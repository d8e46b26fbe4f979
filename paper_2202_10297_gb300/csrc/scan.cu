// VJP of inclusive scan (Sec. 5.2) for ADD, MUL, MIN, MAX and the
// linear-recurrence pair operator, FP32 and FP64.
//
// The return sweep of Sec. 5.2 is the backward linear recurrence
//   rs_bar_i = ys_bar_i + J_left(i+1)^T rs_bar_{i+1}
// followed by the map  as_bar_i = J_right(i)^T rs_bar_i.  We solve it with
// the recurrence re-associated onto the element that carries the factor:
//   u_i = J_left(i)^T (ys_bar_i + u_{i+1}),  u_n = 0,
//   rs_bar_i = ys_bar_i + u_{i+1},
// i.e. a reverse EXCLUSIVE scan of the affine maps x -> c_i ys_bar_i + c_i x
// with lin_o.  It needs no shifted load of as_{i+1}, and c_i = J_left(i)
// depends only on (rs_{i-1}, as_i), both known at position i.
//
// Two kernels, both single-pass with decoupled look-back:
//  pass P (forward; only when the adjoint needs the primal): per tile, the
//         exclusive primal prefix rs_{tile_start-1} ("carry"), reading as.
//  pass R (reverse, tiles taken right to left): recompute the primal inside
//         the tile from its carry, build the lin_o elements, reverse-scan
//         them with look-back, and write as_bar (and optionally ys).
#include <algorithm>
#include <cstring>

#include "scan_runs.cuh"
#include "scan_tiles.cuh"
#include "tc.cuh"

namespace adpar {
namespace {

// Tile shape: K chunks of kScanBlock * E elements; in each chunk a thread
// owns E consecutive elements (kept in registers).  Larger E amortises the
// warp-shuffle scans over more elements, which matters where arithmetic,
// not memory, bounds the kernel (FP64 on GB300).
template <class Op, class T>
struct ScanCfg {
    static constexpr bool kF64 = sizeof(T) == 8;
    static constexpr int E = kF64 ? (Op::kWidth == 2 ? 8 : 4) : 4;
    static constexpr int K = kF64 ? (Op::kWidth == 2 ? 1 : 4) : (Op::kWidth == 2 ? 4 : 8);
    static constexpr int TILE = K * kScanBlock * E;
};

// Zeroes the header and the look-back slots (one contiguous region).
__global__ void scan_init_kernel(WsHeader* hdr, unsigned long long* slots, int64_t nwords) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i < 64) reinterpret_cast<uint32_t*>(hdr)[i] = 0u;
    for (int64_t t = i; t < nwords; t += stride) slots[t] = 0ull;
}

template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_primal_kernel(ScanArgs A) {
    using Cfg = ScanCfg<Op, T>;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    scan_primal_tile<Op, T, Cfg::K, Cfg::E>(A, (int64_t)s_tile);
}

// Pass P as reduce-then-scan, for the return sweeps that read only each
// tile's exclusive carry: every block reduces its tile to the tile's primal
// aggregate (a streaming read of the inputs in which no block waits on
// another), then one block scans the aggregates, in order, into the carries.
// The single-pass form spent most of its time in look-backs: a pass that
// writes nothing per element has little work to hide them behind.
template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_tile_agg_kernel(ScanArgs A, typename Op::P* agg) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    constexpr int K = Cfg::K, V = Cfg::E, NW = kScanBlock / 32, TILE = Cfg::TILE;
    __shared__ P s_tot[K * NW];
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);
    P part[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        T av[V], bv[V];
        load_chunk(a, e, A.n, Op::pad_a(), av);
        if constexpr (Op::kWidth == 2) load_chunk(b, e, A.n, T(0), bv);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[j] = T(0);
        }
        P acc = Op::pelem(av[0], bv[0]);
#pragma unroll
        for (int j = 1; j < V; ++j) acc = Op::pcomb(acc, Op::pelem(av[j], bv[j]));
        part[k] = acc;
    }
    auto comb = [](const P& l, const P& r) { return Op::pcomb(l, r); };
    P wex[K];
    const P total = block_scan_part1<P, false, K, NW>(part, wex, s_tot, Op::pid(), comb);
    if (threadIdx.x == 0) agg[tile] = total;
}

// carry[i] = agg[0] (.) ... (.) agg[i-1], in order, over segments of
// kCarrySeg tiles: carry_local_kernel scans each segment (one block per
// segment) and writes its total, carry_apply_kernel puts the fold of the
// earlier segments' totals in front.  (One block over every tile left the
// FP64 combines to one SM: 116 us for 32768 FP64 tiles.)  segtot holds one
// state per segment.
constexpr int kCarryBlock = 1024;
constexpr int kCarryPer = 4;
constexpr int kCarrySeg = kCarryBlock * kCarryPer;

template <class Op>
__global__ void __launch_bounds__(kCarryBlock) carry_local_kernel(const typename Op::P* agg, typename Op::P* carry,
                                                                  typename Op::P* segtot, int64_t tiles) {
    using P = typename Op::P;
    __shared__ P s_w[kCarryBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCarrySeg + (int64_t)threadIdx.x * kCarryPer;
    P v[kCarryPer];
    P run = Op::pid();
#pragma unroll
    for (int j = 0; j < kCarryPer; ++j) {
        v[j] = base + j < tiles ? agg[base + j] : Op::pid();
        run = Op::pcomb(run, v[j]);
    }
    P inc = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const P o = shfl_up_s(inc, off);
        if (lane >= off) inc = Op::pcomb(o, inc);
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        P w = s_w[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const P o = shfl_up_s(w, off);
            if (lane >= off) w = Op::pcomb(o, w);
        }
        s_w[lane] = w;
    }
    __syncthreads();
    P ex = shfl_up_s(inc, 1);
    if (lane == 0) ex = Op::pid();
    if (warp > 0) ex = Op::pcomb(s_w[warp - 1], ex);
#pragma unroll
    for (int j = 0; j < kCarryPer; ++j) {
        if (base + j < tiles) carry[base + j] = ex;
        ex = Op::pcomb(ex, v[j]);
    }
    if (threadIdx.x == 0) segtot[blockIdx.x] = s_w[kCarryBlock / 32 - 1];
}

template <class Op>
__global__ void __launch_bounds__(256) carry_apply_kernel(typename Op::P* carry, const typename Op::P* segtot,
                                                          int64_t tiles) {
    using P = typename Op::P;
    if (blockIdx.x == 0) return;
    __shared__ P s_pre;
    if (threadIdx.x < 32) {
        // fold of segtot[0 .. blockIdx.x): contiguous pieces per lane, then
        // a warp scan of the pieces in lane order
        const int lane = threadIdx.x;
        const int cnt = (int)blockIdx.x, per = (cnt + 31) / 32;
        P r = Op::pid();
        for (int i = lane * per; i < cnt && i < (lane + 1) * per; ++i) r = Op::pcomb(r, segtot[i]);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const P o = shfl_up_s(r, off);
            if (lane >= off) r = Op::pcomb(o, r);
        }
        if (lane == 31) s_pre = r;
    }
    __syncthreads();
    const P pre = s_pre;
    const int64_t lo = (int64_t)blockIdx.x * kCarrySeg;
    const int64_t hi = lo + kCarrySeg < tiles ? lo + kCarrySeg : tiles;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) carry[i] = Op::pcomb(pre, carry[i]);
}

// the tile carries from the tile aggregates; segtot: room for one state per
// kCarrySeg tiles
template <class Op>
void launch_carry_scan(const typename Op::P* agg, typename Op::P* carry, typename Op::P* segtot, int64_t tiles,
                       cudaStream_t stream) {
    const unsigned nseg = (unsigned)((tiles + kCarrySeg - 1) / kCarrySeg);
    carry_local_kernel<Op><<<nseg, kCarryBlock, 0, stream>>>(agg, carry, segtot, tiles);
    if (nseg > 1) carry_apply_kernel<Op><<<nseg, 256, 0, stream>>>(carry, segtot, tiles);
}

// MIN/MAX scans: the return sweep fused into the forward pass.  For these
// operators J_left(i) = c_i is 0 exactly when a_{i+1} is a record (strictly
// beyond the running extremum; the tie rule keeps the earlier element), so
// the lin_o recurrence rs_bar_i = ybar_i + c_i rs_bar_{i+1} restarts at
// every record, and as_bar_i = J_right(i) rs_bar_i is nonzero only at
// records (and at element 0, which takes rs_bar_0): a record's adjoint is
// the sum of ybar from it to the element before the next record.  No tile
// waits on another: the tile extrema (scan_minmax_tile_kernel) and their
// exclusive scan (one block) give every tile its carry, hence its records;
// a reverse segmented sum inside the tile gives each record's part of that
// sum, and the adjoint is written once.  The part of the last record's sum
// that lies in later tiles is added by scan_minmax_runs_kernel and
// scan_minmax_fixup_kernel from per-tile data: the sum of ybar before the
// tile's first record (lead) and the tile's last record (last).
// Per-tile data of the min/max rule, in the scan workspace.  Tiles form
// groups of kMmGroup; each small scan over the tiles runs as one block per
// group plus a combine of the (few) group aggregates by its consumer.
constexpr int kMmGroup = 1024;

template <class P>
struct MinMaxWs {
    P* tmax;             // [tiles] the tile's extremum
    P* carry;            // [tiles] exclusive within the group; record tiles: the whole carry
    P* gagg;             // [groups] group extremum
    uint32_t* rec_list;  // [tiles] the tiles holding a record
    uint32_t* n_rec;     // their count (zeroed with the workspace header)
    double* lead;        // [tiles] ybar of the tile before its first record
    int64_t* last;       // [tiles] the tile's last record, -1 if none
    double* xloc;        // [tiles] run sum from the tile to its group's end or the first record tile
    uint32_t* floc;      // [tiles] a record tile lies in [tile, group end]
    double* fx;          // [groups] the same for the group's first tile
    uint32_t* ff;
    int64_t tiles;
    int groups;
};

// Extremum of the groups before g (warp 0 of the block; any order: the
// extremum is exact)
template <class Op>
__device__ __forceinline__ typename Op::P mm_group_prefix(const typename Op::P* gagg, int g) {
    using P = typename Op::P;
    const int lane = threadIdx.x & 31;
    P acc = Op::pid();
    for (int h = lane; h < g; h += 32) acc = Op::pcomb(acc, gagg[h]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = Op::pcomb(acc, shfl_down_s(acc, off));
    return acc;  // lane 0
}

template <class T>
struct RunSum {
    T x;         // ybar from the element to the end of its run
    uint32_t f;  // the run ends inside (a record follows)
};

template <class Op, class T, bool WYS>
__global__ void __launch_bounds__(kScanBlock) scan_minmax_fused_kernel(ScanArgs A, const uint32_t* rec_list,
                                                                       const uint32_t* n_rec, double* lead,
                                                                       int64_t* last) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    using R = RunSum<T>;
    constexpr int K = Cfg::K, E = Cfg::E, NW = kScanBlock / 32;
    __shared__ P s_tot[K * NW];
    __shared__ R s_totR[K * NW];
    __shared__ P s_pre;
    __shared__ uint32_t s_rec[K][kScanBlock];  // record bits of each thread's E elements
    __shared__ unsigned long long s_last1;      // 1 + the tile's last record (0: none)
    const T* a = static_cast<const T*>(A.a);
    const T* yb = static_cast<const T*>(A.ya);
    // persistent over the tiles holding a record (listed by the carry scan)
    const uint32_t nrec = *n_rec;
    for (uint32_t q = blockIdx.x; q < nrec; q += gridDim.x) {
        const int64_t t = rec_list[q];
        if (threadIdx.x == 0) {
            s_last1 = 0ull;
            s_pre = static_cast<const P*>(A.carry)[t];  // the extremum before the tile
        }
        __syncthreads();
        const int64_t base = t * Cfg::TILE;
        T av[K][E], yv[K][E];
        P agg[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t e = base + (int64_t)k * kScanBlock * E + threadIdx.x * E;
            load_chunk(a, e, A.n, Op::pad_a(), av[k]);
            load_chunk(yb, e, A.n, T(0), yv[k]);
            P acc = Op::pelem(av[k][0], T(0));
#pragma unroll
            for (int j = 1; j < E; ++j) acc = Op::pcomb(acc, Op::pelem(av[k][j], T(0)));
            agg[k] = acc;
        }
        auto fc = [](const P& l, const P& r) { return Op::pcomb(l, r); };
        P wex[K];
        (void)block_scan_part1<P, false, K, NW>(agg, wex, s_tot, Op::pid(), fc);
        __syncthreads();
        // records: J_right(i) = 1 (a_i strictly beyond everything before it), and element 0
        uint32_t rec[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t e = base + (int64_t)k * kScanBlock * E + threadIdx.x * E;
            P prev = block_scan_excl<P, false, K, NW>(k, wex, s_tot, s_pre, fc);
            uint32_t bits = 0;
            T ys[E];
#pragma unroll
            for (int j = 0; j < E; ++j) {
                T on = T(0), dummy = T(0);
                Op::vjp_right(prev, av[k][j], T(0), T(1), T(0), on, dummy);
                if (e + j < A.n && (e + j == 0 || on != T(0))) bits |= 1u << j;
                prev = Op::pcomb(prev, Op::pelem(av[k][j], T(0)));
                ys[j] = Op::out_a(prev);
            }
            rec[k] = bits;
            s_rec[k][threadIdx.x] = bits;
            if constexpr (WYS) {
                if (e < A.n) store_chunk(static_cast<T*>(A.ys_a), e, A.n, ys);
            }
        }
        __syncthreads();
        // in-tile runs: element i's run ends where element i+1 is a record
        R aggR[K];
        uint32_t nextrec[K];  // record bit of the element after each thread's last one
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int tn = threadIdx.x + 1;
            nextrec[k] = tn < kScanBlock ? (s_rec[k][tn] & 1u) : (k + 1 < K ? (s_rec[k + 1 < K ? k + 1 : k][0] & 1u) : 0u);
            R acc{T(0), 0u};
            uint32_t nxt = nextrec[k];
#pragma unroll
            for (int j = E - 1; j >= 0; --j) {
                const R el{yv[k][j], nxt};
                acc = el.f ? el : R{el.x + acc.x, acc.f};
                nxt = (rec[k] >> j) & 1u;
            }
            aggR[k] = acc;
        }
        auto rc = [](const R& later, const R& earlier) { return earlier.f ? earlier : R{earlier.x + later.x, later.f}; };
        R wexR[K];
        (void)block_scan_part1<R, true, K, NW>(aggR, wexR, s_totR, R{T(0), 0u}, rc);
        __syncthreads();
        T* abar = static_cast<T*>(A.abar);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t e = base + (int64_t)k * kScanBlock * E + threadIdx.x * E;
            if (e >= A.n) continue;
            R after = block_scan_excl<R, true, K, NW>(k, wexR, s_totR, R{T(0), 0u}, rc);
            T out[E];
            uint32_t nxt = nextrec[k];
#pragma unroll
            for (int j = E - 1; j >= 0; --j) {
                const R el{yv[k][j], nxt};
                after = el.f ? el : R{el.x + after.x, after.f};  // after.x = the run sum from element j
                nxt = (rec[k] >> j) & 1u;
                out[j] = nxt ? after.x : T(0);
            }
            if (e == base && k == 0) lead[t] = rec[0] & 1u ? 0.0 : (double)after.x;  // after the loop: element base
            if (rec[k]) atomicMax(&s_last1, (unsigned long long)(e + 31 - __clz(rec[k]) + 1));
            if (A.accumulate) {
                T old[E];
                load_chunk_keep(static_cast<const T*>(A.abar), e, A.n, T(0), old);
#pragma unroll
                for (int j = 0; j < E; ++j) out[j] += old[j];
            }
            store_chunk(abar, e, A.n, out);
        }
        __syncthreads();
        if (threadIdx.x == 0) last[t] = (int64_t)s_last1 - 1;
        __syncthreads();  // the shared state is reused by the next tile
    }
}

// Tiles without a record (nothing beyond the carry): the adjoint is 0, the
// primal is the carry, and all of the tile's ybar belongs to the run of the
// last record before it, so only ybar is read.  A small kernel of its own
// (few registers, many blocks per SM); scan_minmax_fused_kernel skips these
// tiles.
template <class Op, class T, bool WYS>
__global__ void __launch_bounds__(kScanBlock) scan_minmax_zero_kernel(ScanArgs A, MinMaxWs<typename Op::P> M) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    constexpr int K = Cfg::K, E = Cfg::E, NW = kScanBlock / 32;
    __shared__ P s_pre;
    __shared__ uint32_t s_has;
    __shared__ double s_sum[NW];
    const int64_t t = blockIdx.x;
    double* lead = M.lead;
    int64_t* last = M.last;
    if (threadIdx.x < 32) {
        const P gp = mm_group_prefix<Op>(M.gagg, (int)(t / kMmGroup));
        if (threadIdx.x == 0) {
            const P pre = Op::pcomb(gp, M.carry[t]);  // the extremum before the tile
            s_pre = pre;
            T on = T(0), dummy = T(0);
            Op::vjp_right(pre, Op::out_a(M.tmax[t]), T(0), T(1), T(0), on, dummy);
            const bool has = t == 0 || on != T(0);
            s_has = has ? 1u : 0u;
            if (has) {  // scan_minmax_fused_kernel takes the tile, with its whole carry
                M.carry[t] = pre;
                M.rec_list[atomicAdd(M.n_rec, 1u)] = (uint32_t)t;
            }
        }
    }
    __syncthreads();
    if (s_has) return;
    const int64_t base = t * Cfg::TILE;
    const T* yb = static_cast<const T*>(A.ya);
    double sum = 0.0;
    T zero[E], ysv[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        zero[j] = T(0);
        ysv[j] = Op::out_a(s_pre);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * E + threadIdx.x * E;
        T yv[E];
        load_chunk(yb, e, A.n, T(0), yv);
        T ps = T(0);
#pragma unroll
        for (int j = 0; j < E; ++j) ps += yv[j];
        sum += (double)ps;
        if (e < A.n) {
            if (!A.accumulate) store_chunk(static_cast<T*>(A.abar), e, A.n, zero);
            if constexpr (WYS) store_chunk(static_cast<T*>(A.ys_a), e, A.n, ysv);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < NW; ++w) tot += s_sum[w];
        lead[t] = tot;
        last[t] = -1;
    }
}

// Each tile's extremum (no dependence between tiles).
template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_minmax_tile_kernel(ScanArgs A, typename Op::P* tmax) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    constexpr int K = Cfg::K, E = Cfg::E;
    __shared__ P s_w[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * Cfg::TILE;
    const T* a = static_cast<const T*>(A.a);
    P acc = Op::pid();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T av[E];
        load_chunk(a, base + (int64_t)k * kScanBlock * E + threadIdx.x * E, A.n, Op::pad_a(), av);
#pragma unroll
        for (int j = 0; j < E; ++j) acc = Op::pcomb(acc, Op::pelem(av[j], T(0)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = Op::pcomb(acc, shfl_down_s(acc, off));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        P r = s_w[0];
        for (int w = 1; w < kScanBlock / 32; ++w) r = Op::pcomb(r, s_w[w]);
        tmax[blockIdx.x] = r;
    }
}

// Exclusive extremum of the tiles within each group (one block per group,
// one tile per thread) and each group's extremum.
template <class Op, class T>
__global__ void __launch_bounds__(kMmGroup) scan_minmax_group_kernel(MinMaxWs<typename Op::P> M) {
    using P = typename Op::P;
    __shared__ P s_w[kMmGroup / 32];
    const int64_t u = (int64_t)blockIdx.x * kMmGroup + threadIdx.x;
    const P v = u < M.tiles ? M.tmax[u] : Op::pid();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    P inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const P o = shfl_up_s(inc, off);
        if (lane >= off) inc = Op::pcomb(o, inc);
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        P wi = s_w[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const P o = shfl_up_s(wi, off);
            if (lane >= off) wi = Op::pcomb(o, wi);
        }
        if (lane == 31) M.gagg[blockIdx.x] = wi;
        P ex = shfl_up_s(wi, 1);
        if (lane == 0) ex = Op::pid();
        __syncwarp();
        s_w[lane] = ex;
    }
    __syncthreads();
    P ex = shfl_up_s(inc, 1);
    if (lane == 0) ex = Op::pid();
    if (u < M.tiles) M.carry[u] = Op::pcomb(s_w[warp], ex);
}

// The run across tiles, R_t = lead_{t+1} + (tile t+1 has a record ? 0 :
// R_{t+1}), is a reverse segmented sum over the tiles.  Pass 1: within
// each group (one block, one tile per thread, FP64), S(u) = lead_u +
// (u has a record ? 0 : S(u+1)) up to the group's end, whether a record
// tile lies in [u, group end], and the same for the group's first tile.
template <class P>
__global__ void __launch_bounds__(kMmGroup) scan_minmax_runs_kernel(MinMaxWs<P> M) {
    __shared__ double s_x[kMmGroup / 32];
    __shared__ uint32_t s_f[kMmGroup / 32];
    const int64_t u = (int64_t)blockIdx.x * kMmGroup + threadIdx.x;
    double x = 0.0;
    uint32_t f = 0u;
    if (u < M.tiles) {
        x = M.lead[u];
        f = M.last[u] >= 0 ? 1u : 0u;
    }
    // inclusive reverse scan: (x, f) over [u, group end], later lanes first
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double ox = __shfl_down_sync(0xffffffffu, x, off);
        const uint32_t of = __shfl_down_sync(0xffffffffu, f, off);
        if (lane + off < 32 && !f) {
            x += ox;
            f = of;
        }
    }
    if (lane == 0) {
        s_x[warp] = x;
        s_f[warp] = f;
    }
    __syncthreads();
    if (warp == 0) {
        double wx = s_x[lane];
        uint32_t wf = s_f[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double ox = __shfl_down_sync(0xffffffffu, wx, off);
            const uint32_t of = __shfl_down_sync(0xffffffffu, wf, off);
            if (lane + off < 32 && !wf) {
                wx += ox;
                wf = of;
            }
        }
        if (lane == 0) {
            M.fx[blockIdx.x] = wx;
            M.ff[blockIdx.x] = wf;
        }
        const double ex = __shfl_down_sync(0xffffffffu, wx, 1);  // the warps after this one
        const uint32_t ef = __shfl_down_sync(0xffffffffu, wf, 1);
        __syncwarp();
        s_x[lane] = lane < 31 ? ex : 0.0;
        s_f[lane] = lane < 31 ? ef : 0u;
    }
    __syncthreads();
    if (!f) {
        x += s_x[warp];
        f = s_f[warp];
    }
    if (u < M.tiles) {
        M.xloc[u] = x;
        M.floc[u] = f;
    }
}

// Pass 2: adds R_t to each tile's last record; R_t comes from tile t+1's
// group-local value and, where its run leaves the group, the groups after.
template <class P, class T>
__global__ void __launch_bounds__(kMmGroup) scan_minmax_fixup_kernel(MinMaxWs<P> M, T* abar) {
    __shared__ double s_after;  // S of the first tile after this group
    const int g = blockIdx.x;
    if (threadIdx.x < 32) {
        // reverse combine of the groups after g: each lane folds a
        // contiguous part, then the lanes combine right to left
        const int lane = threadIdx.x;
        const int cnt = M.groups - 1 - g;
        const int per = (cnt + 31) / 32;
        const int h0 = g + 1 + lane * per, h1 = min(h0 + per, M.groups);
        double x = 0.0;
        uint32_t f = 0u;
        for (int h = h1 - 1; h >= h0; --h) {
            const double hx = M.fx[h];
            const uint32_t hf = M.ff[h];
            x = hf ? hx : hx + x;
            f = hf ? 1u : f;
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double ox = __shfl_down_sync(0xffffffffu, x, off);
            const uint32_t of = __shfl_down_sync(0xffffffffu, f, off);
            if (lane + off < 32 && !f) {
                x += ox;
                f = of;
            }
        }
        if (lane == 0) s_after = x;
    }
    __syncthreads();
    const int64_t t = (int64_t)g * kMmGroup + threadIdx.x;
    if (t >= M.tiles) return;
    const int64_t p = M.last[t];
    if (p < 0) return;
    double r;
    if (t + 1 >= M.tiles) r = 0.0;
    else if ((t + 1) / kMmGroup == g) r = M.floc[t + 1] ? M.xloc[t + 1] : M.xloc[t + 1] + s_after;
    else r = s_after;
    abar[p] += (T)r;
}

// The factored path (FP64 operators with J_left = a_i): the return sweep's
// tiles are kScanBlock runs of kFacV elements; the primal pass takes
// kFacKP of them per tile (its carries keep the return sweep's indexing),
// so it runs a quarter of the look-backs.  A.tiles is each kernel's own
// tile count.
constexpr int kFacKP = 4;
constexpr int64_t kFacTile = (int64_t)kScanBlock * kFacV;

template <class Op>
__global__ void __launch_bounds__(kScanBlock) scan_primal_fac_kernel(ScanArgs A) {
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    scan_primal_fac_tile<Op, kFacKP>(A, (int64_t)s_tile);
}

// 3 resident blocks per SM for the pair operator, 4 for width 1 (the
// register caps where neither spills much)
template <class Op, bool WYS>
__global__ void __launch_bounds__(kScanBlock, Op::kWidth == 2 ? 3 : 4) scan_adjoint_fac_kernel(ScanArgs A) {
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    scan_adjoint_fac_tile<Op, WYS>(A, (int64_t)s_tile);
}

template <class Op, class T, bool WYS>
__global__ void __launch_bounds__(kScanBlock) scan_adjoint_kernel(ScanArgs A) {
    using Cfg = ScanCfg<Op, T>;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    scan_adjoint_tile<Op, T, Cfg::K, Cfg::E, WYS>(A, (int64_t)s_tile);
}


// The forward operator itself (ys = scan (.) as), used as the primal
// baseline of the VJP/primal time ratio.  One single pass with look-back.
template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_forward_kernel(ScanArgs A) {
    using Cfg = ScanCfg<Op, T>;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    scan_forward_tile<Op, T, Cfg::K, Cfg::E>(A, (int64_t)s_tile);
}

// ---------------------------------------------------- + scan on per-thread runs
// The return sweep of the + scan is the reverse suffix sum
// as_bar_i = sum_{j >= i} ys_bar_j.  One block per tile, tiles taken right to
// left by a ticket.  A tile is kAddRB row blocks of kAddNT rows of 128 bytes
// (runs of V elements), every thread owning one row in each row block.  Each
// row block comes into shared memory by one 3-D TMA copy with the 128-byte
// swizzle of the runs layout (a thread reads its own row without bank
// conflicts); each thread sums its rows, one reverse block scan over the rows
// and the look-back give every row the sum of everything to its right, the
// rows' suffix sums are written back in place and the row blocks leave by
// TMA stores.  A block holds its tile in shared memory from its load to its
// stores, so the loads in flight per SM are bounded by the tiles resident
// there; to keep HBM busy beyond that, each block also asks L2 to prefetch
// the tile kAddAhead tickets later, which a block launched a third of a
// wave later (456 tiles are resident) then finds in L2.  FP32 at 2^28: no
// prefetch 0.500 ms; 76, 152, 228, 456, 912 tiles ahead 0.425, 0.417,
// 0.416, 0.485, 0.575 ms (further ahead, the lines are evicted before use).
constexpr int kAddNT = 256;     // threads, and rows per row block
constexpr int kAddRB = 2;       // row blocks per tile
constexpr int kAddAhead = 152;  // tickets between a tile and the one its block prefetches

template <class T>
struct AddRunCfg {
    static constexpr int V = RunCfg<T>::V;
    static constexpr int TILE = kAddRB * kAddNT * V;  // elements per tile (64 KB)
    static constexpr int RBB = kAddNT * 128;          // bytes per row block
    static constexpr int kSmem = kAddRB * RBB;
};

template <class T>
__global__ void __launch_bounds__(kAddNT) scan_add_runs_kernel(const __grid_constant__ CUtensorMap tmY,
                                                              const __grid_constant__ CUtensorMap tmO, ScanArgs A) {
    using C = AddRunCfg<T>;
    constexpr int V = C::V, EPC = RunCfg<T>::EPC, NW = kAddNT / 32, RB = kAddRB, TILE = C::TILE, RBB = C::RBB;
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tile;
    __shared__ T s_tot[RB * NW];
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;
    const int64_t tile = A.tiles - 1 - t_log;  // right to left
    const int64_t row0 = tile * (RB * kAddNT);
    const int64_t e0 = tile * TILE;
    const bool whole = e0 + TILE <= A.n;
    const T* ya = static_cast<const T*>(A.ya);
    T* abar = static_cast<T*>(A.abar);
    const int t = threadIdx.x;
    if (whole) {
        if (t == 0) {
            tc::mbar_init(&s_bar, 1);
            tc::fence_mbar_init();
            tc::mbar_arrive_expect_tx(&s_bar, (uint32_t)C::kSmem);
#pragma unroll
            for (int k = 0; k < RB; ++k) tma_load_3d(s_dyn + k * RBB, &tmY, (int)(row0 + k * kAddNT), &s_bar);
            // a tile to the left of a whole tile is whole
            if (tile >= kAddAhead) tc::prefetch_l2(ya + (tile - kAddAhead) * TILE, (uint32_t)(TILE * sizeof(T)));
        }
        __syncthreads();
        bool ok = false;
        for (uint32_t w = 0; w < (1u << 20) && !ok; ++w) ok = tc::mbar_try_wait(&s_bar, 0u);
        if (!ok) record_status(A.hdr, ADPAR_ERR_TIMEOUT);
    } else {
        // element by element in the same layout, zero past the end (row q of
        // the tile is row q % kAddNT of row block q / kAddNT)
        for (int i = t; i < RB * kAddNT * kRunChunks; i += kAddNT) {
            const int q = i / kRunChunks, p = i % kRunChunks;
            const int64_t e = e0 + (int64_t)q * V + EPC * p;
            RunVec<T> v;
#pragma unroll
            for (int j = 0; j < EPC; ++j) v.v[j] = e + j < A.n ? ya[e + j] : T(0);
            run_st<T>(s_dyn + (q / kAddNT) * RBB, run_chunk_off(q % kAddNT, p), v);
        }
        __syncthreads();
    }

    // the sums of the thread's rows, reverse block scan over the rows, look-back
    auto add = [](const T& x, const T& y) { return x + y; };
    T agg[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        const unsigned char* base = s_dyn + k * RBB;
        T part[kRunChunks];
#pragma unroll
        for (int p = 0; p < kRunChunks; ++p) {
            const RunVec<T> x = run_ld<T>(base, run_chunk_off(t, p));
            T c = x.v[0];
#pragma unroll
            for (int j = 1; j < EPC; ++j) c += x.v[j];
            part[p] = c;
        }
#pragma unroll
        for (int h = kRunChunks / 2; h > 0; h /= 2)
#pragma unroll
            for (int p = 0; p < h; ++p) part[p] += part[p + h];
        agg[k] = part[0];
    }
    T wex[RB];
    const T total = block_scan_part1<T, true, RB, NW>(agg, wex, s_tot, T(0), add);
    if ((t >> 5) == 0) {
        LookbackState<T> st{A.lbR_agg, A.lbR_incl};
        const T pre = lookback(t_log, st, total, T(0), add, A.hdr);
        block_fold_prefix<T, RB, NW>(s_tot, pre, add);
    }
    __syncthreads();

    // each row's suffix sums plus everything to its right, in place
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        unsigned char* base = s_dyn + k * RBB;
        T run = block_scan_excl_folded<T, true, RB, NW>(k, wex, s_tot, add);
#pragma unroll
        for (int p = kRunChunks - 1; p >= 0; --p) {
            const int off = run_chunk_off(t, p);
            RunVec<T> x = run_ld<T>(base, off);
#pragma unroll
            for (int j = EPC - 1; j >= 0; --j) {
                run += x.v[j];
                x.v[j] = run;
            }
            run_st<T>(base, off, x);
        }
    }

    if (whole && !A.accumulate) {
        tc::fence_proxy_async();
        __syncthreads();
        if (t == 0) {
#pragma unroll
            for (int k = 0; k < RB; ++k) tma_store_3d(&tmO, (int)(row0 + k * kAddNT), s_dyn + k * RBB);
            bulk_commit_and_wait_read();
        }
    } else {
        __syncthreads();
        // coalesced: consecutive threads take consecutive 16-byte chunks
        for (int i = t; i < RB * kAddNT * kRunChunks; i += kAddNT) {
            const int q = i / kRunChunks, p = i % kRunChunks;
            const int64_t e = e0 + (int64_t)q * V + EPC * p;
            if (e >= A.n) continue;
            RunVec<T> v = run_ld<T>(s_dyn + (q / kAddNT) * RBB, run_chunk_off(q % kAddNT, p));
            if (e + EPC <= A.n) {
                RunVec<T>* dst = reinterpret_cast<RunVec<T>*>(abar + e);
                if (A.accumulate) {
                    const RunVec<T> o = *dst;
#pragma unroll
                    for (int j = 0; j < EPC; ++j) v.v[j] += o.v[j];
                }
                *dst = v;
            } else {
#pragma unroll
                for (int j = 0; j < EPC; ++j)
                    if (e + j < A.n) abar[e + j] = A.accumulate ? abar[e + j] + v.v[j] : v.v[j];
            }
        }
    }
}

// ------------------------------------------ linear recurrence, per-thread runs
// Host side of scan_runs.cuh: workspace layout, tensor maps, launches.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// An array of n elements seen as [n / V runs][1][V] (one 128-byte row per
// run): box of NT runs, 128-byte swizzle (one array tile per copy).
template <class T>
bool make_run_map(CUtensorMap* m, const T* ptr, int64_t n) {
    EncodeTiledFn f = encode_tiled();
    if (!f) return false;
    constexpr int V = RunCfg<T>::V;
    cuuint64_t dims[3] = {(cuuint64_t)V, 1, (cuuint64_t)(n / V)};
    cuuint64_t strides[2] = {128, 128};
    cuuint32_t box[3] = {(cuuint32_t)V, 1, (cuuint32_t)RunCfg<T>::NT};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return f(m, dt, 3, const_cast<T*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// An array of n elements as [n / V rows][1][V], box of kAddNT rows, 128-byte
// swizzle: one row block per copy.
template <class T>
bool make_add_map(CUtensorMap* m, const T* ptr, int64_t n) {
    EncodeTiledFn f = encode_tiled();
    if (!f) return false;
    constexpr int V = RunCfg<T>::V;
    cuuint64_t dims[3] = {(cuuint64_t)V, 1, (cuuint64_t)(n / V)};
    cuuint64_t strides[2] = {128, 128};
    cuuint32_t box[3] = {(cuuint32_t)V, 1, (cuuint32_t)kAddNT};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return f(m, dt, 3, const_cast<T*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class T>
int launch_add_runs(ScanArgs A, cudaStream_t stream) {
    using C = AddRunCfg<T>;
    static bool configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ADPAR_ERR_CUDA;
    if (!configured[dev]) {
        if (cudaFuncSetAttribute(scan_add_runs_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem) !=
            cudaSuccess)
            return ADPAR_ERR_CUDA;
        configured[dev] = true;
    }
    A.tiles = (A.n + C::TILE - 1) / C::TILE;
    if (A.tiles == 0) return ADPAR_OK;
    CUtensorMap tm[2];
    memset(tm, 0, sizeof(tm));
    if (A.n >= C::TILE) {  // whole tiles exist: they move by TMA
        if (!make_add_map<T>(&tm[0], static_cast<const T*>(A.ya), A.n) ||
            !make_add_map<T>(&tm[1], static_cast<const T*>(A.abar), A.n))
            return ADPAR_ERR_CUDA;
    }
    scan_add_runs_kernel<T><<<(unsigned)A.tiles, kAddNT, C::kSmem, stream>>>(tm[0], tm[1], A);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

struct RunLayout {
    size_t off_slots, slot_words, off_pA, off_pI, off_rA, off_rI, off_carA, off_carB, off_prod, total;
    int64_t tiles;
};

template <class T>
RunLayout run_layout(int64_t n) {
    RunLayout L;
    L.tiles = (n + RunCfg<T>::TILE - 1) / RunCfg<T>::TILE;
    const size_t t = (size_t)L.tiles;
    const size_t wp = t * (size_t)lb_words<RunP<T>>(), wr = t * (size_t)lb_words<RunL<T>>();
    size_t o = sizeof(WsHeader);
    L.off_slots = o;
    L.off_pA = o; o += wp * 8;
    L.off_pI = o; o += wp * 8;
    L.off_rA = o; o += wr * 8;
    L.off_rI = o; o += wr * 8;
    L.slot_words = (o - L.off_slots) / 8;
    const size_t runs = t * (size_t)RunCfg<T>::NT;
    o = round_up(o, 256);
    L.off_carA = o; o = round_up(o + runs * sizeof(T), 256);
    L.off_carB = o; o = round_up(o + runs * sizeof(T), 256);
    L.off_prod = o; o = round_up(o + runs * sizeof(T), 256);
    L.total = o;
    return L;
}

// The runs path's common part: workspace pointers, tensor maps (a, b and
// the outputs abar, bbar; ya, yb when given) and the carry pass with the
// segmented carry scan.  Returns ADPAR_OK or an error before launching.
template <class T>
int runs_carry_pass(int64_t n, const void* a, const void* b, const void* ya, const void* yb, void* abar, void* bbar,
                    uint32_t flags, void* work, RunArgs<T>& R, CUtensorMap (&tm)[6], cudaStream_t stream) {
    using Cf = RunCfg<T>;
    const RunLayout L = run_layout<T>(n);
    char* w = static_cast<char*>(work);
    R = RunArgs<T>{};
    R.n = n;
    R.tiles = L.tiles;
    R.a = static_cast<const T*>(a);
    R.b = static_cast<const T*>(b);
    R.ya = static_cast<const T*>(ya);
    R.yb = static_cast<const T*>(yb);
    R.abar = static_cast<T*>(abar);
    R.bbar = static_cast<T*>(bbar);
    R.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    R.hdr = reinterpret_cast<WsHeader*>(w);
    R.lbR_agg = reinterpret_cast<unsigned long long*>(w + L.off_rA);
    R.lbR_incl = reinterpret_cast<unsigned long long*>(w + L.off_rI);
    R.carA = reinterpret_cast<T*>(w + L.off_carA);
    R.carB = reinterpret_cast<T*>(w + L.off_carB);
    R.prod = reinterpret_cast<T*>(w + L.off_prod);
    // the tile aggregates and carries take the primal look-back slots
    static_assert(lb_words<RunP<T>>() * 8 >= sizeof(RunP<T>), "a state fits a slot");
    R.tagg = reinterpret_cast<RunP<T>*>(w + L.off_pA);
    R.tcar = reinterpret_cast<RunP<T>*>(w + L.off_pI);
    memset(tm, 0, sizeof(tm));
    if (n >= Cf::TILE) {
        // whole tiles exist: their copies go through TMA (the partial last
        // tile, and every tile when n < one tile, is copied element-wise)
        const T* ptr[6] = {R.a, R.b, R.ya, R.yb, R.abar, R.bbar};
        for (int i = 0; i < 6; ++i)
            if (ptr[i] && !make_run_map<T>(&tm[i], ptr[i], n)) return ADPAR_ERR_CUDA;
    }
    static bool configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ADPAR_ERR_CUDA;
    if (!configured[dev]) {
        if (cudaFuncSetAttribute(linrec_runs_carry_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * Cf::ARR) != cudaSuccess ||
            cudaFuncSetAttribute(linrec_runs_vjp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 3 * Cf::ARR) != cudaSuccess ||
            cudaFuncSetAttribute(linrec_runs_reduce_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * Cf::ARR) != cudaSuccess)
            return ADPAR_ERR_CUDA;
        configured[dev] = true;
    }
    const int64_t words = (int64_t)L.slot_words;
    const int iblocks = (int)std::min<int64_t>((words + 255) / 256 + 1, 2048);
    scan_init_kernel<<<iblocks, 256, 0, stream>>>(R.hdr, reinterpret_cast<unsigned long long*>(w + L.off_slots),
                                                  words);
    linrec_runs_carry_kernel<T><<<(unsigned)L.tiles, Cf::NT, 2 * Cf::ARR, stream>>>(tm[0], tm[1], R);
    // the segment totals take the second half of the tile aggregates' slots
    static_assert(lb_words<RunP<T>>() * 8 >= 2 * sizeof(RunP<T>), "room after the aggregates");
    launch_carry_scan<RunPOp<T>>(R.tagg, R.tcar, R.tagg + L.tiles, L.tiles, stream);
    return ADPAR_OK;
}

// the scan VJP on per-thread runs
template <class T>
int run_linrec_runs(int64_t n, const void* a, const void* b, const void* ya, const void* yb, void* abar,
                    void* bbar, uint32_t flags, void* work, cudaStream_t stream) {
    using Cf = RunCfg<T>;
    RunArgs<T> R;
    CUtensorMap tm[6];
    const int st = runs_carry_pass<T>(n, a, b, ya, yb, abar, bbar, flags, work, R, tm, stream);
    if (st != ADPAR_OK) return st;
    linrec_runs_vjp_kernel<T><<<(unsigned)R.tiles, Cf::NT, 3 * Cf::ARR, stream>>>(tm[0], tm[2], tm[3], tm[4], tm[5], R);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

// the reduce VJP by the general rule on per-thread runs (ybar_a, ybar_b:
// device scalars; y_a, y_b nullable device scalars for the reduction)
template <class T>
int run_linrec_runs_reduce(int64_t n, const void* a, const void* b, const void* ybar_a, const void* ybar_b,
                           void* abar, void* bbar, void* y_a, void* y_b, uint32_t flags, void* work,
                           cudaStream_t stream) {
    using Cf = RunCfg<T>;
    RunArgs<T> R;
    CUtensorMap tm[6];
    const int st = runs_carry_pass<T>(n, a, b, nullptr, nullptr, abar, bbar, flags, work, R, tm, stream);
    if (st != ADPAR_OK) return st;
    linrec_runs_reduce_kernel<T><<<(unsigned)R.tiles, Cf::NT, 2 * Cf::ARR, stream>>>(
        tm[0], tm[1], tm[4], tm[5], R, static_cast<const T*>(ybar_a), static_cast<const T*>(ybar_b),
        static_cast<T*>(y_a), static_cast<T*>(y_b));
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

// ------------------------------------------------------------ host side
struct ScanLayout {
    size_t off_carry, off_slots, off_pA, off_pI, off_rA, off_rI, slot_words, total_min;
    size_t off_loc_a, off_loc_b, off_thc, total;
    size_t off_xloc, off_floc, off_gagg, off_fx, off_ff;  // min/max rule only
};

// The FP64 * scan takes the factored forward result (scan_primal_fac_tile)
// when the workspace holds it; the FP64 linear recurrence takes per-thread
// runs (scan_runs.cuh) instead.
template <class Op, class T>
constexpr bool kFactored = Op::kCoefIsA && sizeof(T) == 8 && Op::kWidth == 1;

// MIN/MAX take the fused single-pass rule (scan_minmax_fused_kernel).
template <class Op, class T>
constexpr bool kMinMax = std::is_same<Op, OpMax<T>>::value || std::is_same<Op, OpMin<T>>::value;

// header | carry[tiles] | look-back slots (primal agg, primal incl,
// adjoint agg, adjoint incl), the slots contiguous so one kernel zeroes
// them  [total_min]  | loc_a | loc_b | thread carries  [total]
template <class Op, class T>
ScanLayout scan_layout(int64_t n) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    using L = Lin<T, Op::kWidth, !Op::kCoefOne>;
    const size_t tiles = (size_t)((n + Cfg::TILE - 1) / Cfg::TILE);
    const size_t wp = tiles * (size_t)lb_words<P>(), wr = tiles * (size_t)lb_words<L>();
    ScanLayout s;
    size_t o = sizeof(WsHeader);
    s.off_carry = o; o = round_up(o + tiles * sizeof(P), 256);
    s.off_slots = o;
    s.off_pA = o; o += wp * 8;
    s.off_pI = o; o += wp * 8;
    s.off_rA = o; o += wr * 8;
    s.off_rI = o; o += wr * 8;
    s.slot_words = (o - s.off_slots) / 8;
    s.off_xloc = s.off_floc = s.off_gagg = s.off_fx = s.off_ff = 0;
    if constexpr (kMinMax<Op, T>) {
        const size_t groups = (tiles + kMmGroup - 1) / kMmGroup;
        o = round_up(o, 256);
        s.off_xloc = o; o = round_up(o + tiles * 8, 256);
        s.off_floc = o; o = round_up(o + tiles * 4, 256);
        s.off_gagg = o; o = round_up(o + groups * sizeof(P), 256);
        s.off_fx = o; o = round_up(o + groups * 8, 256);
        s.off_ff = o; o += groups * 4;
    }
    s.total_min = round_up(o, 256);
    o = s.total_min;
    s.off_loc_a = s.off_loc_b = s.off_thc = 0;
    if constexpr (kFactored<Op, T>) {
        // padded to whole tiles of the factored primal pass; its look-back
        // slots fit in those above (fewer, no larger tiles)
        static_assert(kFacTile >= Cfg::TILE, "factored tiles are no smaller");
        const size_t ftiles = (size_t)((n + kFacTile - 1) / kFacTile);
        const size_t ptiles = round_up(ftiles, (size_t)kFacKP);
        const size_t elems = ptiles * (size_t)kFacTile;
        s.off_loc_a = o; o = round_up(o + elems * sizeof(T), 256);
        if (Op::kWidth == 2) { s.off_loc_b = o; o = round_up(o + elems * sizeof(T), 256); }
        s.off_thc = o; o = round_up(o + ptiles * (size_t)kScanBlock * sizeof(P), 256);
    }
    s.total = o;
    if constexpr (std::is_same<Op, OpLinrec<T>>::value)
        s.total = std::max(s.total, run_layout<T>(n).total);
    return s;
}

inline void set_slots(ScanArgs& A, char* w, const ScanLayout& L) {
    A.carry = w + L.off_carry;
    A.lbP_agg = reinterpret_cast<unsigned long long*>(w + L.off_pA);
    A.lbP_incl = reinterpret_cast<unsigned long long*>(w + L.off_pI);
    A.lbR_agg = reinterpret_cast<unsigned long long*>(w + L.off_rA);
    A.lbR_incl = reinterpret_cast<unsigned long long*>(w + L.off_rI);
}

inline void launch_init(const ScanArgs& A, char* w, const ScanLayout& L, cudaStream_t stream) {
    const int64_t words = (int64_t)L.slot_words;
    const int blocks = (int)std::min<int64_t>((words + 255) / 256 + 1, 2048);
    scan_init_kernel<<<blocks, 256, 0, stream>>>(A.hdr, reinterpret_cast<unsigned long long*>(w + L.off_slots),
                                                 words);
}

// blocks of the persistent min/max pass: two per SM (its register use)
inline int fused_grid() {
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = 2 * (sms > 0 ? sms : 1);
    }
    return g;
}

template <class Op, class T>
int run_scan(int64_t n, const void* a, const void* b, const void* ya, const void* yb, void* abar,
             void* bbar, void* ys_a, void* ys_b, uint32_t flags, void* work, size_t work_bytes,
             cudaStream_t stream) {
    using Cfg = ScanCfg<Op, T>;
    const ScanLayout L = scan_layout<Op, T>(n);
    if (work == nullptr || work_bytes < L.total_min || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) return ADPAR_OK;
    char* w = static_cast<char*>(work);
    ScanArgs A{};
    A.n = n;
    A.a = a; A.b = b; A.ya = ya; A.yb = yb;
    A.abar = abar; A.bbar = bbar; A.ys_a = ys_a; A.ys_b = ys_b;
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    A.tiles = (n + Cfg::TILE - 1) / Cfg::TILE;
    A.hdr = reinterpret_cast<WsHeader*>(w);
    set_slots(A, w, L);
    const bool need_primal = Op::kNeedPrimal || Op::kCoefNeedsPrimal || ys_a != nullptr;
    if constexpr (std::is_same<Op, OpLinrec<T>>::value) {
        // per-thread runs, when the workspace holds the runs' carries
        if (!ys_a && work_bytes >= run_layout<T>(n).total)
            return run_linrec_runs<T>(n, a, b, ya, yb, abar, bbar, flags, work, stream);
    }
    launch_init(A, w, L, stream);
    if constexpr (kFactored<Op, T>) {
        if (work_bytes >= L.total) {
            A.loc_a = w + L.off_loc_a;
            A.loc_b = Op::kWidth == 2 ? w + L.off_loc_b : nullptr;
            A.thr_carry = w + L.off_thc;
            A.tiles = (n + kFacTile - 1) / kFacTile;
            ScanArgs AP = A;
            AP.tiles = (A.tiles + kFacKP - 1) / kFacKP;
            scan_primal_fac_kernel<Op><<<(unsigned)AP.tiles, kScanBlock, 0, stream>>>(AP);
            if (ys_a) scan_adjoint_fac_kernel<Op, true><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
            else scan_adjoint_fac_kernel<Op, false><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
            return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
        }
    }
    if constexpr (kMinMax<Op, T>) {
        // tile extrema, their scan by groups, record-free tiles, tiles with
        // records, and the runs across tiles; the per-tile data take the
        // look-back slots (unused on this path) and the rule's own region
        using P = typename Op::P;
        static_assert(lb_words<P>() * 4 >= sizeof(P) && lb_words<P>() * 4 >= sizeof(uint32_t), "slot size");
        static_assert(lb_words<Lin<T, 1, true>>() * 4 >= 8, "8 bytes of metadata per tile");
        MinMaxWs<P> M;
        M.tmax = reinterpret_cast<P*>(A.lbP_agg);
        M.carry = static_cast<P*>(A.carry);
        M.gagg = reinterpret_cast<P*>(w + L.off_gagg);
        M.rec_list = reinterpret_cast<uint32_t*>(A.lbP_incl);
        M.n_rec = &A.hdr->done[1];  // zeroed by the init kernel
        M.lead = reinterpret_cast<double*>(A.lbR_agg);
        M.last = reinterpret_cast<int64_t*>(A.lbR_incl);
        M.xloc = reinterpret_cast<double*>(w + L.off_xloc);
        M.floc = reinterpret_cast<uint32_t*>(w + L.off_floc);
        M.fx = reinterpret_cast<double*>(w + L.off_fx);
        M.ff = reinterpret_cast<uint32_t*>(w + L.off_ff);
        M.tiles = A.tiles;
        M.groups = (int)((A.tiles + kMmGroup - 1) / kMmGroup);
        const unsigned fgrid = (unsigned)std::min<int64_t>(A.tiles, (int64_t)fused_grid());
        scan_minmax_tile_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A, M.tmax);
        scan_minmax_group_kernel<Op, T><<<M.groups, kMmGroup, 0, stream>>>(M);
        if (ys_a) {
            scan_minmax_zero_kernel<Op, T, true><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A, M);
            scan_minmax_fused_kernel<Op, T, true><<<fgrid, kScanBlock, 0, stream>>>(A, M.rec_list, M.n_rec, M.lead,
                                                                                     M.last);
        } else {
            scan_minmax_zero_kernel<Op, T, false><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A, M);
            scan_minmax_fused_kernel<Op, T, false><<<fgrid, kScanBlock, 0, stream>>>(A, M.rec_list, M.n_rec, M.lead,
                                                                                      M.last);
        }
        scan_minmax_runs_kernel<P><<<M.groups, kMmGroup, 0, stream>>>(M);
        scan_minmax_fixup_kernel<P, T><<<M.groups, kMmGroup, 0, stream>>>(M, static_cast<T*>(A.abar));
    } else {
        if constexpr (std::is_same<Op, OpAdd<T>>::value) {
            // the tile in shared memory needs fewer look-back slots than the
            // register tile the layout is sized for (its tiles are larger)
            static_assert(AddRunCfg<T>::TILE >= ScanCfg<Op, T>::TILE, "no more tiles than slots");
            if (!ys_a) return launch_add_runs<T>(A, stream);
        }
        if (need_primal) {
            // the tile aggregates take the primal aggregate slots, unused here
            using P = typename Op::P;
            // (and the segment totals of the carry scan their second half)
            static_assert(lb_words<P>() * 8 >= 2 * sizeof(P), "an aggregate and a total fit a slot");
            P* agg = reinterpret_cast<P*>(A.lbP_agg);
            scan_tile_agg_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A, agg);
            launch_carry_scan<Op>(agg, static_cast<P*>(A.carry), agg + A.tiles, A.tiles, stream);
        }
        if (ys_a) scan_adjoint_kernel<Op, T, true><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
        else scan_adjoint_kernel<Op, T, false><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    }
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T>
ScanLayout scan_layout_of(int op, int64_t n, bool& ok) {
    ok = true;
    switch (op) {
    case ADPAR_OP_ADD: return scan_layout<OpAdd<T>, T>(n);
    case ADPAR_OP_MUL: return scan_layout<OpMul<T>, T>(n);
    case ADPAR_OP_MIN: return scan_layout<OpMin<T>, T>(n);
    case ADPAR_OP_MAX: return scan_layout<OpMax<T>, T>(n);
    case ADPAR_OP_LINREC: return scan_layout<OpLinrec<T>, T>(n);
    }
    ok = false;
    return ScanLayout{};
}

template <class T>
int dispatch_scan(int op, int64_t n, const void* a, const void* b, const void* ya, const void* yb,
                  void* abar, void* bbar, void* ys_a, void* ys_b, uint32_t flags, void* work,
                  size_t work_bytes, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD:
        return run_scan<OpAdd<T>, T>(n, a, b, ya, yb, abar, bbar, ys_a, ys_b, flags, work, work_bytes, s);
    case ADPAR_OP_MUL:
        return run_scan<OpMul<T>, T>(n, a, b, ya, yb, abar, bbar, ys_a, ys_b, flags, work, work_bytes, s);
    case ADPAR_OP_MIN:
        return run_scan<OpMin<T>, T>(n, a, b, ya, yb, abar, bbar, ys_a, ys_b, flags, work, work_bytes, s);
    case ADPAR_OP_MAX:
        return run_scan<OpMax<T>, T>(n, a, b, ya, yb, abar, bbar, ys_a, ys_b, flags, work, work_bytes, s);
    case ADPAR_OP_LINREC:
        return run_scan<OpLinrec<T>, T>(n, a, b, ya, yb, abar, bbar, ys_a, ys_b, flags, work, work_bytes, s);
    }
    return ADPAR_ERR_INVALID;
}

template <class Op, class T>
int run_scan_forward(int64_t n, const void* a, const void* b, void* ys_a, void* ys_b, void* work,
                     size_t work_bytes, cudaStream_t stream) {
    using Cfg = ScanCfg<Op, T>;
    const ScanLayout L = scan_layout<Op, T>(n);
    if (work == nullptr || work_bytes < L.total_min || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) return ADPAR_OK;
    char* w = static_cast<char*>(work);
    ScanArgs A{};
    A.n = n;
    A.a = a; A.b = b; A.ys_a = ys_a; A.ys_b = ys_b;
    A.tiles = (n + Cfg::TILE - 1) / Cfg::TILE;
    A.hdr = reinterpret_cast<WsHeader*>(w);
    set_slots(A, w, L);
    launch_init(A, w, L, stream);
    scan_forward_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T>
int dispatch_scan_forward(int op, int64_t n, const void* a, const void* b, void* ys_a, void* ys_b,
                          void* work, size_t work_bytes, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD: return run_scan_forward<OpAdd<T>, T>(n, a, b, ys_a, ys_b, work, work_bytes, s);
    case ADPAR_OP_MUL: return run_scan_forward<OpMul<T>, T>(n, a, b, ys_a, ys_b, work, work_bytes, s);
    case ADPAR_OP_MIN: return run_scan_forward<OpMin<T>, T>(n, a, b, ys_a, ys_b, work, work_bytes, s);
    case ADPAR_OP_MAX: return run_scan_forward<OpMax<T>, T>(n, a, b, ys_a, ys_b, work, work_bytes, s);
    case ADPAR_OP_LINREC: return run_scan_forward<OpLinrec<T>, T>(n, a, b, ys_a, ys_b, work, work_bytes, s);
    }
    return ADPAR_ERR_INVALID;
}

// ----------------------------------------------------- forward mode (JVP)
template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_jvp_kernel(ScanArgs A, const T* ad, const T* bd, T* yd_a,
                                                               T* yd_b) {
    using Cfg = ScanCfg<Op, T>;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    scan_jvp_tile<Op, T, Cfg::K, Cfg::E>(A, (int64_t)s_tile, ad, bd, yd_a, yd_b);
}

template <class Op, class T>
int run_scan_jvp(int64_t n, const void* a, const void* b, const void* ad, const void* bd, void* ys_a, void* ys_b,
                 void* yd_a, void* yd_b, void* work, size_t work_bytes, cudaStream_t stream) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    const ScanLayout L = scan_layout<Op, T>(n);
    if (work == nullptr || work_bytes < L.total_min || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) return ADPAR_OK;
    // the dual state's slots: 2 words(P) per tile in each of the two regions
    static_assert(lb_words<DualState<Op>>() == 2 * lb_words<P>(), "dual slots");
    static_assert(lb_words<P>() <= lb_words<Lin<T, Op::kWidth, !Op::kCoefOne>>(), "slot width");
    char* w = static_cast<char*>(work);
    ScanArgs A{};
    A.n = n;
    A.a = a; A.b = b; A.ys_a = ys_a; A.ys_b = ys_b;
    A.tiles = (n + Cfg::TILE - 1) / Cfg::TILE;
    A.hdr = reinterpret_cast<WsHeader*>(w);
    set_slots(A, w, L);
    launch_init(A, w, L, stream);
    scan_jvp_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(
        A, static_cast<const T*>(ad), static_cast<const T*>(bd), static_cast<T*>(yd_a), static_cast<T*>(yd_b));
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

// the linear recurrence's forward mode on per-thread runs (scan_runs.cuh);
// its tiles are the scan engine's, so the minimal workspace's dual-state
// slots serve it
template <class T>
int run_linrec_runs_jvp(int64_t n, const void* a, const void* b, const void* ad, const void* bd, void* ys_a,
                        void* ys_b, void* yd_a, void* yd_b, void* work, size_t work_bytes, cudaStream_t stream) {
    using Cf = RunCfg<T>;
    using Op = OpLinrec<T>;
    static_assert(Cf::TILE == ScanCfg<Op, T>::TILE, "runs tiles are the engine's tiles");
    static_assert(lb_words<RunD<T>>() == lb_words<DualState<Op>>(), "dual slots");
    const ScanLayout L = scan_layout<Op, T>(n);
    if (work == nullptr || work_bytes < L.total_min || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) return ADPAR_OK;
    char* w = static_cast<char*>(work);
    RunJvpArgs<T> R{};
    R.n = n;
    R.tiles = (n + Cf::TILE - 1) / Cf::TILE;
    R.a = static_cast<const T*>(a);
    R.b = static_cast<const T*>(b);
    R.ad = static_cast<const T*>(ad);
    R.bd = static_cast<const T*>(bd);
    R.ys_a = static_cast<T*>(ys_a);
    R.ys_b = static_cast<T*>(ys_b);
    R.yd_a = static_cast<T*>(yd_a);
    R.yd_b = static_cast<T*>(yd_b);
    R.hdr = reinterpret_cast<WsHeader*>(w);
    // a dual state is twice a primal state: its aggregate slots span the
    // primal aggregate and inclusive regions, its inclusive slots the
    // adjoint ones (as for the engine's forward mode)
    R.lb_agg = reinterpret_cast<unsigned long long*>(w + L.off_pA);
    R.lb_incl = reinterpret_cast<unsigned long long*>(w + L.off_rA);
    static_assert(lb_words<RunD<T>>() <= 2 * lb_words<RunL<T>>(), "inclusive slots fit the adjoint regions");
    CUtensorMap tm[8];
    memset(tm, 0, sizeof(tm));
    if (n >= Cf::TILE) {
        const T* ptr[8] = {R.a, R.b, R.ad, R.bd, R.ys_a, R.ys_b, R.yd_a, R.yd_b};
        for (int i = 0; i < 8; ++i)
            if (ptr[i] && !make_run_map<T>(&tm[i], ptr[i], n)) return ADPAR_ERR_CUDA;
    }
    static bool configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ADPAR_ERR_CUDA;
    if (!configured[dev]) {
        if (cudaFuncSetAttribute(linrec_runs_jvp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * Cf::ARR) != cudaSuccess)
            return ADPAR_ERR_CUDA;
        configured[dev] = true;
    }
    ScanArgs A{};
    A.hdr = R.hdr;
    A.tiles = R.tiles;
    set_slots(A, w, L);
    launch_init(A, w, L, stream);
    linrec_runs_jvp_kernel<T><<<(unsigned)R.tiles, Cf::NT, 4 * Cf::ARR, stream>>>(tm[0], tm[1], tm[2], tm[3], tm[4],
                                                                                   tm[5], tm[6], tm[7], R);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T>
int dispatch_scan_jvp(int op, int64_t n, const void* a, const void* b, const void* ad, const void* bd, void* ys_a,
                      void* ys_b, void* yd_a, void* yd_b, void* work, size_t work_bytes, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD: return run_scan_jvp<OpAdd<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_MUL: return run_scan_jvp<OpMul<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_MIN: return run_scan_jvp<OpMin<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_MAX: return run_scan_jvp<OpMax<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_LINREC:
        return run_linrec_runs_jvp<T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    }
    return ADPAR_ERR_INVALID;
}

// --------------------------------------------- reduce, general rule (Sec. 5.1)
// y = a_0 (.) ... (.) a_{n-1} for any operator above, and
//   a_bar_i (+)= d(l_i (.) a_i (.) r_i)/d a_i ^T y_bar
// with l_i = a_0 (.) ... (.) a_{i-1} (forward exclusive scan) and
// r_i = a_{i+1} (.) ... (.) a_{n-1} (reverse exclusive scan).  Pass P above
// gives every tile's l at its first element; this pass takes tiles right to
// left, re-forms l inside the tile from that carry, forms r with a reverse
// block scan of the operator's own state and a look-back over the tiles to
// the right, and applies mid_vjp per element.
template <class Op, class T, int K, int V>
__device__ __forceinline__ void reduce_general_tile(const ScanArgs& A, int64_t t_log, const T* ybar_a,
                                                    const T* ybar_b, T* y_a, T* y_b) {
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, TILE = K * kScanBlock * V;
    __shared__ P s_totF[K * NW];
    __shared__ P s_totR[K * NW];
    __shared__ P s_carry;
    __shared__ P s_suf;
    const int64_t tile = A.tiles - 1 - t_log;  // data tile (t_log counts from the right)
    const int64_t base = tile * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);

    T av[K][V], bv[K][V];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        load_chunk(a, e, A.n, Op::pad_a(), av[k]);  // padding is the neutral element
        if constexpr (W == 2) load_chunk(b, e, A.n, T(0), bv[k]);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[k][j] = T(0);
        }
    }
    if (threadIdx.x == 0) s_carry = static_cast<const P*>(A.carry)[tile];
    P agg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        P acc = Op::pelem(av[k][0], bv[k][0]);
#pragma unroll
        for (int j = 1; j < V; ++j) acc = Op::pcomb(acc, Op::pelem(av[k][j], bv[k][j]));
        agg[k] = acc;
    }
    auto fc = [](const P& l, const P& r) { return Op::pcomb(l, r); };
    // reverse scan order: e holds elements later in the array, l earlier ones
    auto rc = [](const P& e, const P& l) { return Op::pcomb(l, e); };
    P wexF[K], wexR[K];
    const P totF = block_scan_part1<P, false, K, NW>(agg, wexF, s_totF, Op::pid(), fc);
    const P totR = block_scan_part1<P, true, K, NW>(agg, wexR, s_totR, Op::pid(), rc);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<P> st{A.lbR_agg, A.lbR_incl};
        const P suf = lookback(t_log, st, totR, Op::pid(), rc, A.hdr);
        if ((threadIdx.x & 31) == 0) {
            s_suf = suf;
            if (tile == A.tiles - 1 && y_a) {  // y = (everything before this tile) (.) this tile
                const P y = Op::pcomb(s_carry, totF);
                *y_a = Op::out_a(y);
                if constexpr (W == 2) *y_b = Op::out_b(y);
            }
        }
    }
    __syncthreads();

    const T ya = *ybar_a;
    const T yb = W == 2 ? *ybar_b : T(0);
    T* abar = static_cast<T*>(A.abar);
    T* bbar = static_cast<T*>(A.bbar);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        if (e >= A.n) continue;
        P lj[V];
        lj[0] = block_scan_excl<P, false, K, NW>(k, wexF, s_totF, s_carry, fc);
#pragma unroll
        for (int j = 1; j < V; ++j) lj[j] = Op::pcomb(lj[j - 1], Op::pelem(av[k][j - 1], bv[k][j - 1]));
        P r = block_scan_excl<P, true, K, NW>(k, wexR, s_totR, s_suf, rc);
        T oa[V], ob[V];
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {
            T o1 = T(0), o2 = T(0);
            Op::mid_vjp(lj[j], av[k][j], bv[k][j], r, ya, yb, o1, o2);
            oa[j] = o1;
            ob[j] = o2;
            if (j > 0) r = Op::pcomb(Op::pelem(av[k][j], bv[k][j]), r);
        }
        if (A.accumulate) {
            T old[V];
            load_chunk_keep(static_cast<const T*>(A.abar), e, A.n, T(0), old);
#pragma unroll
            for (int j = 0; j < V; ++j) oa[j] += old[j];
            if constexpr (W == 2) {
                load_chunk_keep(static_cast<const T*>(A.bbar), e, A.n, T(0), old);
#pragma unroll
                for (int j = 0; j < V; ++j) ob[j] += old[j];
            }
        }
        store_chunk(abar, e, A.n, oa);
        if constexpr (W == 2) store_chunk(bbar, e, A.n, ob);
    }
}

template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) reduce_general_kernel(ScanArgs A, const T* ybar_a, const T* ybar_b,
                                                                     T* y_a, T* y_b) {
    using Cfg = ScanCfg<Op, T>;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    reduce_general_tile<Op, T, Cfg::K, Cfg::E>(A, (int64_t)s_tile, ybar_a, ybar_b, y_a, y_b);
}

// n = 0: y is the neutral element
template <class Op, class T>
__global__ void reduce_neutral_kernel(T* y_a, T* y_b) {
    if (y_a) *y_a = Op::out_a(Op::pid());
    if (y_b) *y_b = Op::out_b(Op::pid());
}

template <class Op, class T>
int run_reduce_general(int64_t n, const void* a, const void* b, const void* ybar_a, const void* ybar_b,
                       void* abar, void* bbar, void* y_a, void* y_b, uint32_t flags, void* work,
                       size_t work_bytes, cudaStream_t stream) {
    using Cfg = ScanCfg<Op, T>;
    const ScanLayout L = scan_layout<Op, T>(n);
    if (work == nullptr || work_bytes < L.total_min || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) {
        if (y_a) reduce_neutral_kernel<Op, T><<<1, 1, 0, stream>>>(static_cast<T*>(y_a), static_cast<T*>(y_b));
        return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
    }
    if constexpr (std::is_same<Op, OpLinrec<T>>::value) {
        // per-thread runs, when the workspace holds the runs' carries
        if (work_bytes >= run_layout<T>(n).total)
            return run_linrec_runs_reduce<T>(n, a, b, ybar_a, ybar_b, abar, bbar, y_a, y_b, flags, work, stream);
    }
    char* w = static_cast<char*>(work);
    ScanArgs A{};
    A.n = n;
    A.a = a; A.b = b;
    A.abar = abar; A.bbar = bbar;
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    A.tiles = (n + Cfg::TILE - 1) / Cfg::TILE;
    A.hdr = reinterpret_cast<WsHeader*>(w);
    set_slots(A, w, L);  // the reverse pass's slots hold operator states (no wider than lin_o's)
    static_assert(lb_words<typename Op::P>() <= lb_words<Lin<T, Op::kWidth, !Op::kCoefOne>>(), "slot width");
    launch_init(A, w, L, stream);
    scan_primal_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    reduce_general_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(
        A, static_cast<const T*>(ybar_a), static_cast<const T*>(ybar_b), static_cast<T*>(y_a), static_cast<T*>(y_b));
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T>
int dispatch_reduce_general(int op, int64_t n, const void* a, const void* b, const void* ya, const void* yb,
                            void* abar, void* bbar, void* y_a, void* y_b, uint32_t flags, void* work,
                            size_t work_bytes, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD:
        return run_reduce_general<OpAdd<T>, T>(n, a, b, ya, yb, abar, bbar, y_a, y_b, flags, work, work_bytes, s);
    case ADPAR_OP_MUL:
        return run_reduce_general<OpMul<T>, T>(n, a, b, ya, yb, abar, bbar, y_a, y_b, flags, work, work_bytes, s);
    case ADPAR_OP_MIN:
        return run_reduce_general<OpMin<T>, T>(n, a, b, ya, yb, abar, bbar, y_a, y_b, flags, work, work_bytes, s);
    case ADPAR_OP_MAX:
        return run_reduce_general<OpMax<T>, T>(n, a, b, ya, yb, abar, bbar, y_a, y_b, flags, work, work_bytes, s);
    case ADPAR_OP_LINREC:
        return run_reduce_general<OpLinrec<T>, T>(n, a, b, ya, yb, abar, bbar, y_a, y_b, flags, work, work_bytes,
                                                  s);
    }
    return ADPAR_ERR_INVALID;
}

}  // namespace

// minimal = false: the size that runs every pass at full speed (the
// factored forward result included); minimal = true: the smallest accepted
size_t scan_workspace_size(adpar_opdesc d, int64_t n, bool minimal) {
    if (n < 0) return (size_t)-1;
    bool ok = false;
    ScanLayout L{};
    if (d.dtype == ADPAR_F32) L = scan_layout_of<float>(d.op, n, ok);
    else if (d.dtype == ADPAR_F64) L = scan_layout_of<double>(d.op, n, ok);
    if (!ok) return (size_t)-1;
    return minimal ? L.total_min : L.total;
}

// the general reduce rule: the scan's slots, and for the linear recurrence
// (unless minimal) room for the runs path's carries
size_t reduce_general_workspace_size(adpar_opdesc d, int64_t n, bool minimal) {
    const size_t base = scan_workspace_size(d, n, true);
    if (base == (size_t)-1 || minimal || d.op != ADPAR_OP_LINREC) return base;
    const size_t runs = d.dtype == ADPAR_F32 ? run_layout<float>(n).total : run_layout<double>(n).total;
    return std::max(base, runs);
}

}  // namespace adpar

extern "C" int adpar_vjp_scan(adpar_opdesc d, int64_t n, const void* a, const void* b,
                              const void* ybar_a, const void* ybar_b, void* abar, void* bbar,
                              void* ys_a, void* ys_b, uint32_t flags, void* work,
                              size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0) return ADPAR_ERR_INVALID;
    if (d.op < ADPAR_OP_ADD || d.op > ADPAR_OP_LINREC) return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    const int want_w = d.op == ADPAR_OP_LINREC ? 2 : 1;
    if (d.width != want_w) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    if (n > 0) {
        if (!ybar_a || !abar) return ADPAR_ERR_INVALID;
        const bool needs_a = d.op != ADPAR_OP_ADD || ys_a != nullptr;
        if (needs_a && !a) return ADPAR_ERR_INVALID;
        if (want_w == 2 && (!b || !ybar_b || !bbar)) return ADPAR_ERR_INVALID;
        if (want_w == 2 && ys_a && !ys_b) return ADPAR_ERR_INVALID;
        const void* ptrs[] = {a, b, ybar_a, ybar_b, abar, bbar, ys_a, ys_b};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.dtype == ADPAR_F32)
        return dispatch_scan<float>(d.op, n, a, b, ybar_a, ybar_b, abar, bbar, ys_a, ys_b, flags,
                                    work, work_bytes, s);
    return dispatch_scan<double>(d.op, n, a, b, ybar_a, ybar_b, abar, bbar, ys_a, ys_b, flags,
                                 work, work_bytes, s);
}

extern "C" int adpar_scan(adpar_opdesc d, int64_t n, const void* a, const void* b, void* ys_a,
                          void* ys_b, void* work, size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0) return ADPAR_ERR_INVALID;
    if (d.op < ADPAR_OP_ADD || d.op > ADPAR_OP_LINREC) return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    const int want_w = d.op == ADPAR_OP_LINREC ? 2 : 1;
    if (d.width != want_w) return ADPAR_ERR_INVALID;
    if (n > 0) {
        if (!a || !ys_a) return ADPAR_ERR_INVALID;
        if (want_w == 2 && (!b || !ys_b)) return ADPAR_ERR_INVALID;
        const void* ptrs[] = {a, b, ys_a, ys_b};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.dtype == ADPAR_F32) return dispatch_scan_forward<float>(d.op, n, a, b, ys_a, ys_b, work, work_bytes, s);
    return dispatch_scan_forward<double>(d.op, n, a, b, ys_a, ys_b, work, work_bytes, s);
}

extern "C" int adpar_vjp_reduce_general(adpar_opdesc d, int64_t n, const void* a, const void* b,
                                        const void* ybar_a, const void* ybar_b, void* abar, void* bbar,
                                        void* y_out_a, void* y_out_b, uint32_t flags, void* work,
                                        size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0) return ADPAR_ERR_INVALID;
    if (d.op < ADPAR_OP_ADD || d.op > ADPAR_OP_LINREC) return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    const int want_w = d.op == ADPAR_OP_LINREC ? 2 : 1;
    if (d.width != want_w) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    if (want_w == 2 && y_out_a && !y_out_b) return ADPAR_ERR_INVALID;
    if (n > 0) {
        if (!a || !ybar_a || !abar) return ADPAR_ERR_INVALID;
        if (want_w == 2 && (!b || !ybar_b || !bbar)) return ADPAR_ERR_INVALID;
        const void* ptrs[] = {a, b, abar, bbar};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.dtype == ADPAR_F32)
        return dispatch_reduce_general<float>(d.op, n, a, b, ybar_a, ybar_b, abar, bbar, y_out_a, y_out_b, flags,
                                              work, work_bytes, s);
    return dispatch_reduce_general<double>(d.op, n, a, b, ybar_a, ybar_b, abar, bbar, y_out_a, y_out_b, flags,
                                           work, work_bytes, s);
}

extern "C" int adpar_jvp_scan(adpar_opdesc d, int64_t n, const void* a, const void* b, const void* adot,
                              const void* bdot, void* ys_a, void* ys_b, void* ysdot_a, void* ysdot_b, void* work,
                              size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0) return ADPAR_ERR_INVALID;
    if (d.op < ADPAR_OP_ADD || d.op > ADPAR_OP_LINREC) return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    const int want_w = d.op == ADPAR_OP_LINREC ? 2 : 1;
    if (d.width != want_w) return ADPAR_ERR_INVALID;
    if (n > 0) {
        if (!a || !adot || !ysdot_a) return ADPAR_ERR_INVALID;
        if (want_w == 2 && (!b || !bdot || !ysdot_b)) return ADPAR_ERR_INVALID;
        if (want_w == 2 && ys_a && !ys_b) return ADPAR_ERR_INVALID;
        const void* ptrs[] = {a, b, adot, bdot, ys_a, ys_b, ysdot_a, ysdot_b};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.dtype == ADPAR_F32)
        return dispatch_scan_jvp<float>(d.op, n, a, b, adot, bdot, ys_a, ys_b, ysdot_a, ysdot_b, work, work_bytes, s);
    return dispatch_scan_jvp<double>(d.op, n, a, b, adot, bdot, ys_a, ys_b, ysdot_a, ysdot_b, work, work_bytes, s);
}
