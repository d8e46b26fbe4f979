// Tile-level bodies of the single-pass scans (Sec. 5.2), shared by the
// scan kernels and the batched kernel.  Each function processes one tile
// of one problem with the whole block; the caller hands out tiles (the
// "logical" tile order is the order in which look-back predecessors are
// guaranteed to have been handed out) and separates consecutive tiles of
// one block with __syncthreads().
//
// Tile shape: K chunks of kScanBlock * V elements; in each chunk a thread
// owns V consecutive elements (V a multiple of the 16-byte vector width).
#pragma once

#include "scan_engine.cuh"
#include "scan_ops.cuh"

namespace adpar {

constexpr int kScanBlock = 256;

struct ScanArgs {
    int64_t n;
    const void* a;
    const void* b;
    const void* ya;
    const void* yb;
    void* abar;
    void* bbar;
    void* ys_a;
    void* ys_b;
    int accumulate;
    int64_t tiles;
    WsHeader* hdr;
    void* carry;  // [tiles] P
    unsigned long long* lbP_agg;  // look-back slots of the primal pass
    unsigned long long* lbP_incl;
    unsigned long long* lbR_agg;  // look-back slots of the adjoint pass
    unsigned long long* lbR_incl;
};

// A thread's E consecutive elements of a chunk, as E / (16 / sizeof(T))
// 16-byte vectors; a partial chunk at the end of the data is read element
// by element and padded with `pad`.
template <int E, bool STREAM, class T>
__device__ __forceinline__ void load_chunk_e(const T* p, int64_t e, int64_t n, T pad, T (&out)[E]) {
    constexpr int VV = Vec16<T>::N;
    static_assert(E % VV == 0, "whole vectors");
    if (e + E <= n) {
#pragma unroll
        for (int q = 0; q < E / VV; ++q) {
            Vec16<T> x = STREAM ? ld_vec_stream(p + e + q * VV) : ld_vec(p + e + q * VV);
#pragma unroll
            for (int j = 0; j < VV; ++j) out[q * VV + j] = x.v[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) out[j] = (e + j < n) ? p[e + j] : pad;
    }
}

template <int E, class T>
__device__ __forceinline__ void load_chunk(const T* p, int64_t e, int64_t n, T pad, T (&out)[E]) {
    load_chunk_e<E, true>(p, e, n, pad, out);
}

template <int E, class T>
__device__ __forceinline__ void load_chunk_keep(const T* p, int64_t e, int64_t n, T pad, T (&out)[E]) {
    load_chunk_e<E, false>(p, e, n, pad, out);
}

template <int E, class T>
__device__ __forceinline__ void store_chunk(T* p, int64_t e, int64_t n, const T (&v)[E]) {
    constexpr int VV = Vec16<T>::N;
    if (e + E <= n) {
#pragma unroll
        for (int q = 0; q < E / VV; ++q) {
            Vec16<T> x;
#pragma unroll
            for (int j = 0; j < VV; ++j) x.v[j] = v[q * VV + j];
            st_vec(p + e + q * VV, x);
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (e + j < n) p[e + j] = v[j];
    }
}

// ---------------------------------------------------------------- pass P
template <class Op, class T, int K, int V>
__device__ __forceinline__ void scan_primal_tile(const ScanArgs& A, int64_t tile) {
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, TILE = K * kScanBlock * V;
    __shared__ P s_tot[K * NW];
    const int64_t base = tile * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);

    P agg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        T av[V], bv[V];
        load_chunk_keep(a, e, A.n, Op::pad_a(), av);
        if constexpr (Op::kWidth == 2) load_chunk_keep(b, e, A.n, T(0), bv);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[j] = T(0);
        }
        P acc = Op::pelem(av[0], bv[0]);
#pragma unroll
        for (int j = 1; j < V; ++j) acc = Op::pcomb(acc, Op::pelem(av[j], bv[j]));
        agg[k] = acc;
    }
    auto comb = [](const P& l, const P& r) { return Op::pcomb(l, r); };
    P wex[K];
    P total = block_scan_part1<P, false, K, NW>(agg, wex, s_tot, Op::pid(), comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<P> st{A.lbP_agg, A.lbP_incl};
        P prefix = lookback(tile, st, total, Op::pid(), comb, A.hdr);
        if ((threadIdx.x & 31) == 0 && A.carry) static_cast<P*>(A.carry)[tile] = prefix;
    }
}

// ---------------------------------------------------------------- pass R
// A full tile's input arrays staged in shared memory (the persistent
// kernel copies them there with bulk asynchronous copies): each array holds
// the tile's TILE elements contiguously, in data order.
template <class T>
struct StagedTile {
    const T* ya;
    const T* yb;
    const T* a;
    const T* b;
};

template <int E, class T>
__device__ __forceinline__ void load_smem_chunk(const T* p, int off, T (&out)[E]) {
    constexpr int VV = Vec16<T>::N;
#pragma unroll
    for (int q = 0; q < E / VV; ++q) {
        if constexpr (sizeof(T) == 4) {
            const float4 x = *reinterpret_cast<const float4*>(p + off + q * VV);
            out[q * VV + 0] = x.x; out[q * VV + 1] = x.y; out[q * VV + 2] = x.z; out[q * VV + 3] = x.w;
        } else {
            const double2 x = *reinterpret_cast<const double2*>(p + off + q * VV);
            out[q * VV + 0] = x.x; out[q * VV + 1] = x.y;
        }
    }
}

// SMEM: the inputs of this (full) tile are read from the staged copy.
template <class Op, class T, int K, int V, bool WYS, bool SMEM = false>
__device__ __forceinline__ void scan_adjoint_tile(const ScanArgs& A, int64_t t_log,
                                                  StagedTile<T> st = StagedTile<T>{}) {
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, TILE = K * kScanBlock * V;
    using L = Lin<T, W, !Op::kCoefOne>;
    constexpr bool kPrimal = Op::kNeedPrimal || Op::kCoefNeedsPrimal;

    __shared__ P s_totP[K * NW];
    __shared__ L s_totR[K * NW];
    __shared__ P s_carry;
    __shared__ L s_prefR;

    const int64_t tile = A.tiles - 1 - t_log;  // data tile (t_log counts from the right)
    const int64_t base = tile * TILE;
    constexpr bool write_ys = WYS;
    constexpr bool need_primal = kPrimal || WYS;

    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);
    const T* ya = static_cast<const T*>(A.ya);
    const T* yb = static_cast<const T*>(A.yb);

    T av[K][V], bv[K][V], yav[K][V], ybv[K][V];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if constexpr (SMEM) {
            const int off = k * kScanBlock * V + threadIdx.x * V;
            load_smem_chunk<V>(st.ya, off, yav[k]);
            if constexpr (W == 2) load_smem_chunk<V>(st.yb, off, ybv[k]);
            if constexpr (need_primal || !Op::kCoefOne) {
                load_smem_chunk<V>(st.a, off, av[k]);
                if constexpr (W == 2) load_smem_chunk<V>(st.b, off, bv[k]);
            }
        } else {
            const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
            load_chunk(ya, e, A.n, T(0), yav[k]);
            if constexpr (W == 2) load_chunk(yb, e, A.n, T(0), ybv[k]);
            if constexpr (need_primal || !Op::kCoefOne) {
                load_chunk(a, e, A.n, Op::pad_a(), av[k]);
                if constexpr (W == 2) load_chunk(b, e, A.n, T(0), bv[k]);
            }
        }
    }

    // ---- primal: exclusive prefix of every element (forward), from the carry
    P pex[K];  // thread's exclusive primal prefix per chunk
    if constexpr (need_primal) {
        if (threadIdx.x == 0) {
            if (A.carry) {
                s_carry = static_cast<const P*>(A.carry)[tile];
            } else {
                // the primal pass may still be running (batched launch): the
                // carry of this tile is the inclusive prefix the primal pass
                // publishes for the previous tile
                s_carry = Op::pid();
                if (tile > 0) {
                    constexpr int WP = lb_words<P>();
                    uint32_t it = 0;
                    while (!lb_read(A.lbP_incl + (tile - 1) * WP, 2u, s_carry)) {
                        if (++it > kSpinLimit || ((it & 255u) == 0 && gave_up(A.hdr))) {
                            record_status(A.hdr, ADPAR_ERR_TIMEOUT);
                            s_carry = Op::pid();
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
        }
        P agg[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            P acc = Op::pelem(av[k][0], W == 2 ? bv[k][0] : T(0));
#pragma unroll
            for (int j = 1; j < V; ++j) acc = Op::pcomb(acc, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
            agg[k] = acc;
        }
        auto pc = [](const P& l, const P& r) { return Op::pcomb(l, r); };
        P wex[K];
        (void)block_scan_part1<P, false, K, NW>(agg, wex, s_totP, Op::pid(), pc);
        __syncthreads();  // warp 0's exclusive totals (and s_carry) are visible
#pragma unroll
        for (int k = 0; k < K; ++k) pex[k] = block_scan_excl<P, false, K, NW>(k, wex, s_totP, s_carry, pc);
    }

    // ---- adjoint: lin_o elements, reverse scan with look-back
    T cf[K][V];
    L aggR[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        P cur = need_primal ? pex[k] : Op::pid();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            cf[k][j] = Op::kCoefOne ? T(1) : Op::coef(cur, av[k][j]);
            if constexpr (Op::kCoefNeedsPrimal) cur = Op::pcomb(cur, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
        }
        // fold the thread's V elements right to left (reverse scan order)
        L acc = L::id();
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {
            L el;
            if constexpr (!Op::kCoefOne) {
                el.c = cf[k][j];
                el.d[0] = cf[k][j] * yav[k][j];
                if constexpr (W == 2) el.d[1] = cf[k][j] * ybv[k][j];
            } else {
                el.d[0] = yav[k][j];
                if constexpr (W == 2) el.d[1] = ybv[k][j];
            }
            acc = L::comb(acc, el);
        }
        aggR[k] = acc;
    }
    auto lc = [](const L& e, const L& l) { return L::comb(e, l); };
    L wexR[K];
    L totR = block_scan_part1<L, true, K, NW>(aggR, wexR, s_totR, L::id(), lc);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<L> st{A.lbR_agg, A.lbR_incl};
        L pre = lookback(t_log, st, totR, L::id(), lc, A.hdr);
        if ((threadIdx.x & 31) == 0) s_prefR = pre;
    }
    __syncthreads();

    // ---- outputs: re-run both recurrences through the thread's elements
    T* abar = static_cast<T*>(A.abar);
    T* bbar = static_cast<T*>(A.bbar);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        if (e >= A.n) continue;
        L ex = block_scan_excl<L, true, K, NW>(k, wexR, s_totR, s_prefR, lc);
        P prev[V];
        {
            P cur = need_primal ? pex[k] : Op::pid();
#pragma unroll
            for (int j = 0; j < V; ++j) {
                prev[j] = cur;
                if (need_primal) cur = Op::pcomb(cur, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
            }
        }
        T oa[V], ob[V];
        T ua = ex.d[0];
        T ub = (W == 2) ? ex.d[W - 1] : T(0);
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {
            const T ra = yav[k][j] + ua;
            const T rb = (W == 2) ? ybv[k][j] + ub : T(0);
            T o1 = T(0), o2 = T(0);
            Op::vjp_right(prev[j], W == 2 || need_primal ? av[k][j] : T(0), T(0), ra, rb, o1, o2);
            oa[j] = o1;
            ob[j] = o2;
            ua = cf[k][j] * ra;
            if constexpr (W == 2) ub = cf[k][j] * rb;
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
        if constexpr (write_ys) {
            T y1[V], y2[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                P inc = Op::pcomb(prev[j], Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
                y1[j] = Op::out_a(inc);
                y2[j] = Op::out_b(inc);
            }
            store_chunk(static_cast<T*>(A.ys_a), e, A.n, y1);
            if constexpr (W == 2) store_chunk(static_cast<T*>(A.ys_b), e, A.n, y2);
        }
    }
}

// ------------------------------------------------------- primal forward scan
// The forward operator itself (ys = scan (.) as), used as the primal
// baseline of the VJP/primal time ratio.  One single pass with look-back.
template <class Op, class T, int K, int V>
__device__ __forceinline__ void scan_forward_tile(const ScanArgs& A, int64_t tile) {
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, TILE = K * kScanBlock * V;
    __shared__ P s_tot[K * NW];
    __shared__ P s_pref;
    const int64_t base = tile * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);

    T av[K][V], bv[K][V];
    P agg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        load_chunk(a, e, A.n, Op::pad_a(), av[k]);
        if constexpr (W == 2) load_chunk(b, e, A.n, T(0), bv[k]);
        P acc = Op::pelem(av[k][0], W == 2 ? bv[k][0] : T(0));
#pragma unroll
        for (int j = 1; j < V; ++j) acc = Op::pcomb(acc, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
        agg[k] = acc;
    }
    auto comb = [](const P& l, const P& r) { return Op::pcomb(l, r); };
    P wex[K];
    P total = block_scan_part1<P, false, K, NW>(agg, wex, s_tot, Op::pid(), comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<P> st{A.lbP_agg, A.lbP_incl};
        P pre = lookback(tile, st, total, Op::pid(), comb, A.hdr);
        if ((threadIdx.x & 31) == 0) s_pref = pre;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        if (e >= A.n) continue;
        P cur = block_scan_excl<P, false, K, NW>(k, wex, s_tot, s_pref, comb);
        T y1[V], y2[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            cur = Op::pcomb(cur, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
            y1[j] = Op::out_a(cur);
            y2[j] = Op::out_b(cur);
        }
        store_chunk(static_cast<T*>(A.ys_a), e, A.n, y1);
        if constexpr (W == 2) store_chunk(static_cast<T*>(A.ys_b), e, A.n, y2);
    }
}


}  // namespace adpar
