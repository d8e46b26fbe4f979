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
    // factored forward result (scan_primal_fac_tile): per element the
    // thread-local inclusive prefix (out_a, out_b) over the padded tiles,
    // per thread and chunk the exclusive carry; null on the other paths
    void* loc_a;      // [tiles * TILE] T
    void* loc_b;      // [tiles * TILE] T (width 2)
    void* thr_carry;  // [tiles * K * kScanBlock] P
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
template <class Op, class T, int K, int V, bool WYS>
__device__ __forceinline__ void scan_adjoint_tile(const ScanArgs& A, int64_t t_log) {
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
    static_assert(!Op::kCoefIsA || need_primal, "the J_left products come from the primal fold");

    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);
    const T* ya = static_cast<const T*>(A.ya);
    const T* yb = static_cast<const T*>(A.yb);

    T av[K][V], bv[K][V], yav[K][V], ybv[K][V];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        load_chunk(ya, e, A.n, T(0), yav[k]);
        if constexpr (W == 2) load_chunk(yb, e, A.n, T(0), ybv[k]);
        if constexpr (need_primal || !Op::kCoefOne) {
            load_chunk(a, e, A.n, Op::pad_a(), av[k]);
            if constexpr (W == 2) load_chunk(b, e, A.n, T(0), bv[k]);
        }
    }

    T cf[K][V];  // J_left factor of every element
    L aggR[K];   // the thread's lin_o aggregate per chunk (reverse order)

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
            if constexpr (Op::kCoefIsA) {
                // the reverse aggregate of the thread's run (see below):
                // x -> sum_j P_j ybar_j + P_last x, with P_j = c_0 ... c_j
                // the running product that this fold already forms
                T p = Op::out_a(acc);
                aggR[k].d[0] = p * yav[k][0];
                if constexpr (W == 2) aggR[k].d[1] = p * ybv[k][0];
            }
#pragma unroll
            for (int j = 1; j < V; ++j) {
                acc = Op::pcomb(acc, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
                if constexpr (Op::kCoefIsA) {
                    const T p = Op::out_a(acc);
                    aggR[k].d[0] = fma(p, yav[k][j], aggR[k].d[0]);
                    if constexpr (W == 2) aggR[k].d[1] = fma(p, ybv[k][j], aggR[k].d[1]);
                }
            }
            if constexpr (Op::kCoefIsA) aggR[k].c = Op::out_a(acc);
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
#pragma unroll
    for (int k = 0; k < K; ++k) {
        P cur = need_primal ? pex[k] : Op::pid();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            cf[k][j] = Op::kCoefOne ? T(1) : Op::coef(cur, av[k][j]);
            if constexpr (Op::kCoefNeedsPrimal) cur = Op::pcomb(cur, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
        }
        if constexpr (Op::kCoefIsA) continue;  // aggregate formed in the primal fold
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

    // ---- outputs: re-run both recurrences through the thread's elements.
    // Right to left, rs_bar_j = ybar_j + c_{j+1} rs_bar_{j+1} replaces ybar_j
    // in place; then left to right the primal prefix is re-formed and the
    // adjoint of every element replaces its input a_j (b's adjoint is
    // rs_bar's second component, already in place).
    T* abar = static_cast<T*>(A.abar);
    T* bbar = static_cast<T*>(A.bbar);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        if (e >= A.n) continue;
        const L ex = block_scan_excl<L, true, K, NW>(k, wexR, s_totR, s_prefR, lc);
        yav[k][V - 1] += ex.d[0];
        if constexpr (W == 2) ybv[k][V - 1] += ex.d[W - 1];
#pragma unroll
        for (int j = V - 1; j > 0; --j) {
            if constexpr (Op::kCoefOne) {
                yav[k][j - 1] += yav[k][j];
            } else {
                yav[k][j - 1] = fma(cf[k][j], yav[k][j], yav[k][j - 1]);
                if constexpr (W == 2) ybv[k][j - 1] = fma(cf[k][j], ybv[k][j], ybv[k][j - 1]);
            }
        }
        T y1[V], y2[V];
        P cur = need_primal ? pex[k] : Op::pid();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            T o1 = T(0), o2 = T(0);
            Op::vjp_right(cur, W == 2 || need_primal ? av[k][j] : T(0), T(0), yav[k][j],
                          W == 2 ? ybv[k][j] : T(0), o1, o2);
            if (need_primal) cur = Op::pcomb(cur, Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)));
            if constexpr (write_ys) {
                y1[j] = Op::out_a(cur);
                y2[j] = Op::out_b(cur);
            }
            av[k][j] = o1;
        }
        if (A.accumulate) {
            T old[V];
            load_chunk_keep(static_cast<const T*>(A.abar), e, A.n, T(0), old);
#pragma unroll
            for (int j = 0; j < V; ++j) av[k][j] += old[j];
            if constexpr (W == 2) {
                load_chunk_keep(static_cast<const T*>(A.bbar), e, A.n, T(0), old);
#pragma unroll
                for (int j = 0; j < V; ++j) ybv[k][j] += old[j];
            }
        }
        store_chunk(abar, e, A.n, av[k]);
        if constexpr (W == 2) store_chunk(bbar, e, A.n, ybv[k]);
        if constexpr (write_ys) {
            store_chunk(static_cast<T*>(A.ys_a), e, A.n, y1);
            if constexpr (W == 2) store_chunk(static_cast<T*>(A.ys_b), e, A.n, y2);
        }
    }
}

// ------------------------------------------ factored forward result (FP64)
// For operators whose J_left is the element's own a_i (kCoefIsA) the primal
// pass can hand the return sweep the forward scan result ys that the VJP of
// Sec. 5.2 reads, in factored form: for each thread and chunk, its local
// inclusive prefixes l_j = as_0 (.) ... (.) as_j of its V elements (started
// from the neutral element; out_a and out_b stored per element) and its
// exclusive carry c, so that ys_j = c (.) l_j.  The return sweep then runs
// neither the primal fold nor the primal block scan, and out_a(l_j) is the
// product c_0 ... c_j of J_left factors its reverse aggregate needs.  This
// trades 2 W sizeof(T) bytes per element of traffic for about a third of the
// FP64 operations, which pays where FP64 arithmetic, not HBM, is the bound.
template <class Op, class T, int K, int V>
__device__ __forceinline__ void scan_primal_fac_tile(const ScanArgs& A, int64_t tile) {
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, TILE = K * kScanBlock * V;
    static_assert(Op::kCoefIsA, "factored form is for J_left = a_i operators");
    __shared__ P s_tot[K * NW];
    __shared__ P s_pre;
    const int64_t base = tile * TILE;
    const int64_t padded = A.tiles * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);
    T* la = static_cast<T*>(A.loc_a);
    T* lb = static_cast<T*>(A.loc_b);

    P agg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        T av[V], bv[V], oa[V], ob[V];
        load_chunk_keep(a, e, A.n, Op::pad_a(), av);
        if constexpr (W == 2) load_chunk_keep(b, e, A.n, T(0), bv);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[j] = T(0);
        }
        P acc = Op::pelem(av[0], bv[0]);
        oa[0] = Op::out_a(acc);
        ob[0] = Op::out_b(acc);
#pragma unroll
        for (int j = 1; j < V; ++j) {
            acc = Op::pcomb(acc, Op::pelem(av[j], bv[j]));
            oa[j] = Op::out_a(acc);
            ob[j] = Op::out_b(acc);
        }
        store_chunk(la, e, padded, oa);
        if constexpr (W == 2) store_chunk(lb, e, padded, ob);
        agg[k] = acc;
    }
    auto comb = [](const P& l, const P& r) { return Op::pcomb(l, r); };
    P wex[K];
    P total = block_scan_part1<P, false, K, NW>(agg, wex, s_tot, Op::pid(), comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<P> st{A.lbP_agg, A.lbP_incl};
        P prefix = lookback(tile, st, total, Op::pid(), comb, A.hdr);
        if ((threadIdx.x & 31) == 0) s_pre = prefix;
    }
    __syncthreads();
    P* thc = static_cast<P*>(A.thr_carry);
#pragma unroll
    for (int k = 0; k < K; ++k)
        thc[(tile * K + k) * kScanBlock + threadIdx.x] = block_scan_excl<P, false, K, NW>(k, wex, s_tot, s_pre, comb);
}

// The return sweep on the factored forward result.  Per element it reads
// a_i (its J_left factor), ybar_i and the local prefix l_i; the reverse
// aggregate of a thread's run is x -> sum_j out_a(l_j) ybar_j + out_a(l_last) x,
// and rs_{i-1} = c (.) l_{i-1} (c itself for the run's first element) is
// what J_right(i)^T needs.  Same outputs as scan_adjoint_tile.
template <class Op, class T, int K, int V, bool WYS>
__device__ __forceinline__ void scan_adjoint_fac_tile(const ScanArgs& A, int64_t t_log) {
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, TILE = K * kScanBlock * V;
    using L = Lin<T, W, true>;
    static_assert(Op::kCoefIsA, "factored form is for J_left = a_i operators");
    __shared__ L s_totR[K * NW];
    __shared__ L s_prefR;

    const int64_t tile = A.tiles - 1 - t_log;  // data tile (t_log counts from the right)
    const int64_t base = tile * TILE;
    const int64_t padded = A.tiles * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* ya = static_cast<const T*>(A.ya);
    const T* yb = static_cast<const T*>(A.yb);
    const T* la = static_cast<const T*>(A.loc_a);
    const T* lb = static_cast<const T*>(A.loc_b);
    const P* thc = static_cast<const P*>(A.thr_carry);

    T av[K][V], yav[K][V], ybv[K][V], lav[K][V], lbv[K][V];
    P carry[K];
    L aggR[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        load_chunk(ya, e, A.n, T(0), yav[k]);
        if constexpr (W == 2) load_chunk(yb, e, A.n, T(0), ybv[k]);
        load_chunk(a, e, A.n, Op::pad_a(), av[k]);
        load_chunk(la, e, padded, T(0), lav[k]);
        if constexpr (W == 2) load_chunk(lb, e, padded, T(0), lbv[k]);
        carry[k] = thc[(tile * K + k) * kScanBlock + threadIdx.x];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        aggR[k].d[0] = lav[k][0] * yav[k][0];
        if constexpr (W == 2) aggR[k].d[1] = lav[k][0] * ybv[k][0];
#pragma unroll
        for (int j = 1; j < V; ++j) {
            aggR[k].d[0] = fma(lav[k][j], yav[k][j], aggR[k].d[0]);
            if constexpr (W == 2) aggR[k].d[1] = fma(lav[k][j], ybv[k][j], aggR[k].d[1]);
        }
        aggR[k].c = lav[k][V - 1];
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

    T* abar = static_cast<T*>(A.abar);
    T* bbar = static_cast<T*>(A.bbar);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        if (e >= A.n) continue;
        const L ex = block_scan_excl<L, true, K, NW>(k, wexR, s_totR, s_prefR, lc);
        yav[k][V - 1] += ex.d[0];
        if constexpr (W == 2) ybv[k][V - 1] += ex.d[W - 1];
#pragma unroll
        for (int j = V - 1; j > 0; --j) {
            yav[k][j - 1] = fma(av[k][j], yav[k][j], yav[k][j - 1]);
            if constexpr (W == 2) ybv[k][j - 1] = fma(av[k][j], ybv[k][j], ybv[k][j - 1]);
        }
        T y1[V], y2[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const P prev = j == 0 ? carry[k]
                                  : Op::pcomb(carry[k], Op::pelem(lav[k][j - 1], W == 2 ? lbv[k][j - 1] : T(0)));
            T o1 = T(0), o2 = T(0);
            Op::vjp_right(prev, av[k][j], T(0), yav[k][j], W == 2 ? ybv[k][j] : T(0), o1, o2);
            if constexpr (WYS) {
                const P inc = Op::pcomb(carry[k], Op::pelem(lav[k][j], W == 2 ? lbv[k][j] : T(0)));
                y1[j] = Op::out_a(inc);
                y2[j] = Op::out_b(inc);
            }
            av[k][j] = o1;
        }
        if (A.accumulate) {
            T old[V];
            load_chunk_keep(static_cast<const T*>(A.abar), e, A.n, T(0), old);
#pragma unroll
            for (int j = 0; j < V; ++j) av[k][j] += old[j];
            if constexpr (W == 2) {
                load_chunk_keep(static_cast<const T*>(A.bbar), e, A.n, T(0), old);
#pragma unroll
                for (int j = 0; j < V; ++j) ybv[k][j] += old[j];
            }
        }
        store_chunk(abar, e, A.n, av[k]);
        if constexpr (W == 2) store_chunk(bbar, e, A.n, ybv[k]);
        if constexpr (WYS) {
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
