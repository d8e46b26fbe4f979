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

// E consecutive elements of a shared-memory array as 16-byte vectors
template <int E, class T>
__device__ __forceinline__ void load_chunk_smem(const T* p, int64_t off, T (&out)[E]) {
    constexpr int VV = Vec16<T>::N;
    static_assert(E % VV == 0, "whole vectors");
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
// Sec. 5.2 reads, in factored form: for each thread's run of kFacV elements,
// its local inclusive prefixes l_j = as_0 (.) ... (.) as_j (started from the
// neutral element; out_a and out_b stored per element) and the run's
// exclusive carry c, so that ys_j = c (.) l_j.  The return sweep then runs
// neither the primal fold nor the primal block scan, and out_a(l_j) is the
// product c_0 ... c_j of J_left factors its reverse aggregate needs.  This
// trades 2 W sizeof(T) bytes per element of traffic for about a third of the
// FP64 operations, which pays where FP64 arithmetic, not HBM, is the bound.
//
// Tiles of the return sweep are kScanBlock runs of kFacV = 16 elements; a
// run is handled in groups of kFacG = 4 so that few registers stay live.
constexpr int kFacV = 16;
constexpr int kFacG = 4;

// L2 policies for data that a tile reads twice: kept on the first read,
// dropped on the second
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_drop() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// E consecutive doubles at p + e (16-byte aligned) under an L2 policy; past
// n the values are `pad`
template <int E>
__device__ __forceinline__ void load_run_pol(const double* p, int64_t e, int64_t n, double pad, double (&out)[E],
                                             uint64_t pol) {
    static_assert(E % 2 == 0, "whole 16-byte vectors");
    if (e + E <= n) {
#pragma unroll
        for (int q = 0; q < E / 2; ++q)
            asm volatile("ld.global.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                         : "=d"(out[2 * q]), "=d"(out[2 * q + 1])
                         : "l"(p + e + 2 * q), "l"(pol));
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) out[j] = (e + j < n) ? p[e + j] : pad;
    }
}
// Primal pass: KC runs per thread (KC kFacV-runs of consecutive threads
// make one tile of KC * kScanBlock * kFacV elements); stores the local
// prefixes and each run's carry, indexed by the return sweep's tiles.
template <class Op, int KC>
__device__ __forceinline__ void scan_primal_fac_tile(const ScanArgs& A, int64_t tile) {
    using T = double;
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, V = kFacV, G = kFacG, TILE = KC * kScanBlock * V;
    static_assert(Op::kCoefIsA, "factored form is for J_left = a_i operators");
    __shared__ P s_tot[KC * NW];
    __shared__ P s_pre;
    const int64_t base = tile * TILE;
    const int64_t padded = A.tiles * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);
    T* la = static_cast<T*>(A.loc_a);
    T* lb = static_cast<T*>(A.loc_b);

    P agg[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        // the whole run is loaded before any of it is stored, so its loads
        // are all in flight at once
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        T av[V], bv[V];
        load_chunk_keep(a, e, A.n, Op::pad_a(), av);
        if constexpr (W == 2) load_chunk_keep(b, e, A.n, T(0), bv);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[j] = T(0);
        }
        P acc = Op::pelem(av[0], bv[0]);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (j > 0) acc = Op::pcomb(acc, Op::pelem(av[j], bv[j]));
            av[j] = Op::out_a(acc);  // the local prefix replaces the input
            bv[j] = Op::out_b(acc);
        }
        store_chunk(la, e, padded, av);
        if constexpr (W == 2) store_chunk(lb, e, padded, bv);
        agg[k] = acc;
    }
    auto comb = [](const P& l, const P& r) { return Op::pcomb(l, r); };
    P wex[KC];
    P total = block_scan_part1<P, false, KC, NW>(agg, wex, s_tot, Op::pid(), comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<P> st{A.lbP_agg, A.lbP_incl};
        P prefix = lookback(tile, st, total, Op::pid(), comb, A.hdr);
        if ((threadIdx.x & 31) == 0) s_pre = prefix;
    }
    __syncthreads();
    P* thc = static_cast<P*>(A.thr_carry);
#pragma unroll
    for (int k = 0; k < KC; ++k)
        thc[(tile * KC + k) * kScanBlock + threadIdx.x] = block_scan_excl<P, false, KC, NW>(k, wex, s_tot, s_pre, comb);
}

// The return sweep on the factored forward result, one kFacV-run per
// thread.  Phase 1 streams the run's local prefixes and cotangents to form
// its reverse aggregate  x -> sum_j out_a(l_j) ybar_j + out_a(l_last) x
// (loaded with a keep-in-L2 policy).  After the block
// scan and look-back, phase 2 re-reads the run from L2 in groups of kFacG,
// right to left: rs_bar_j = ybar_j + a_{j+1} rs_bar_{j+1}, and with
// rs_{j-1} = c (.) l_{j-1} (c itself for the run's first element) the
// adjoint J_right(j)^T rs_bar_j.  Same outputs as scan_adjoint_tile.
template <class Op, bool WYS>
__device__ __forceinline__ void scan_adjoint_fac_tile(const ScanArgs& A, int64_t t_log) {
    using T = double;
    using P = typename Op::P;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, V = kFacV, G = kFacG, TILE = kScanBlock * V;
    using L = Lin<T, W, true>;
    static_assert(Op::kCoefIsA, "factored form is for J_left = a_i operators");
    __shared__ L s_totR[NW];
    __shared__ L s_prefR;

    const int64_t tile = A.tiles - 1 - t_log;  // data tile (t_log counts from the right)
    const int64_t e0 = tile * TILE + threadIdx.x * V;
    const int64_t padded = A.tiles * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* ya = static_cast<const T*>(A.ya);
    const T* yb = static_cast<const T*>(A.yb);
    const T* la = static_cast<const T*>(A.loc_a);
    const T* lb = static_cast<const T*>(A.loc_b);
    const uint64_t keep = l2_policy_keep();

    // ---- phase 1: the run's reverse aggregate
    L agg[1];
#pragma unroll
    for (int i = 0; i < W; ++i) agg[0].d[i] = T(0);
#pragma unroll
    for (int g = 0; g < V / G; ++g) {
        T lv[G], y1[G], y2[G];
        load_run_pol(la, e0 + g * G, padded, T(0), lv, keep);
        load_run_pol(ya, e0 + g * G, A.n, T(0), y1, keep);
        if constexpr (W == 2) load_run_pol(yb, e0 + g * G, A.n, T(0), y2, keep);
#pragma unroll
        for (int j = 0; j < G; ++j) {
            agg[0].d[0] = fma(lv[j], y1[j], agg[0].d[0]);
            if constexpr (W == 2) agg[0].d[1] = fma(lv[j], y2[j], agg[0].d[1]);
        }
        if (g == V / G - 1) agg[0].c = lv[G - 1];
    }
    auto lc = [](const L& e, const L& l) { return L::comb(e, l); };
    L wexR[1];
    L totR = block_scan_part1<L, true, 1, NW>(agg, wexR, s_totR, L::id(), lc);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<L> st{A.lbR_agg, A.lbR_incl};
        L pre = lookback(t_log, st, totR, L::id(), lc, A.hdr);
        if ((threadIdx.x & 31) == 0) s_prefR = pre;
    }
    __syncthreads();
    if (e0 >= A.n) return;  // no barrier follows

    // ---- phase 2: outputs, groups right to left
    const uint64_t drop = l2_policy_drop();
    const L ex = block_scan_excl<L, true, 1, NW>(0, wexR, s_totR, s_prefR, lc);
    const P carry = static_cast<const P*>(A.thr_carry)[tile * kScanBlock + threadIdx.x];
    T* abar = static_cast<T*>(A.abar);
    T* bbar = static_cast<T*>(A.bbar);
    T a_up = T(1), r_upA = ex.d[0], r_upB = ex.d[W - 1];  // rs_bar of the run's right neighbour is ex.d
#pragma unroll
    for (int g = V / G - 1; g >= 0; --g) {
        const int64_t e = e0 + g * G;
        T av[G], y1[G], y2[G], lv[G], lw[G];
        load_run_pol(a, e, A.n, Op::pad_a(), av, drop);
        load_run_pol(ya, e, A.n, T(0), y1, drop);
        load_run_pol(la, e, padded, T(0), lv, drop);
        if constexpr (W == 2) {
            load_run_pol(yb, e, A.n, T(0), y2, drop);
            load_run_pol(lb, e, padded, T(0), lw, drop);
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j) y2[j] = lw[j] = T(0);
        }
        // l_{j-1} of the group's first element: the previous group's last
        T lpA = T(1), lpB = T(0);
        if (g > 0) {
            lpA = la[e - 1];
            if constexpr (W == 2) lpB = lb[e - 1];
        }
        // rs_bar, right to left (the run's last element adds the carry ex.d)
#pragma unroll
        for (int j = G - 1; j >= 0; --j) {
            if (g == V / G - 1 && j == G - 1) {
                y1[j] += r_upA;
                if constexpr (W == 2) y2[j] += r_upB;
            } else {
                const T c = j == G - 1 ? a_up : av[j + 1];
                y1[j] = fma(c, j == G - 1 ? r_upA : y1[j + 1], y1[j]);
                if constexpr (W == 2) y2[j] = fma(c, j == G - 1 ? r_upB : y2[j + 1], y2[j]);
            }
        }
        a_up = av[0];
        r_upA = y1[0];
        r_upB = y2[0];
        T o1v[G], ysa[G], ysb[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            P prev;
            if (g == 0 && j == 0) prev = carry;
            else if (j == 0) prev = Op::pcomb(carry, Op::pelem(lpA, lpB));
            else prev = Op::pcomb(carry, Op::pelem(lv[j - 1], lw[j - 1]));
            T o1 = T(0), o2 = T(0);
            Op::vjp_right(prev, av[j], T(0), y1[j], y2[j], o1, o2);
            o1v[j] = o1;
            if constexpr (WYS) {
                const P inc = Op::pcomb(carry, Op::pelem(lv[j], lw[j]));
                ysa[j] = Op::out_a(inc);
                ysb[j] = Op::out_b(inc);
            }
        }
        if (A.accumulate) {
            T old[G];
            load_chunk_keep(static_cast<const T*>(A.abar), e, A.n, T(0), old);
#pragma unroll
            for (int j = 0; j < G; ++j) o1v[j] += old[j];
            if constexpr (W == 2) {
                load_chunk_keep(static_cast<const T*>(A.bbar), e, A.n, T(0), old);
#pragma unroll
                for (int j = 0; j < G; ++j) y2[j] += old[j];
            }
        }
        store_chunk(abar, e, A.n, o1v);
        if constexpr (W == 2) store_chunk(bbar, e, A.n, y2);
        if constexpr (WYS) {
            store_chunk(static_cast<T*>(A.ys_a), e, A.n, ysa);
            if constexpr (W == 2) store_chunk(static_cast<T*>(A.ys_b), e, A.n, ysb);
        }
    }
}

// ----------------------------------------------------- forward mode (JVP)
// The tangent of ys = scan (.) as along asdot: one forward single-pass scan
// of dual elements (value, tangent) whose combine is (l (.) r, tcomb).  The
// tangent of the padding (and of the neutral element) is zero.
template <class Op>
struct DualState {
    typename Op::P v, t;
};

template <class Op, class T, int K, int V>
__device__ __forceinline__ void scan_jvp_tile(const ScanArgs& A, int64_t tile, const T* ad, const T* bd, T* yd_a,
                                              T* yd_b) {
    using D = DualState<Op>;
    constexpr int NW = kScanBlock / 32, W = Op::kWidth, TILE = K * kScanBlock * V;
    __shared__ D s_tot[K * NW];
    __shared__ D s_pref;
    const int64_t base = tile * TILE;
    const T* a = static_cast<const T*>(A.a);
    const T* b = static_cast<const T*>(A.b);

    T av[K][V], bv[K][V], tav[K][V], tbv[K][V];
    D agg[K];
    auto delem = [&](int k, int j) {
        return D{Op::pelem(av[k][j], W == 2 ? bv[k][j] : T(0)), Op::pelem(tav[k][j], W == 2 ? tbv[k][j] : T(0))};
    };
    auto comb = [](const D& l, const D& r) { return D{Op::pcomb(l.v, r.v), Op::tcomb(l.v, l.t, r.v, r.t)}; };
    const D ident{Op::pid(), Op::pelem(T(0), T(0))};
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        load_chunk(a, e, A.n, Op::pad_a(), av[k]);
        load_chunk(ad, e, A.n, T(0), tav[k]);
        if constexpr (W == 2) {
            load_chunk(b, e, A.n, T(0), bv[k]);
            load_chunk(bd, e, A.n, T(0), tbv[k]);
        }
        D acc = delem(k, 0);
#pragma unroll
        for (int j = 1; j < V; ++j) acc = comb(acc, delem(k, j));
        agg[k] = acc;
    }
    D wex[K];
    const D total = block_scan_part1<D, false, K, NW>(agg, wex, s_tot, ident, comb);
    if ((threadIdx.x >> 5) == 0) {
        // a dual state is two primal states: its aggregate and inclusive
        // slots take the primal and the adjoint slot regions
        LookbackState<D> st{A.lbP_agg, A.lbR_agg};
        const D pre = lookback(tile, st, total, ident, comb, A.hdr);
        if ((threadIdx.x & 31) == 0) s_pref = pre;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kScanBlock * V + threadIdx.x * V;
        if (e >= A.n) continue;
        D cur = block_scan_excl<D, false, K, NW>(k, wex, s_tot, s_pref, comb);
        T y1[V], y2[V], t1[V], t2[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            cur = comb(cur, delem(k, j));
            y1[j] = Op::out_a(cur.v);
            y2[j] = Op::out_b(cur.v);
            t1[j] = Op::out_a(cur.t);
            t2[j] = Op::out_b(cur.t);
        }
        if (A.ys_a) {
            store_chunk(static_cast<T*>(A.ys_a), e, A.n, y1);
            if constexpr (W == 2) store_chunk(static_cast<T*>(A.ys_b), e, A.n, y2);
        }
        store_chunk(yd_a, e, A.n, t1);
        if constexpr (W == 2) store_chunk(yd_b, e, A.n, t2);
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
