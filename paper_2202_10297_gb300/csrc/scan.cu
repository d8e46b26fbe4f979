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

#include "scan_engine.cuh"
#include "scan_ops.cuh"

namespace adpar {
namespace {

constexpr int kScanBlock = 256;

// Tile shape: K chunks of kScanBlock * E elements; in each chunk a thread
// owns E consecutive elements (kept in registers).  Larger E amortises the
// warp-shuffle scans over more elements, which matters where arithmetic,
// not memory, bounds the kernel (FP64 on GB300).
template <class Op, class T>
struct ScanCfg {
    static constexpr bool kF64 = sizeof(T) == 8;
    static constexpr int E = kF64 ? (Op::kWidth == 2 ? 8 : 4) : 4;
    static constexpr int K = kF64 ? (Op::kWidth == 2 ? 1 : 4) : (Op::kWidth == 2 ? 4 : 8);
    static constexpr int V = E;
    static constexpr int TILE = K * kScanBlock * E;
};

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

// Zeroes the header and the look-back slots (one contiguous region).
__global__ void scan_init_kernel(WsHeader* hdr, unsigned long long* slots, int64_t nwords) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i < 64) reinterpret_cast<uint32_t*>(hdr)[i] = 0u;
    for (int64_t t = i; t < nwords; t += stride) slots[t] = 0ull;
}

// ---------------------------------------------------------------- pass P
template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_primal_kernel(ScanArgs A) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    constexpr int K = Cfg::K, V = Cfg::V, NW = kScanBlock / 32;
    __shared__ P s_tot[K * NW];
    __shared__ uint32_t s_tile;

    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * Cfg::TILE;
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
        if ((threadIdx.x & 31) == 0) static_cast<P*>(A.carry)[tile] = prefix;
    }
}

// ---------------------------------------------------------------- pass R
template <class Op, class T, bool WYS>
__global__ void __launch_bounds__(kScanBlock) scan_adjoint_kernel(ScanArgs A) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    constexpr int K = Cfg::K, V = Cfg::V, NW = kScanBlock / 32, W = Op::kWidth;
    using L = Lin<T, W, !Op::kCoefOne>;
    constexpr bool kPrimal = Op::kNeedPrimal || Op::kCoefNeedsPrimal;

    __shared__ P s_totP[K * NW];
    __shared__ L s_totR[K * NW];
    __shared__ P s_carry;
    __shared__ L s_prefR;
    __shared__ uint32_t s_tile;

    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;             // logical tile in reverse scan order
    const int64_t tile = A.tiles - 1 - t_log;  // data tile
    const int64_t base = tile * Cfg::TILE;
    constexpr bool write_ys = WYS;
    constexpr bool need_primal = kPrimal || WYS;

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

    // ---- primal: exclusive prefix of every element (forward), from the carry
    P pex[K];  // thread's exclusive primal prefix per chunk
    if constexpr (need_primal) {
        if (threadIdx.x == 0) s_carry = static_cast<const P*>(A.carry)[tile];
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
template <class Op, class T>
__global__ void __launch_bounds__(kScanBlock) scan_forward_kernel(ScanArgs A) {
    using Cfg = ScanCfg<Op, T>;
    using P = typename Op::P;
    constexpr int K = Cfg::K, V = Cfg::V, NW = kScanBlock / 32, W = Op::kWidth;
    __shared__ P s_tot[K * NW];
    __shared__ P s_pref;
    __shared__ uint32_t s_tile;

    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * Cfg::TILE;
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

// ------------------------------------------------------------ host side
struct ScanLayout {
    size_t off_carry, off_slots, off_pA, off_pI, off_rA, off_rI, slot_words, total;
};

// header | carry[tiles] | look-back slots (primal agg, primal incl,
// adjoint agg, adjoint incl), the slots contiguous so one kernel zeroes them
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
    s.total = round_up(o, 256);
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

template <class Op, class T>
int run_scan(int64_t n, const void* a, const void* b, const void* ya, const void* yb, void* abar,
             void* bbar, void* ys_a, void* ys_b, uint32_t flags, void* work, size_t work_bytes,
             cudaStream_t stream) {
    using Cfg = ScanCfg<Op, T>;
    const ScanLayout L = scan_layout<Op, T>(n);
    if (work == nullptr || work_bytes < L.total || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) return ADPAR_OK;
    char* w = static_cast<char*>(work);
    ScanArgs A;
    A.n = n;
    A.a = a; A.b = b; A.ya = ya; A.yb = yb;
    A.abar = abar; A.bbar = bbar; A.ys_a = ys_a; A.ys_b = ys_b;
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    A.tiles = (n + Cfg::TILE - 1) / Cfg::TILE;
    A.hdr = reinterpret_cast<WsHeader*>(w);
    set_slots(A, w, L);
    const bool need_primal = Op::kNeedPrimal || Op::kCoefNeedsPrimal || ys_a != nullptr;
    launch_init(A, w, L, stream);
    if (need_primal) scan_primal_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    if (ys_a) scan_adjoint_kernel<Op, T, true><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    else scan_adjoint_kernel<Op, T, false><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T>
size_t scan_ws_bytes(int op, int64_t n) {
    switch (op) {
    case ADPAR_OP_ADD: return scan_layout<OpAdd<T>, T>(n).total;
    case ADPAR_OP_MUL: return scan_layout<OpMul<T>, T>(n).total;
    case ADPAR_OP_MIN: return scan_layout<OpMin<T>, T>(n).total;
    case ADPAR_OP_MAX: return scan_layout<OpMax<T>, T>(n).total;
    case ADPAR_OP_LINREC: return scan_layout<OpLinrec<T>, T>(n).total;
    }
    return (size_t)-1;
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
    if (work == nullptr || work_bytes < L.total || (reinterpret_cast<uintptr_t>(work) & 255u))
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

}  // namespace

size_t scan_workspace_size(adpar_opdesc d, int64_t n) {
    if (n < 0) return (size_t)-1;
    if (d.dtype == ADPAR_F32) return scan_ws_bytes<float>(d.op, n);
    if (d.dtype == ADPAR_F64) return scan_ws_bytes<double>(d.op, n);
    return (size_t)-1;
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
