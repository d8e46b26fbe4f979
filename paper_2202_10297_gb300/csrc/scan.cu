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

#include "scan_tiles.cuh"

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

// ------------------------------------------------------------ host side
struct ScanLayout {
    size_t off_carry, off_slots, off_pA, off_pI, off_rA, off_rI, slot_words, total_min;
    size_t off_loc_a, off_loc_b, off_thc, total;
};

// The FP64 operators with J_left = a_i take the factored forward result
// (scan_primal_fac_tile) when the workspace holds it.
template <class Op, class T>
constexpr bool kFactored = Op::kCoefIsA && sizeof(T) == 8;

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
    if (need_primal) scan_primal_kernel<Op, T><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    if (ys_a) scan_adjoint_kernel<Op, T, true><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
    else scan_adjoint_kernel<Op, T, false><<<(unsigned)A.tiles, kScanBlock, 0, stream>>>(A);
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

template <class T>
int dispatch_scan_jvp(int op, int64_t n, const void* a, const void* b, const void* ad, const void* bd, void* ys_a,
                      void* ys_b, void* yd_a, void* yd_b, void* work, size_t work_bytes, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD: return run_scan_jvp<OpAdd<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_MUL: return run_scan_jvp<OpMul<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_MIN: return run_scan_jvp<OpMin<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_MAX: return run_scan_jvp<OpMax<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    case ADPAR_OP_LINREC:
        return run_scan_jvp<OpLinrec<T>, T>(n, a, b, ad, bd, ys_a, ys_b, yd_a, yd_b, work, work_bytes, s);
    }
    return ADPAR_ERR_INVALID;
}

// ------------------------------------------- reduce, general rule (Sec. 5.1.1)
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
