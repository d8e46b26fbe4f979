// VJP of a scan over vectors with an elementwise operator (Sec. 5.2, the
// vectorised case): xs is row-major [n][d] and
//   scan (map (.)) e xs == transpose xs |> map (scan (.) e) |> transpose,
// i.e. d independent scans down the columns.  No transpose is materialised:
// a thread owns one column and one chunk of kVecR rows, so a warp's loads
// cover 32 consecutive columns of a row (coalesced).  Five kernels, no
// block waits on another:
//   1. per (chunk, column): the aggregate of the operator's state;
//   2. per column, one warp scans the chunk aggregates (exclusive carries);
//   3. per (chunk, column): the aggregate of the return sweep's lin_o state
//      (MIN/MAX re-form the primal prefix from the carry for J_left);
//   4. per column, one warp scans those right to left (exclusive carries);
//   5. per (chunk, column): a backward sweep of rs_bar_r = ybar_r +
//      c_{r+1} rs_bar_{r+1} into shared memory, then a forward sweep with
//      the primal prefix writing as_bar = J_right^T rs_bar.
#include <algorithm>

#include "scan_tiles.cuh"

namespace adpar {
namespace {

constexpr int kVecBlock = 256;
constexpr int kVecOutBlock = 64;  // the output pass keeps 32 rows x width of rs_bar per thread in shared memory
constexpr int kVecR = 32;         // rows per chunk (the J_left bits of a chunk fit one word)

// operators whose return sweep reads the primal (the input a)
template <class Op>
constexpr bool kVecPrimal = Op::kNeedPrimal || Op::kCoefNeedsPrimal || !Op::kCoefOne;

struct VecArgs {
    int64_t n, d, C;  // rows, columns, chunks
    const void* a;
    const void* b;
    const void* ya;
    const void* yb;
    void* abar;
    void* bbar;
    int accumulate;
    void* aggP;  // [C][d] P: chunk aggregates, then exclusive prefixes
    void* aggL;  // [C][d] L: chunk aggregates, then exclusive suffixes
};

template <class Op, class T>
__device__ __forceinline__ typename Op::P vec_elem(const VecArgs& V, int64_t i) {
    return Op::pelem(__ldg(static_cast<const T*>(V.a) + i),
                     Op::kWidth == 2 ? __ldg(static_cast<const T*>(V.b) + i) : T(0));
}

template <class Op, class T>
__global__ void __launch_bounds__(kVecBlock) vec_primal_agg_kernel(VecArgs V) {
    using P = typename Op::P;
    const int64_t col = blockIdx.x * (int64_t)kVecBlock + threadIdx.x, c = blockIdx.y;
    if (col >= V.d) return;
    const int64_t r0 = c * kVecR, r1 = std::min<int64_t>(V.n, r0 + kVecR);
    P acc = Op::pid();
    for (int64_t r = r0; r < r1; ++r) acc = Op::pcomb(acc, vec_elem<Op, T>(V, r * V.d + col));
    static_cast<P*>(V.aggP)[c * V.d + col] = acc;
}

// One warp per column turns the column's C chunk aggregates into exclusive
// prefixes (REV: exclusive suffixes, composed right to left), 32 chunks per
// round with a shuffle scan and a carry between rounds.
template <class S, bool REV, class Comb>
__device__ __forceinline__ void vec_scan_column(S* agg, int64_t C, int64_t d, int64_t col, const S& ident,
                                                Comb comb) {
    const int lane = threadIdx.x & 31;
    S carry = ident;
    for (int64_t base = 0; base < C; base += 32) {
        const int64_t q = REV ? C - 1 - (base + lane) : base + lane;  // chunk of this lane
        const bool ok = base + lane < C;
        S v = ok ? agg[q * d + col] : ident;
        S inc = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const S o = shfl_up_s(inc, off);
            if (lane >= off) inc = comb(o, inc);
        }
        S ex = shfl_up_s(inc, 1);
        if (lane == 0) ex = ident;
        if (ok) agg[q * d + col] = comb(carry, ex);
        carry = comb(carry, shfl_idx_s(inc, 31));
    }
}

template <class Op, class T>
__global__ void vec_scan_P_kernel(VecArgs V) {
    using P = typename Op::P;
    const int64_t col = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (col >= V.d) return;  // whole warps leave together
    vec_scan_column<P, false>(static_cast<P*>(V.aggP), V.C, V.d, col, Op::pid(),
                              [](const P& l, const P& r) { return Op::pcomb(l, r); });
}

template <class Op, class T>
__global__ void vec_scan_L_kernel(VecArgs V) {
    using L = Lin<T, Op::kWidth, !Op::kCoefOne>;
    const int64_t col = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (col >= V.d) return;
    // scan order is right to left: e holds later rows, l earlier ones
    vec_scan_column<L, true>(static_cast<L*>(V.aggL), V.C, V.d, col, L::id(),
                             [](const L& e, const L& l) { return L::comb(e, l); });
}

// J_left of the chunk's rows as bits (MIN/MAX: needs the primal prefix)
template <class Op, class T>
__device__ __forceinline__ uint32_t vec_coef_bits(const VecArgs& V, int64_t col, int64_t r0, int64_t r1,
                                                  const typename Op::P& carry) {
    uint32_t bits = 0u;
    typename Op::P cur = carry;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * V.d + col;
        const T a = __ldg(static_cast<const T*>(V.a) + i);
        if (Op::coef(cur, a) != T(0)) bits |= 1u << (r - r0);
        cur = Op::pcomb(cur, vec_elem<Op, T>(V, i));
    }
    return bits;
}

template <class Op, class T>
__device__ __forceinline__ T vec_coef(const VecArgs& V, int64_t i, uint32_t bits, int64_t rr) {
    if constexpr (Op::kCoefOne) return T(1);
    else if constexpr (Op::kCoefNeedsPrimal) return ((bits >> rr) & 1u) ? T(1) : T(0);
    else return Op::coef(Op::pid(), __ldg(static_cast<const T*>(V.a) + i));
}

template <class Op, class T>
__global__ void __launch_bounds__(kVecBlock) vec_adjoint_agg_kernel(VecArgs V) {
    using P = typename Op::P;
    constexpr int W = Op::kWidth;
    using L = Lin<T, W, !Op::kCoefOne>;
    const int64_t col = blockIdx.x * (int64_t)kVecBlock + threadIdx.x, c = blockIdx.y;
    if (col >= V.d) return;
    const int64_t r0 = c * kVecR, r1 = std::min<int64_t>(V.n, r0 + kVecR);
    uint32_t bits = 0u;
    if constexpr (Op::kCoefNeedsPrimal)
        bits = vec_coef_bits<Op, T>(V, col, r0, r1, static_cast<const P*>(V.aggP)[c * V.d + col]);
    // x -> c_r (ybar_r + x) folded over the rows, bottom to top
    L acc = L::id();
    for (int64_t r = r1 - 1; r >= r0; --r) {
        const int64_t i = r * V.d + col;
        L el;
        const T y1 = __ldg(static_cast<const T*>(V.ya) + i);
        const T y2 = W == 2 ? __ldg(static_cast<const T*>(V.yb) + i) : T(0);
        if constexpr (!Op::kCoefOne) {
            const T cr = vec_coef<Op, T>(V, i, bits, r - r0);
            el.c = cr;
            el.d[0] = cr * y1;
            if constexpr (W == 2) el.d[1] = cr * y2;
        } else {
            el.d[0] = y1;
            if constexpr (W == 2) el.d[1] = y2;
        }
        acc = L::comb(acc, el);
    }
    static_cast<L*>(V.aggL)[c * V.d + col] = acc;
}

template <class Op, class T>
__global__ void __launch_bounds__(kVecOutBlock) vec_output_kernel(VecArgs V) {
    using P = typename Op::P;
    constexpr int W = Op::kWidth;
    constexpr bool kP = kVecPrimal<Op>;
    using L = Lin<T, W, !Op::kCoefOne>;
    __shared__ T s_r[kVecR * W * kVecOutBlock];  // rs_bar of the thread's rows, [row][component][thread]
    const int64_t col = blockIdx.x * (int64_t)kVecOutBlock + threadIdx.x, c = blockIdx.y;
    if (col >= V.d) return;
    const int64_t r0 = c * kVecR, r1 = std::min<int64_t>(V.n, r0 + kVecR);
    const P carry = kP ? static_cast<const P*>(V.aggP)[c * V.d + col] : Op::pid();
    const L suf = static_cast<const L*>(V.aggL)[c * V.d + col];
    uint32_t bits = 0u;
    if constexpr (Op::kCoefNeedsPrimal) bits = vec_coef_bits<Op, T>(V, col, r0, r1, carry);
    // backward: rs_bar of the last row gets the chunks below through suf.d
    T ra = T(0), rb = T(0);
    for (int64_t r = r1 - 1; r >= r0; --r) {
        const int64_t i = r * V.d + col;
        const T y1 = __ldg(static_cast<const T*>(V.ya) + i);
        const T y2 = W == 2 ? __ldg(static_cast<const T*>(V.yb) + i) : T(0);
        if (r == r1 - 1) {
            ra = y1 + suf.d[0];
            if constexpr (W == 2) rb = y2 + suf.d[W - 1];
        } else {
            const T cn = vec_coef<Op, T>(V, i + V.d, bits, r + 1 - r0);  // J_left of the row below
            ra = fma(cn, ra, y1);
            if constexpr (W == 2) rb = fma(cn, rb, y2);
        }
        s_r[((r - r0) * W) * kVecOutBlock + threadIdx.x] = ra;
        if constexpr (W == 2) s_r[((r - r0) * W + 1) * kVecOutBlock + threadIdx.x] = rb;
    }
    // forward: the primal prefix and the adjoints
    T* abar = static_cast<T*>(V.abar);
    T* bbar = static_cast<T*>(V.bbar);
    P prev = carry;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * V.d + col;
        T av = T(0), bv = T(0);
        if constexpr (kP) {
            av = __ldg(static_cast<const T*>(V.a) + i);
            if constexpr (W == 2) bv = __ldg(static_cast<const T*>(V.b) + i);
        }
        const T q1 = s_r[((r - r0) * W) * kVecOutBlock + threadIdx.x];
        const T q2 = W == 2 ? s_r[((r - r0) * W + 1) * kVecOutBlock + threadIdx.x] : T(0);
        T o1 = T(0), o2 = T(0);
        Op::vjp_right(prev, av, bv, q1, q2, o1, o2);
        if constexpr (kP) prev = Op::pcomb(prev, Op::pelem(av, bv));
        if (V.accumulate) {
            abar[i] += o1;
            if constexpr (W == 2) bbar[i] += o2;
        } else {
            abar[i] = o1;
            if constexpr (W == 2) bbar[i] = o2;
        }
    }
}

template <class Op, class T>
size_t vec_workspace(int64_t n, int64_t d) {
    using L = Lin<T, Op::kWidth, !Op::kCoefOne>;
    const int64_t C = (n + kVecR - 1) / kVecR;
    return sizeof(WsHeader) + round_up((size_t)C * d * sizeof(typename Op::P), 256) +
           round_up((size_t)C * d * sizeof(L), 256);
}

template <class Op, class T>
int run_vec(int64_t n, int64_t d, const void* a, const void* b, const void* ya, const void* yb, void* abar,
            void* bbar, uint32_t flags, void* work, size_t work_bytes, cudaStream_t s) {
    using L = Lin<T, Op::kWidth, !Op::kCoefOne>;
    const size_t need = vec_workspace<Op, T>(n, d);
    if (!work || work_bytes < need || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    if (n == 0 || d == 0) return ADPAR_OK;
    VecArgs V{};
    V.n = n; V.d = d; V.C = (n + kVecR - 1) / kVecR;
    V.a = a; V.b = b; V.ya = ya; V.yb = yb; V.abar = abar; V.bbar = bbar;
    V.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    char* w = static_cast<char*>(work);
    cudaMemsetAsync(w, 0, sizeof(WsHeader), s);  // the status word starts at ok
    V.aggP = w + sizeof(WsHeader);
    V.aggL = w + sizeof(WsHeader) + round_up((size_t)V.C * d * sizeof(typename Op::P), 256);
    const dim3 g2((unsigned)((d + kVecBlock - 1) / kVecBlock), (unsigned)V.C);
    const dim3 g5((unsigned)((d + kVecOutBlock - 1) / kVecOutBlock), (unsigned)V.C);
    const unsigned gw = (unsigned)((d + 7) / 8);  // 8 warps (columns) per block
    if constexpr (kVecPrimal<Op>) {
        vec_primal_agg_kernel<Op, T><<<g2, kVecBlock, 0, s>>>(V);
        vec_scan_P_kernel<Op, T><<<gw, 256, 0, s>>>(V);
    }
    vec_adjoint_agg_kernel<Op, T><<<g2, kVecBlock, 0, s>>>(V);
    vec_scan_L_kernel<Op, T><<<gw, 256, 0, s>>>(V);
    vec_output_kernel<Op, T><<<g5, kVecOutBlock, 0, s>>>(V);
    (void)sizeof(L);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T>
int dispatch_vec(int op, int64_t n, int64_t d, const void* a, const void* b, const void* ya, const void* yb,
                 void* abar, void* bbar, uint32_t flags, void* work, size_t work_bytes, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD: return run_vec<OpAdd<T>, T>(n, d, a, b, ya, yb, abar, bbar, flags, work, work_bytes, s);
    case ADPAR_OP_MUL: return run_vec<OpMul<T>, T>(n, d, a, b, ya, yb, abar, bbar, flags, work, work_bytes, s);
    case ADPAR_OP_MIN: return run_vec<OpMin<T>, T>(n, d, a, b, ya, yb, abar, bbar, flags, work, work_bytes, s);
    case ADPAR_OP_MAX: return run_vec<OpMax<T>, T>(n, d, a, b, ya, yb, abar, bbar, flags, work, work_bytes, s);
    case ADPAR_OP_LINREC:
        return run_vec<OpLinrec<T>, T>(n, d, a, b, ya, yb, abar, bbar, flags, work, work_bytes, s);
    }
    return ADPAR_ERR_INVALID;
}

template <class T>
size_t vec_ws_bytes(int op, int64_t n, int64_t d) {
    switch (op) {
    case ADPAR_OP_ADD: return vec_workspace<OpAdd<T>, T>(n, d);
    case ADPAR_OP_MUL: return vec_workspace<OpMul<T>, T>(n, d);
    case ADPAR_OP_MIN: return vec_workspace<OpMin<T>, T>(n, d);
    case ADPAR_OP_MAX: return vec_workspace<OpMax<T>, T>(n, d);
    case ADPAR_OP_LINREC: return vec_workspace<OpLinrec<T>, T>(n, d);
    }
    return (size_t)-1;
}

}  // namespace

size_t scan_vec_workspace_size(adpar_opdesc desc, int64_t n, int64_t d) {
    if (n < 0 || d < 0) return (size_t)-1;
    if (desc.dtype == ADPAR_F32) return vec_ws_bytes<float>(desc.op, n, d);
    if (desc.dtype == ADPAR_F64) return vec_ws_bytes<double>(desc.op, n, d);
    return (size_t)-1;
}

}  // namespace adpar

extern "C" int adpar_vjp_scan_vec(adpar_opdesc desc, int64_t n, int64_t d, const void* a, const void* b,
                                  const void* ybar_a, const void* ybar_b, void* abar, void* bbar, uint32_t flags,
                                  void* work, size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0 || d < 0) return ADPAR_ERR_INVALID;
    if (desc.op < ADPAR_OP_ADD || desc.op > ADPAR_OP_LINREC) return ADPAR_ERR_INVALID;
    if (desc.dtype != ADPAR_F32 && desc.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    const int want_w = desc.op == ADPAR_OP_LINREC ? 2 : 1;
    if (desc.width != want_w) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    if (n > 0 && d > 0) {
        if (!ybar_a || !abar) return ADPAR_ERR_INVALID;
        if (desc.op != ADPAR_OP_ADD && !a) return ADPAR_ERR_INVALID;
        if (want_w == 2 && (!b || !ybar_b || !bbar)) return ADPAR_ERR_INVALID;
        const void* ptrs[] = {a, b, ybar_a, ybar_b, abar, bbar};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    if (n > 0 && d > ((int64_t)1 << 31) / kVecBlock * kVecBlock) return ADPAR_ERR_UNSUPPORTED;  // grid x
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (desc.dtype == ADPAR_F32)
        return dispatch_vec<float>(desc.op, n, d, a, b, ybar_a, ybar_b, abar, bbar, flags, work, work_bytes, s);
    return dispatch_vec<double>(desc.op, n, d, a, b, ybar_a, ybar_b, abar, bbar, flags, work, work_bytes, s);
}
