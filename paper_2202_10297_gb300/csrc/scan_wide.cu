// Scan VJP over elements of D scalars with the general lin_o of Sec. 5.2:
// any element type is a vector of D scalars, J_left and J_right are D x D
// matrices, and the return sweep's recurrence
//   rs_bar_i = ybar_i + J_left(i+1)^T rs_bar_{i+1}
// is a reverse scan of affine maps x -> d + C x (d a D-vector, C a D x D
// matrix), whose combine multiplies two matrices:
//   lin_o (d1, C1) (d2, C2) = (d1 + C1 d2, C1 C2)   (1 earlier, 2 later)
// with neutral element (0, I).  Then as_bar_i = J_right(i)^T rs_bar_i for
// i >= 1 and as_bar_0 = rs_bar_0.
//
// Layout: the element i is the row [i*D, (i+1)*D) of a row-major [n][D]
// array; a thread owns two consecutive rows, so its loads are whole 16-byte
// vectors.  Two single-pass look-back kernels: the forward pass keeps each
// tile's primal carry (and writes ys when asked); the reverse pass re-forms
// the primal inside the tile from that carry, forms (ybar_i, J_left(i+1)^T)
// per element, scans the affine maps right to left and applies J_right^T.
// Where J_left acts alike on blocks of the element (the matrix recurrence:
// M on both columns of the matrix part and on the vector part), C stays
// I (x) N with a small N, and that lin_o (LinBlock) replaces the full one
// (LinFull) unless ADPAR_FULL_LIN_O asks for it.
#include <type_traits>

#include "common.cuh"
#include "scan_engine.cuh"

namespace adpar {
namespace {

constexpr int kWideBlock = 256;
constexpr int kWideV = 2;  // rows per thread
constexpr int kWideTile = kWideBlock * kWideV;

template <class T, int D>
struct WState {
    T v[D];
};

// x -> d + C x
template <class T, int D>
struct WLin {
    T d[D];
    T c[D][D];
};

// Linear recurrence as a width-2 element (a, b): (a1,b1) (.) (a2,b2) =
// (a2 a1, a2 b1 + b2);  J_left = a2 I;  J_right = [[A, 0], [B, 1]].
template <class T>
struct WLinrec {
    static constexpr int D = 2;
    using S = WState<T, 2>;
    __device__ static S id() { return S{{T(1), T(0)}}; }
    __device__ static S comb(const S& l, const S& r) { return S{{r.v[0] * l.v[0], fma(r.v[0], l.v[1], r.v[1])}}; }
    // J_left(prev, x): rows the output components, columns prev's
    __device__ static void jleft(const S&, const S& x, T (&J)[D][D]) {
        J[0][0] = x.v[0]; J[0][1] = T(0);
        J[1][0] = T(0);   J[1][1] = x.v[0];
    }
    // J_right(prev, x)^T g
    __device__ static void vjp_right(const S& prev, const S&, const T (&g)[D], T (&o)[D]) {
        o[0] = fma(prev.v[0], g[0], prev.v[1] * g[1]);
        o[1] = g[1];
    }
};

// 2x2 matrix linear recurrence: an element is (M, v) with M row-major in
// v[0..3] and the vector in v[4..5]; (M1, v1) (.) (M2, v2) = (M2 M1,
// M2 v1 + v2), i.e. the affine maps h -> M h + v composed in scan order.
// out P[j][k] = sum_m X[j][m] P[m][k];  out h[j] = sum_m X[j][m] h[m] + xv[j].
template <class T>
struct WMatrec2 {
    static constexpr int D = 6;
    using S = WState<T, 6>;
    __device__ static S id() { return S{{T(1), T(0), T(0), T(1), T(0), T(0)}}; }
    __device__ static S comb(const S& l, const S& r) {
        S o;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int k = 0; k < 2; ++k) o.v[2 * j + k] = fma(r.v[2 * j], l.v[k], r.v[2 * j + 1] * l.v[2 + k]);
            o.v[4 + j] = fma(r.v[2 * j], l.v[4], fma(r.v[2 * j + 1], l.v[5], r.v[4 + j]));
        }
        return o;
    }
    __device__ static void jleft(const S&, const S& x, T (&J)[D][D]) {
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) J[r][c] = T(0);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int m = 0; m < 2; ++m) {
#pragma unroll
                for (int k = 0; k < 2; ++k) J[2 * j + k][2 * m + k] = x.v[2 * j + m];
                J[4 + j][4 + m] = x.v[2 * j + m];
            }
    }
    // J_left = I_3 (x) M on three 2-vectors: block j < 2 is column j of the
    // matrix part (components j, 2 + j), block 2 the vector part (4, 5)
    static constexpr int kB = 2;
    __device__ static int blk(int j, int i) { return j < 2 ? 2 * i + j : 4 + i; }
    __device__ static T block_m(const S& x, int r, int m) { return x.v[2 * r + m]; }
    __device__ static void vjp_right(const S& prev, const S&, const T (&g)[D], T (&o)[D]) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int m = 0; m < 2; ++m)
                o[2 * j + m] = fma(g[2 * j], prev.v[2 * m], fma(g[2 * j + 1], prev.v[2 * m + 1], g[4 + j] * prev.v[4 + m]));
            o[4 + j] = g[4 + j];
        }
    }
};

template <class T, int D>
__device__ __forceinline__ WLin<T, D> wlin_id() {
    WLin<T, D> r;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        r.d[i] = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) r.c[i][j] = i == j ? T(1) : T(0);
    }
    return r;
}

// e holds later elements, l earlier ones: x -> l.d + l.c (e.d + e.c x)
template <class T, int D>
__device__ __forceinline__ WLin<T, D> wlin_comb(const WLin<T, D>& e, const WLin<T, D>& l) {
    WLin<T, D> r;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = l.d[i];
#pragma unroll
        for (int k = 0; k < D; ++k) s = fma(l.c[i][k], e.d[k], s);
        r.d[i] = s;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T t = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) t = fma(l.c[i][k], e.c[k][j], t);
            r.c[i][j] = t;
        }
    }
    return r;
}

// The return sweep's lin_o, in full: C = J_left^T as a D x D matrix.
template <class Op, class T>
struct LinFull {
    static constexpr int D = Op::D;
    using S = typename Op::S;
    using L = WLin<T, D>;
    __device__ static L id() { return wlin_id<T, D>(); }
    __device__ static L comb(const L& later, const L& earlier) { return wlin_comb<T, D>(later, earlier); }
    // (ybar_i, J_left(i+1)^T) from rs_i and a_{i+1}
    __device__ static L elem(const S& prev, const S& xn, const S& y) {
        L el;
        T J[D][D];
        Op::jleft(prev, xn, J);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            el.d[i] = y.v[i];
#pragma unroll
            for (int j = 0; j < D; ++j) el.c[i][j] = J[j][i];
        }
        return el;
    }
    // o = el.d + el.C g
    __device__ static void apply(const L& el, const T (&g)[D], T (&o)[D]) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T s = el.d[i];
#pragma unroll
            for (int k = 0; k < D; ++k) s = fma(el.c[i][k], g[k], s);
            o[i] = s;
        }
    }
};

// The same lin_o when J_left = I (x) M acts alike on D / B blocks of B
// components (Op::blk), so C = I (x) N with N = M^T a B x B matrix and the
// maps compose blockwise: (d1, N1) after (d2, N2) = (d1 + N1 d2, N1 N2).
template <class T, int D, int B>
struct WLinB {
    T d[D];
    T n[B][B];
};

template <class Op, class T>
struct LinBlock {
    static constexpr int D = Op::D, B = Op::kB, NB = D / B;
    using S = typename Op::S;
    using L = WLinB<T, D, B>;
    __device__ static L id() {
        L r;
#pragma unroll
        for (int i = 0; i < D; ++i) r.d[i] = T(0);
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int m = 0; m < B; ++m) r.n[i][m] = i == m ? T(1) : T(0);
        return r;
    }
    __device__ static L comb(const L& e, const L& l) {  // e later, l earlier
        L r;
#pragma unroll
        for (int j = 0; j < NB; ++j)
#pragma unroll
            for (int i = 0; i < B; ++i) {
                T s = l.d[Op::blk(j, i)];
#pragma unroll
                for (int m = 0; m < B; ++m) s = fma(l.n[i][m], e.d[Op::blk(j, m)], s);
                r.d[Op::blk(j, i)] = s;
            }
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int m = 0; m < B; ++m) {
                T s = T(0);
#pragma unroll
                for (int k = 0; k < B; ++k) s = fma(l.n[i][k], e.n[k][m], s);
                r.n[i][m] = s;
            }
        return r;
    }
    __device__ static L elem(const S&, const S& xn, const S& y) {
        L el;
#pragma unroll
        for (int i = 0; i < D; ++i) el.d[i] = y.v[i];
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int m = 0; m < B; ++m) el.n[i][m] = Op::block_m(xn, m, i);  // N = M^T
        return el;
    }
    __device__ static void apply(const L& el, const T (&g)[D], T (&o)[D]) {
#pragma unroll
        for (int j = 0; j < NB; ++j)
#pragma unroll
            for (int i = 0; i < B; ++i) {
                T s = el.d[Op::blk(j, i)];
#pragma unroll
                for (int m = 0; m < B; ++m) s = fma(el.n[i][m], g[Op::blk(j, m)], s);
                o[Op::blk(j, i)] = s;
            }
    }
};

template <class T, int D>
struct WideArgs {
    int64_t n, tiles;
    const T* a;
    const T* ybar;
    T* abar;
    T* ys;
    void* carry;  // [tiles] primal state before each tile
    unsigned long long* lbP_agg;
    unsigned long long* lbP_incl;
    unsigned long long* lbR_agg;
    unsigned long long* lbR_incl;
    WsHeader* hdr;
    int accumulate;
};

// rows [e, e + kWideV) of a [n][D] array (pad rows past n)
template <class T, int D>
__device__ __forceinline__ void ld_rows(const T* p, int64_t e, int64_t n, const WState<T, D>& pad,
                                        WState<T, D> (&o)[kWideV]) {
    constexpr int NV = kWideV * D;
    constexpr int VV = Vec16<T>::N;
    if (e + kWideV <= n) {
        T buf[NV];
#pragma unroll
        for (int q = 0; q < NV / VV; ++q) {
            const Vec16<T> x = ld_vec_stream(p + e * D + q * VV);
#pragma unroll
            for (int j = 0; j < VV; ++j) buf[q * VV + j] = x.v[j];
        }
#pragma unroll
        for (int r = 0; r < kWideV; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) o[r].v[c] = buf[r * D + c];
    } else {
#pragma unroll
        for (int r = 0; r < kWideV; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) o[r].v[c] = e + r < n ? p[(e + r) * D + c] : pad.v[c];
    }
}

template <class T, int D>
__device__ __forceinline__ void st_rows(T* p, int64_t e, int64_t n, const T (&v)[kWideV][D], bool add) {
#pragma unroll
    for (int r = 0; r < kWideV; ++r) {
        if (e + r >= n) break;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T* q = p + (e + r) * D + c;
            *q = add ? *q + v[r][c] : v[r][c];
        }
    }
}

// Forward pass: each tile's primal prefix (carry) by look-back; ys if asked.
template <class Op, class T>
__global__ void __launch_bounds__(kWideBlock) wide_primal_kernel(WideArgs<T, Op::D> A) {
    constexpr int D = Op::D, NW = kWideBlock / 32;
    using S = typename Op::S;
    __shared__ uint32_t s_tile;
    __shared__ S s_tot[NW];
    __shared__ S s_pre;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    const int64_t t = s_tile;
    const int64_t e = t * kWideTile + (int64_t)threadIdx.x * kWideV;
    S x[kWideV];
    ld_rows<T, D>(A.a, e, A.n, Op::id(), x);
    S agg[1];
    agg[0] = x[0];
#pragma unroll
    for (int r = 1; r < kWideV; ++r) agg[0] = Op::comb(agg[0], x[r]);
    auto comb = [](const S& l, const S& r) { return Op::comb(l, r); };
    S wex[1];
    const S total = block_scan_part1<S, false, 1, NW>(agg, wex, s_tot, Op::id(), comb);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<S> st{A.lbP_agg, A.lbP_incl};
        const S pre = lookback(t, st, total, Op::id(), comb, A.hdr);
        if ((threadIdx.x & 31) == 0) {
            static_cast<S*>(A.carry)[t] = pre;
            s_pre = pre;
        }
    }
    __syncthreads();
    if (A.ys && e < A.n) {
        S run = block_scan_excl<S, false, 1, NW>(0, wex, s_tot, s_pre, comb);
        T out[kWideV][D];
#pragma unroll
        for (int r = 0; r < kWideV; ++r) {
            run = Op::comb(run, x[r]);
#pragma unroll
            for (int c = 0; c < D; ++c) out[r][c] = run.v[c];
        }
        st_rows<T, D>(A.ys, e, A.n, out, false);
    }
}

// Reverse pass (tiles right to left).
template <class Op, class T, class LP>
__global__ void __launch_bounds__(kWideBlock) wide_adjoint_kernel(WideArgs<T, Op::D> A) {
    constexpr int D = Op::D, NW = kWideBlock / 32;
    using S = typename Op::S;
    using L = typename LP::L;
    __shared__ uint32_t s_tile;
    __shared__ S s_totP[NW];
    __shared__ L s_totR[NW];
    __shared__ S s_carry;
    __shared__ L s_suf;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;
    const int64_t tile = A.tiles - 1 - t_log;
    const int64_t e = tile * kWideTile + (int64_t)threadIdx.x * kWideV;
    if (threadIdx.x == 0) s_carry = static_cast<const S*>(A.carry)[tile];
    S x[kWideV], yb[kWideV];
    ld_rows<T, D>(A.a, e, A.n, Op::id(), x);
    ld_rows<T, D>(A.ybar, e, A.n, S{}, yb);
    S xnext = Op::id();  // the element after the thread's last row
    if (e + kWideV < A.n) {
#pragma unroll
        for (int c = 0; c < D; ++c) xnext.v[c] = A.a[(e + kWideV) * D + c];
    }
    // primal: the thread's exclusive prefix
    auto comb = [](const S& l, const S& r) { return Op::comb(l, r); };
    S aggP[1];
    aggP[0] = x[0];
#pragma unroll
    for (int r = 1; r < kWideV; ++r) aggP[0] = Op::comb(aggP[0], x[r]);
    S wexP[1];
    (void)block_scan_part1<S, false, 1, NW>(aggP, wexP, s_totP, Op::id(), comb);
    __syncthreads();
    S prev[kWideV + 1];  // prev[r] = rs before row r; prev[kWideV] = rs of the last row
    prev[0] = block_scan_excl<S, false, 1, NW>(0, wexP, s_totP, s_carry, comb);
#pragma unroll
    for (int r = 0; r < kWideV; ++r) prev[r + 1] = Op::comb(prev[r], x[r]);
    // lin_o element of row r: (ybar_r, J_left(r+1)^T), formed when needed
    auto element = [&](int r) { return LP::elem(prev[r + 1], r + 1 < kWideV ? x[r + 1] : xnext, yb[r]); };
    L agg[1];
    agg[0] = element(kWideV - 1);
#pragma unroll
    for (int r = kWideV - 2; r >= 0; --r) agg[0] = LP::comb(agg[0], element(r));
    auto rc = [](const L& later, const L& earlier) { return LP::comb(later, earlier); };
    L wexR[1];
    const L totR = block_scan_part1<L, true, 1, NW>(agg, wexR, s_totR, LP::id(), rc);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<L> st{A.lbR_agg, A.lbR_incl};
        const L suf = lookback(t_log, st, totR, LP::id(), rc, A.hdr);
        if ((threadIdx.x & 31) == 0) s_suf = suf;
    }
    __syncthreads();
    if (e >= A.n) return;
    const L after = block_scan_excl<L, true, 1, NW>(0, wexR, s_totR, s_suf, rc);
    // rs_bar after the thread's rows is after(0) = after.d
    T g[D];
#pragma unroll
    for (int i = 0; i < D; ++i) g[i] = after.d[i];
    T out[kWideV][D];
#pragma unroll
    for (int r = kWideV - 1; r >= 0; --r) {
        // rs_bar_r = ybar_r + J_left(r+1)^T rs_bar_{r+1}
        T ng[D];
        LP::apply(element(r), g, ng);
#pragma unroll
        for (int i = 0; i < D; ++i) g[i] = ng[i];
        if (e + r == 0) {
#pragma unroll
            for (int i = 0; i < D; ++i) out[r][i] = g[i];
        } else {
            Op::vjp_right(prev[r], x[r], g, out[r]);
        }
    }
    st_rows<T, D>(A.abar, e, A.n, out, A.accumulate != 0);
}

// operators whose J_left acts blockwise (Op::kB, Op::blk, Op::block_m)
template <class Op, class = void>
struct HasBlocks : std::false_type {};
template <class Op>
struct HasBlocks<Op, std::void_t<decltype(Op::kB)>> : std::true_type {};
template <class Op>
constexpr bool kHasBlocks = HasBlocks<Op>::value;

template <class Op, class T>
struct WideLayout {
    size_t off_carry, off_pA, off_pI, off_rA, off_rI, total;
    int64_t tiles;
};

template <class Op, class T>
WideLayout<Op, T> wide_layout(int64_t n) {
    using S = typename Op::S;
    using L = WLin<T, Op::D>;
    WideLayout<Op, T> W{};
    W.tiles = (n + kWideTile - 1) / kWideTile;
    if (W.tiles < 1) W.tiles = 1;
    size_t o = sizeof(WsHeader);
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = round_up(o + bytes, 256);
        return at;
    };
    W.off_carry = take(sizeof(S) * (size_t)W.tiles);
    W.off_pA = take(8 * (size_t)lb_words<S>() * (size_t)W.tiles);
    W.off_pI = take(8 * (size_t)lb_words<S>() * (size_t)W.tiles);
    W.off_rA = take(8 * (size_t)lb_words<L>() * (size_t)W.tiles);
    W.off_rI = take(8 * (size_t)lb_words<L>() * (size_t)W.tiles);
    W.total = o;
    return W;
}

template <class Op, class T>
int run_wide(int64_t n, const void* a, const void* ybar, void* abar, void* ys, uint32_t flags, void* work,
             size_t work_bytes, cudaStream_t s) {
    const WideLayout<Op, T> W = wide_layout<Op, T>(n);
    if (work == nullptr || work_bytes < W.total || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (n == 0) return ADPAR_OK;
    char* w = static_cast<char*>(work);
    if (cudaMemsetAsync(w, 0, sizeof(WsHeader), s) != cudaSuccess) return ADPAR_ERR_CUDA;
    if (cudaMemsetAsync(w + W.off_pA, 0, W.total - W.off_pA, s) != cudaSuccess) return ADPAR_ERR_CUDA;
    WideArgs<T, Op::D> A{};
    A.n = n;
    A.tiles = W.tiles;
    A.a = static_cast<const T*>(a);
    A.ybar = static_cast<const T*>(ybar);
    A.abar = static_cast<T*>(abar);
    A.ys = static_cast<T*>(ys);
    A.carry = w + W.off_carry;
    A.lbP_agg = reinterpret_cast<unsigned long long*>(w + W.off_pA);
    A.lbP_incl = reinterpret_cast<unsigned long long*>(w + W.off_pI);
    A.lbR_agg = reinterpret_cast<unsigned long long*>(w + W.off_rA);
    A.lbR_incl = reinterpret_cast<unsigned long long*>(w + W.off_rI);
    A.hdr = reinterpret_cast<WsHeader*>(w);
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    wide_primal_kernel<Op, T><<<(unsigned)W.tiles, kWideBlock, 0, s>>>(A);
    if constexpr (kHasBlocks<Op>) {
        if (!(flags & ADPAR_FULL_LIN_O)) {
            wide_adjoint_kernel<Op, T, LinBlock<Op, T>><<<(unsigned)W.tiles, kWideBlock, 0, s>>>(A);
            return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
        }
    }
    wide_adjoint_kernel<Op, T, LinFull<Op, T>><<<(unsigned)W.tiles, kWideBlock, 0, s>>>(A);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

int wide_width(int op) { return op == ADPAR_OP_LINREC ? 2 : (op == ADPAR_OP_MATREC2 ? 6 : 0); }

}  // namespace

size_t scan_wide_workspace_size(adpar_opdesc d, int64_t n) {
    if (n < 0 || wide_width(d.op) == 0) return (size_t)-1;
    if (d.dtype == ADPAR_F32)
        return d.op == ADPAR_OP_LINREC ? wide_layout<WLinrec<float>, float>(n).total
                                       : wide_layout<WMatrec2<float>, float>(n).total;
    if (d.dtype == ADPAR_F64)
        return d.op == ADPAR_OP_LINREC ? wide_layout<WLinrec<double>, double>(n).total
                                       : wide_layout<WMatrec2<double>, double>(n).total;
    return (size_t)-1;
}

}  // namespace adpar

extern "C" int adpar_vjp_scan_wide(adpar_opdesc d, int64_t n, const void* a, const void* ybar, void* abar,
                                   void* ys_out, uint32_t flags, void* work, size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0) return ADPAR_ERR_INVALID;
    const int D = wide_width(d.op);
    if (D == 0 || d.width != D) return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)(ADPAR_ACCUMULATE | ADPAR_FULL_LIN_O)) return ADPAR_ERR_UNSUPPORTED;
    if (n > 0) {
        if (!a || !ybar || !abar) return ADPAR_ERR_INVALID;
        const void* ptrs[] = {a, ybar, abar, ys_out};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.dtype == ADPAR_F32) {
        if (d.op == ADPAR_OP_LINREC)
            return run_wide<WLinrec<float>, float>(n, a, ybar, abar, ys_out, flags, work, work_bytes, s);
        return run_wide<WMatrec2<float>, float>(n, a, ybar, abar, ys_out, flags, work, work_bytes, s);
    }
    if (d.op == ADPAR_OP_LINREC)
        return run_wide<WLinrec<double>, double>(n, a, ybar, abar, ys_out, flags, work, work_bytes, s);
    return run_wide<WMatrec2<double>, double>(n, a, ybar, abar, ys_out, flags, work, work_bytes, s);
}
