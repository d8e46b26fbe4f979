// VJP of reduce (Sec. 5.1 and its special cases in Sec. 5.1.1).
//
//   ADD      abar_i = ybar (a broadcast; y itself only if asked for).
//   MIN/MAX  the forward sweep is re-executed as argmin/argmax with the
//            lowest index on ties; abar_{i_y} = ybar and 0 elsewhere.  In
//            overwrite mode the zero fill of abar rides along with the
//            reduction pass, so the whole VJP is one read of a and one
//            write of abar.
//   MUL      the forward sweep is re-executed as a map-reduce of (zero
//            count, lowest zero index, scaled product of the nonzeros);
//            then one map applies the three cases of Sec. 5.1.1.
//
// Pass 1 is a grid-stride map-reduce whose last block to finish (atomic
// ticket) combines the per-block partials, so the reduction needs no second
// launch; the * rule adds one map launch.
#include <algorithm>
#include <type_traits>
#include <math_constants.h>

#include "common.cuh"
#include "prod.cuh"
#include "scan_ops.cuh"

namespace adpar {
namespace {

constexpr int kRedBlock = 256;
constexpr int kRedMaxBlocks = 1024;

template <class T>
struct ArgState {
    T v;
    int64_t i;
};

// max / min with the lowest index on ties
template <class T, bool MAX>
__device__ __forceinline__ ArgState<T> arg_comb(const ArgState<T>& x, const ArgState<T>& y) {
    const bool take_y = MAX ? (y.v > x.v || (y.v == x.v && y.i < x.i))
                            : (y.v < x.v || (y.v == x.v && y.i < x.i));
    return take_y ? y : x;
}

struct ReduceArgs {
    int op;
    int64_t n;
    const void* a;
    const void* ybar;
    void* abar;
    void* y_out;
    int64_t* argidx_out;
    adpar_prod_aux* aux_out;
    int8_t* abar_sign;
    int accumulate;
    int logdomain;
    int primal_only;  // forward operator only: no adjoint is written
    WsHeader* hdr;
    void* partials;  // [gridDim.x] states
    void* final_state;
};

__global__ void header_init_kernel(WsHeader* hdr) {
    reinterpret_cast<uint32_t*>(hdr)[threadIdx.x] = 0u;
}

template <class S, class Comb>
__device__ __forceinline__ S block_reduce(S v, Comb comb, S* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        S o = shfl_down_s(v, off);
        v = comb(v, o);
    }
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : s_warp[0];
        // lanes past the warp count repeat warp 0: harmless for min/max/argmin;
        // for sums only lanes < nwarps are combined below
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            S o = shfl_down_s(v, off);
            if (lane + off < (int)(blockDim.x >> 5)) v = comb(v, o);
        }
    }
    return v;  // valid in thread 0
}

// Returns true in the block that finished last (all partials are visible).
__device__ __forceinline__ bool last_block(WsHeader* hdr) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t t = atomicAdd(&hdr->done[0], 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// ------------------------------------------------------------------ ADD
template <class T>
__global__ void __launch_bounds__(kRedBlock) reduce_add_kernel(ReduceArgs A) {
    __shared__ T s_warp[kRedBlock / 32];
    const T* a = static_cast<const T*>(A.a);
    T* abar = static_cast<T*>(A.abar);
    const T yb = A.primal_only ? T(0) : *static_cast<const T*>(A.ybar);
    constexpr int V = Vec16<T>::N;
    const int64_t nvec = A.n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool want_y = A.y_out != nullptr;
    T acc = T(0);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvec; v += stride) {
        if (want_y) {
            Vec16<T> x = ld_vec_stream(a + v * V);
#pragma unroll
            for (int j = 0; j < V; ++j) acc += x.v[j];
        }
        if (A.primal_only) continue;
        Vec16<T> o;
        if (A.accumulate) {
            o = ld_vec(abar + v * V);
#pragma unroll
            for (int j = 0; j < V; ++j) o.v[j] += yb;
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) o.v[j] = yb;
        }
        st_vec(abar + v * V, o);
    }
    if (blockIdx.x == 0 && threadIdx.x < A.n - nvec * V) {
        const int64_t i = nvec * V + threadIdx.x;
        if (want_y) acc += a[i];
        if (!A.primal_only) abar[i] = A.accumulate ? abar[i] + yb : yb;
    }
    if (!want_y) return;
    auto add = [](T x, T y) { return x + y; };
    T bsum = block_reduce(acc, add, s_warp);
    if (threadIdx.x == 0) static_cast<T*>(A.partials)[blockIdx.x] = bsum;
    if (!last_block(A.hdr)) return;
    T tot = T(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) tot += ld_cg(static_cast<T*>(A.partials) + b);
    __syncthreads();
    tot = block_reduce(tot, add, s_warp);
    if (threadIdx.x == 0) {
        *static_cast<T*>(A.y_out) = tot;
        A.hdr->done[0] = 0u;
    }
}

// -------------------------------------------------------------- MIN/MAX
template <class T, bool MAX>
__global__ void __launch_bounds__(kRedBlock) reduce_arg_kernel(ReduceArgs A) {
    using S = ArgState<T>;
    __shared__ S s_warp[kRedBlock / 32];
    const T* a = static_cast<const T*>(A.a);
    T* abar = static_cast<T*>(A.abar);
    constexpr int V = Vec16<T>::N;
    const int64_t nvec = A.n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool fill = !A.accumulate && !A.primal_only;
    S st{MAX ? -pos_inf<T>() : pos_inf<T>(), INT64_MAX};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvec; v += stride) {
        Vec16<T> x = ld_vec_stream(a + v * V);
#pragma unroll
        for (int j = 0; j < V; ++j) st = arg_comb<T, MAX>(st, S{x.v[j], v * V + j});
        if (fill) {
            Vec16<T> z;
#pragma unroll
            for (int j = 0; j < V; ++j) z.v[j] = T(0);
            st_vec(abar + v * V, z);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < A.n - nvec * V) {
        const int64_t i = nvec * V + threadIdx.x;
        st = arg_comb<T, MAX>(st, S{a[i], i});
        if (fill) abar[i] = T(0);
    }
    auto comb = [](const S& x, const S& y) { return arg_comb<T, MAX>(x, y); };
    S bs = block_reduce(st, comb, s_warp);
    if (threadIdx.x == 0) static_cast<S*>(A.partials)[blockIdx.x] = bs;
    if (!last_block(A.hdr)) return;
    S tot{MAX ? -pos_inf<T>() : pos_inf<T>(), INT64_MAX};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        tot = arg_comb<T, MAX>(tot, ld_cg(static_cast<S*>(A.partials) + b));
    __syncthreads();
    tot = block_reduce(tot, comb, s_warp);
    if (threadIdx.x == 0) {
        const bool any = A.n > 0;
        if (A.y_out) *static_cast<T*>(A.y_out) = tot.v;
        if (A.argidx_out) *A.argidx_out = any ? tot.i : -1;
        if (any && !A.primal_only) {
            const T yb = *static_cast<const T*>(A.ybar);
            abar[tot.i] = A.accumulate ? abar[tot.i] + yb : yb;
        }
        A.hdr->done[0] = 0u;
    }
}

// ------------------------------------------------------------------ MUL
// The recompute multiplies mantissas in fixed point on the integer pipes
// (no FP64 instruction per element for either dtype).
template <class T>
__global__ void __launch_bounds__(kRedBlock) reduce_prod_kernel(ReduceArgs A) {
    using S = ProdStateQ;
    __shared__ S s_warp[kRedBlock / 32];
    const T* a = static_cast<const T*>(A.a);
    constexpr int V = Vec16<T>::N;
    const int64_t nvec = A.n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    S st = S::id();
    constexpr int U = 4;  // vectors in flight per thread
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; v + (U - 1) * stride < nvec; v += U * stride) {
        Vec16<T> x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = ld_vec(a + (v + u * stride) * V);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < V; ++j) st.push(x[u].v[j], (v + u * stride) * V + j);
    }
    for (; v < nvec; v += stride) {
        Vec16<T> x = ld_vec(a + v * V);
#pragma unroll
        for (int j = 0; j < V; ++j) st.push(x.v[j], v * V + j);
    }
    if (blockIdx.x == 0 && threadIdx.x < A.n - nvec * V) {
        const int64_t i = nvec * V + threadIdx.x;
        st.push(a[i], i);
    }
    auto comb = [](const S& x, const S& y) { return S::comb(x, y); };
    S bs = block_reduce(st, comb, s_warp);
    if (threadIdx.x == 0) static_cast<S*>(A.partials)[blockIdx.x] = bs;
    if (!last_block(A.hdr)) return;
    S totq = S::id();
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        totq = S::comb(totq, ld_cg(static_cast<S*>(A.partials) + b));
    __syncthreads();
    totq = block_reduce(totq, comb, s_warp);
    if (threadIdx.x == 0) {
        const ProdState tot = totq.to_state();
        *static_cast<ProdState*>(A.final_state) = tot;
        if (A.y_out)
            *static_cast<T*>(A.y_out) = tot.nz > 0 ? T(0) : (T)ldexp_clamped(tot.m, tot.e);
        if (A.aux_out) {
            adpar_prod_aux x;
            x.nzero = tot.nz;
            x.first_zero = tot.nz > 0 ? tot.first : -1;
            x.exp2 = tot.e;
            x.mant = tot.m;
            x.log_abs_nz = log(fabs(tot.m)) + (double)tot.e * 0.69314718055994530942;
            x.sign = tot.m > 0 ? 1 : -1;
            x.reserved = 0;
            *A.aux_out = x;
        }
        A.hdr->done[0] = 0u;
    }
}

// The three cases of Sec. 5.1.1 with z = number of zeros, p = product of
// the nonzeros (scaled):  z = 0: abar_i = p / a_i * ybar;  z = 1: only the
// zero at i0 gets p * ybar;  z >= 2: nothing.  In log mode abar_i holds
// ln|contribution| (-inf for none) and abar_sign its sign.
// The map over elements t0, t0 + stride, ... (t0 = 0 writes the single-
// element cases); st is the recomputed forward state.
template <class T>
__device__ __forceinline__ void prod_adjoint_body(const ReduceArgs& A, const ProdState& st, int64_t t0,
                                                  int64_t stride) {
    const double yb = (double)*static_cast<const T*>(A.ybar);
    T* abar = static_cast<T*>(A.abar);
    const T* a = static_cast<const T*>(A.a);
    // ybar as (mantissa, exponent) so every factor has a bounded mantissa
    double ym = 0.0;
    int64_t ye = 0;
    if (yb != 0.0) split_pow2(yb, ym, ye);
    const float qf = (float)(st.m * ym);  // the FP32 path's factor, in [0.25, 1]
    const double lg_p = log(fabs(st.m)) + (double)st.e * 0.69314718055994530942;
    const double lg_y = yb != 0.0 ? log(fabs(yb)) : -CUDART_INF;
    const int sgn_py = (st.m > 0 ? 1 : -1) * (yb > 0 ? 1 : (yb < 0 ? -1 : 0));

    if (A.logdomain) {
        for (int64_t i = t0; i < A.n; i += stride) {
            double lg = -CUDART_INF;
            int sg = 0;
            if (yb != 0.0) {
                if (st.nz == 0) {
                    const double ai = (double)a[i];
                    lg = lg_p - log(fabs(ai)) + lg_y;
                    sg = sgn_py * (ai > 0 ? 1 : -1);
                } else if (st.nz == 1 && i == st.first) {
                    lg = lg_p + lg_y;
                    sg = sgn_py;
                }
            }
            abar[i] = (T)lg;
            if (A.abar_sign) A.abar_sign[i] = (int8_t)sg;
        }
        return;
    }
    if (A.accumulate && st.nz >= 2) return;  // nothing changes
    if (A.accumulate && st.nz == 1) {
        if (t0 == 0 && yb != 0.0) {
            const double c = ldexp_clamped(st.m * ym, st.e + ye);
            abar[st.first] = (T)((double)abar[st.first] + c);
        }
        return;
    }
    if constexpr (sizeof(T) == 4) {
        // FP32, no zero: abar_i = p / a_i * ybar in FP32 arithmetic with the
        // exponent kept apart (qf = the mantissa of p * ybar), 4 per thread
        if (st.nz == 0 && yb != 0.0) {
            const int64_t nv = A.n / 4;
            const int64_t eb = st.e + ye;
            auto one = [&](float x) {
                float mf;
                int ef;
                split_pow2_f32m(x, mf, ef);
                return scale_pow2f(qf * __frcp_rn(mf), eb - ef);
            };
            for (int64_t v = t0; v < nv; v += stride) {
                const float4 x = __ldcs(reinterpret_cast<const float4*>(a) + v);
                float4 o = make_float4(one(x.x), one(x.y), one(x.z), one(x.w));
                if (A.accumulate) {
                    const float4 p = reinterpret_cast<const float4*>(abar)[v];
                    o.x += p.x; o.y += p.y; o.z += p.z; o.w += p.w;
                }
                __stcs(reinterpret_cast<float4*>(abar) + v, o);
            }
            const int64_t i = nv * 4 + t0;
            if (i < A.n) abar[i] = A.accumulate ? abar[i] + one(a[i]) : one(a[i]);
            return;
        }
    }
    const double kq = st.m * ym;  // the FP64 path's numerator mantissa, in [0.25, 1)
    if constexpr (sizeof(T) == 8) {
        // FP64, no zero: abar_i = p / a_i * ybar, two elements per 16-byte vector
        if (st.nz == 0 && yb != 0.0) {
            const int64_t nv = A.n / 2;
            const int64_t eb = st.e + ye;
            auto one = [&](double x) {
                double mi;
                int64_t ei;
                split_pow2(x, mi, ei);
                return scale_pow2(quot_mantissa(kq, mi), eb - ei);
            };
            for (int64_t v = t0; v < nv; v += stride) {
                const double2 x = __ldcs(reinterpret_cast<const double2*>(a) + v);
                double2 o = make_double2(one(x.x), one(x.y));
                if (A.accumulate) {
                    const double2 p = reinterpret_cast<const double2*>(abar)[v];
                    o.x += p.x;
                    o.y += p.y;
                }
                __stcs(reinterpret_cast<double2*>(abar) + v, o);
            }
            if (t0 == 0 && (A.n & 1)) {
                const int64_t i = A.n - 1;
                abar[i] = A.accumulate ? abar[i] + one(a[i]) : one(a[i]);
            }
            return;
        }
    }
    for (int64_t i = t0; i < A.n; i += stride) {
        double c = 0.0;
        if (yb != 0.0) {
            if (st.nz == 0) {
                double mi;
                int64_t ei;
                split_pow2((double)a[i], mi, ei);
                c = scale_pow2(quot_mantissa(kq, mi), st.e + ye - ei);
            } else if (st.nz == 1 && i == st.first) {
                c = ldexp_clamped(st.m * ym, st.e + ye);
            }
        }
        abar[i] = A.accumulate ? (T)((double)abar[i] + c) : (T)c;
    }
}

template <class T>
__global__ void __launch_bounds__(kRedBlock) prod_adjoint_kernel(ReduceArgs A) {
    const ProdState st = *static_cast<const ProdState*>(A.final_state);
    prod_adjoint_body<T>(A, st, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------ host side
size_t state_bytes(int op, int dtype) {
    const size_t t = dtype == ADPAR_F64 ? 8 : 4;
    switch (op) {
    case ADPAR_OP_ADD: return t;
    case ADPAR_OP_MIN:
    case ADPAR_OP_MAX: return 16;
    case ADPAR_OP_MUL: return std::max(sizeof(ProdState), sizeof(ProdStateQ));
    }
    return 0;
}

int grid_for(int64_t n, int dtype) {
    const int64_t per_block = (int64_t)kRedBlock * (dtype == ADPAR_F64 ? 2 : 4) * 8;
    int64_t g = (n + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, kRedMaxBlocks));
}

template <class T>
int run_reduce(ReduceArgs A, int op, cudaStream_t s) {
    const int grid = grid_for(A.n, sizeof(T) == 8 ? ADPAR_F64 : ADPAR_F32);
    switch (op) {
    case ADPAR_OP_ADD:
        reduce_add_kernel<T><<<grid, kRedBlock, 0, s>>>(A);
        break;
    case ADPAR_OP_MIN:
        reduce_arg_kernel<T, false><<<grid, kRedBlock, 0, s>>>(A);
        break;
    case ADPAR_OP_MAX:
        reduce_arg_kernel<T, true><<<grid, kRedBlock, 0, s>>>(A);
        break;
    case ADPAR_OP_MUL: {
        reduce_prod_kernel<T><<<grid, kRedBlock, 0, s>>>(A);
        if (A.primal_only) break;
        const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>((A.n + 1023) / 1024, 4 * 152));
        prod_adjoint_kernel<T><<<g2, kRedBlock, 0, s>>>(A);
        break;
    }
    default:
        return ADPAR_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

}  // namespace

size_t reduce_workspace_size(adpar_opdesc d) {
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return (size_t)-1;
    const size_t sb = state_bytes(d.op, d.dtype);
    if (sb == 0) return (size_t)-1;
    return sizeof(WsHeader) + round_up(kRedMaxBlocks * sb, 256) + 256;
}

}  // namespace adpar

extern "C" int adpar_vjp_reduce(adpar_opdesc d, int64_t n, const void* a, const void* ybar, void* abar,
                                void* y_out, int64_t* argidx_out, adpar_prod_aux* aux_out,
                                int8_t* abar_sign, uint32_t flags, void* work, size_t work_bytes,
                                void* stream) {
    using namespace adpar;
    if (n < 0 || d.width != 1) return ADPAR_ERR_INVALID;
    if (d.op != ADPAR_OP_ADD && d.op != ADPAR_OP_MUL && d.op != ADPAR_OP_MIN && d.op != ADPAR_OP_MAX)
        return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)(ADPAR_ACCUMULATE | ADPAR_PROD_LOGDOMAIN)) return ADPAR_ERR_UNSUPPORTED;
    const bool logd = (flags & ADPAR_PROD_LOGDOMAIN) != 0;
    if (logd && (d.op != ADPAR_OP_MUL || (flags & ADPAR_ACCUMULATE))) return ADPAR_ERR_UNSUPPORTED;
    if (abar_sign && !logd) return ADPAR_ERR_INVALID;
    if (!ybar || (n > 0 && !abar)) return ADPAR_ERR_INVALID;
    if (n > 0 && !a && !(d.op == ADPAR_OP_ADD && !y_out)) return ADPAR_ERR_INVALID;
    if ((a && !aligned16(a)) || (abar && !aligned16(abar))) return ADPAR_ERR_ALIGN;
    const size_t need = reduce_workspace_size(d);
    if (!work || work_bytes < need || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    ReduceArgs A{};
    A.op = d.op;
    A.n = n;
    A.a = a;
    A.ybar = ybar;
    A.abar = abar;
    A.y_out = y_out;
    A.argidx_out = argidx_out;
    A.aux_out = aux_out;
    A.abar_sign = abar_sign;
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    A.logdomain = logd ? 1 : 0;
    char* w = static_cast<char*>(work);
    A.hdr = reinterpret_cast<WsHeader*>(w);
    A.partials = w + sizeof(WsHeader);
    A.final_state = w + sizeof(WsHeader) + round_up(kRedMaxBlocks * state_bytes(d.op, d.dtype), 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the "last block" counter must start at zero in a workspace of unknown
    // contents
    header_init_kernel<<<1, 64, 0, s>>>(A.hdr);
    if (d.dtype == ADPAR_F32) return run_reduce<float>(A, d.op, s);
    return run_reduce<double>(A, d.op, s);
}

extern "C" int adpar_reduce(adpar_opdesc d, int64_t n, const void* a, void* y_out, int64_t* argidx_out,
                            adpar_prod_aux* aux_out, void* work, size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0 || d.width != 1) return ADPAR_ERR_INVALID;
    if (d.op != ADPAR_OP_ADD && d.op != ADPAR_OP_MUL && d.op != ADPAR_OP_MIN && d.op != ADPAR_OP_MAX)
        return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (!y_out || (n > 0 && !a)) return ADPAR_ERR_INVALID;
    if (a && !aligned16(a)) return ADPAR_ERR_ALIGN;
    const size_t need = reduce_workspace_size(d);
    if (!work || work_bytes < need || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    ReduceArgs A{};
    A.op = d.op;
    A.n = n;
    A.a = a;
    A.y_out = y_out;
    A.argidx_out = argidx_out;
    A.aux_out = aux_out;
    A.primal_only = 1;
    char* w = static_cast<char*>(work);
    A.hdr = reinterpret_cast<WsHeader*>(w);
    A.partials = w + sizeof(WsHeader);
    A.final_state = w + sizeof(WsHeader) + round_up(kRedMaxBlocks * state_bytes(d.op, d.dtype), 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    header_init_kernel<<<1, 64, 0, s>>>(A.hdr);
    if (d.dtype == ADPAR_F32) return run_reduce<float>(A, d.op, s);
    return run_reduce<double>(A, d.op, s);
}
