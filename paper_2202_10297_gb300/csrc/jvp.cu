// Forward mode (Sec. 3) of the bulk operators: the tangent of the output
// along a tangent of the inputs, i.e. each operator run on dual numbers.
//
//   reduce           +: ydot = sum_i adot_i.  min/max: ydot = adot[i_y], i_y
//                    the recomputed argmin/argmax (lowest index on ties).
//                    *: the product rule on the recomputed forward sweep of
//                    Sec. 5.1.1 (zero count z, lowest zero i0, scaled
//                    nonzero product p):  z = 0: ydot = p sum_i adot_i / a_i,
//                    z = 1: ydot = p adot_i0,  z >= 2: ydot = 0.
//   reduce_by_index  the same per bin (Sec. 5.1.2); its + case is
//                    reduce_by_index + applied to the tangents.
//   scatter          linear in (xs, vs): its tangent is the scatter of the
//                    tangents (Sec. 5.3).
//   map_acc          xsdot_j = dg/da asdot[is_j] + dg/dw wsdot_j (Sec. 5.4).
//   k-means          forward over reverse (Sec. 7.4): the reverse sweep of
//                    the cost run on dual numbers along a tangent Cdot of the
//                    centroids, giving the tangent of the gradient (a
//                    Hessian-vector product) and of the loss.
//
// The recomputed primal states come from the library's own forward
// kernels (adpar_reduce, adpar_hist, adpar_kmeans_vjp).  The reduce sums
// accumulate in FP64 in a fixed order; the per-bin sums of the * rule use
// FP64 atomics (privatised in shared memory for up to 4096 bins).
#include <algorithm>
#include <math_constants.h>

#include "common.cuh"
#include "prod.cuh"

namespace adpar {
size_t reduce_workspace_size(adpar_opdesc d);
size_t hist_workspace_size(adpar_opdesc d, int64_t m);
size_t kmeans_workspace_size(int64_t k);

namespace {

constexpr int kJBlock = 256;
constexpr int kJMaxBlocks = 1024;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_w[kJBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();  // s_w may be reused by a previous call
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < kJBlock / 32 ? s_w[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    }
    return r;  // thread 0
}

// Per-block FP64 partial sums over a grid-stride range:
//   MODE 0: sum of adot;  MODE 1: sum of adot_i / a_i over the nonzero a_i.
template <class T, int MODE>
__global__ void __launch_bounds__(kJBlock) jvp_partial_sum_kernel(int64_t n, const T* a, const T* ad,
                                                                  double* partials) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kJBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kJBlock) {
        if (MODE == 0) {
            s += (double)ad[i];
        } else {
            const double x = (double)a[i];
            if (x != 0.0) s += (double)ad[i] / x;
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

struct JvpOut {
    double v, lg;
    int sg;
};

__device__ __forceinline__ int sgn(double x) { return (x > 0.0) - (x < 0.0); }

__device__ __forceinline__ JvpOut plain_out(double v) {
    return JvpOut{v, v != 0.0 ? log(fabs(v)) : -CUDART_INF, sgn(v)};
}

// The * case given the recomputed aux record and, for z = 0, the sum S of
// adot_i / a_i; t0 = adot at the lowest zero (z = 1).
__device__ __forceinline__ JvpOut prod_tangent(const adpar_prod_aux& ax, double S, double t0) {
    if (ax.nzero == 0) {
        if (S == 0.0) return JvpOut{0.0, -CUDART_INF, 0};
        return JvpOut{ldexp_clamped(ax.mant * S, ax.exp2), ax.log_abs_nz + log(fabs(S)), ax.sign * sgn(S)};
    }
    if (ax.nzero == 1) {
        if (t0 == 0.0) return JvpOut{0.0, -CUDART_INF, 0};
        return JvpOut{ldexp_clamped(ax.mant * t0, ax.exp2), ax.log_abs_nz + log(fabs(t0)), ax.sign * sgn(t0)};
    }
    return JvpOut{0.0, -CUDART_INF, 0};
}

template <class T>
__global__ void __launch_bounds__(kJBlock) jvp_reduce_finalize_kernel(int op, int64_t n, const T* ad,
                                                                      const double* partials, int nparts,
                                                                      const adpar_prod_aux* paux,
                                                                      const int64_t* argidx, T* ydot,
                                                                      adpar_jvp_aux* jaux) {
    double S = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kJBlock) S += partials[i];
    S = block_sum(S);
    if (threadIdx.x != 0) return;
    JvpOut r{0.0, -CUDART_INF, 0};
    if (n > 0) {
        if (op == ADPAR_OP_ADD) {
            r = plain_out(S);
        } else if (op == ADPAR_OP_MIN || op == ADPAR_OP_MAX) {
            const int64_t k = *argidx;
            r = plain_out(k >= 0 ? (double)ad[k] : 0.0);
        } else {
            const adpar_prod_aux ax = *paux;
            const double t0 = ax.nzero == 1 ? (double)ad[ax.first_zero] : 0.0;
            r = prod_tangent(ax, S, t0);
        }
    }
    *ydot = (T)r.v;
    if (jaux) {
        jaux->log_abs = r.lg;
        jaux->sign = r.sg;
        jaux->reserved = 0;
    }
}

// ---------------------------------------------------------------- hist
// hsdot[b] = adot[argidx[b]] (0 for an empty bin)
template <class T>
__global__ void jvp_hist_gather_kernel(int64_t m, const int64_t* argidx, const T* vd, T* hsd) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = argidx[b];
        hsd[b] = k >= 0 ? vd[k] : T(0);
    }
}

__global__ void jvp_zero_f64_kernel(double* p, int64_t m) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m; b += (int64_t)gridDim.x * blockDim.x)
        p[b] = 0.0;
}

constexpr int kPrivBins = 4096;  // bins privatised in shared memory (32 KB of FP64)

// S[b] += adot_i / a_i over the in-range elements with a_i != 0
template <class T, class I, bool PRIV>
__global__ void __launch_bounds__(kJBlock) jvp_hist_ratio_kernel(int64_t n, int64_t m, const T* v, const T* vd,
                                                                 const I* inds, double* S) {
    __shared__ double s_acc[PRIV ? kPrivBins : 1];
    if constexpr (PRIV) {
        for (int64_t b = threadIdx.x; b < m; b += kJBlock) s_acc[b] = 0.0;
        __syncthreads();
    }
    for (int64_t i = blockIdx.x * (int64_t)kJBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kJBlock) {
        const int64_t b = (int64_t)inds[i];
        if (b < 0 || b >= m) continue;
        const double x = (double)v[i];
        if (x == 0.0) continue;
        const double q = (double)vd[i] / x;
        if constexpr (PRIV) atomicAdd(&s_acc[b], q);
        else atomicAdd(&S[b], q);
    }
    if constexpr (PRIV) {
        __syncthreads();
        for (int64_t b = threadIdx.x; b < m; b += kJBlock)
            if (s_acc[b] != 0.0) atomicAdd(&S[b], s_acc[b]);
    }
}

template <class T>
__global__ void jvp_hist_prod_finalize_kernel(int64_t m, const adpar_prod_aux* aux, const double* S, const T* vd,
                                              T* hsd, adpar_jvp_aux* jaux) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m; b += (int64_t)gridDim.x * blockDim.x) {
        const adpar_prod_aux ax = aux[b];
        const double t0 = ax.nzero == 1 ? (double)vd[ax.first_zero] : 0.0;
        const JvpOut r = prod_tangent(ax, S[b], t0);
        hsd[b] = (T)r.v;
        if (jaux) {
            jaux[b].log_abs = r.lg;
            jaux[b].sign = r.sg;
            jaux[b].reserved = 0;
        }
    }
}

// ------------------------------------------------------------- map_acc
template <class T, class I>
__global__ void jvp_map_acc_kernel(int g, int64_t nj, int64_t na, int width, const T* as, const I* is, const T* ws,
                                   const T* asd, const T* wsd, T* xsd) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nj; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)is[j];
        if (i < 0 || i >= na) {
            xsd[j] = T(0);
            continue;
        }
        if (g == ADPAR_G_GATHER) {
            xsd[j] = asd[i];
        } else if (g == ADPAR_G_SCALE) {
            T r = asd[i] * ws[j];
            if (wsd) r = fma(as[i], wsd[j], r);
            xsd[j] = r;
        } else {
            T s = T(0);
            for (int k = 0; k < width; ++k) {
                const T diff = ws[j * width + k] - as[i * width + k];
                const T dd = (wsd ? wsd[j * width + k] : T(0)) - asd[i * width + k];
                s = fma(T(2) * diff, dd, s);
            }
            xsd[j] = s;
        }
    }
}

// -------------------------------------------------------------- k-means
constexpr int kKmD = 32;
constexpr int kKmMaxK = 256;

// One warp per point, lane = coordinate.  With k* the point's certified
// argmin: the tangent of its distance  sum_j 2 (c_k*j - x_ij) cdot_k*j  adds
// to the loss tangent, and the tangent of the reverse step
// Cbar[k*] += ybar (-2)(x_i - c_k*), with x fixed, is ybar (-2)(0 - cdot_k*)
// = 2 ybar cdot_k*, accumulated per block in shared memory.
__global__ void __launch_bounds__(256) kmeans_fwd_rev_kernel(int64_t N, int k, const float* X, const float* C,
                                                             const float* Cd, const int32_t* argmin,
                                                             const float* ybar, float* Cbd, double* ydot_acc) {
    __shared__ float s_acc[kKmMaxK * kKmD];
    for (int q = threadIdx.x; q < k * kKmD; q += blockDim.x) s_acc[q] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float tw = 2.0f * *ybar;
    double yd = 0.0;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += warps) {
        const int c = argmin[i];
        const float x = X[i * kKmD + lane];
        const float cc = C[c * kKmD + lane];
        const float cd = Cd[c * kKmD + lane];
        yd += 2.0 * ((double)cc - (double)x) * (double)cd;
        atomicAdd(&s_acc[c * kKmD + lane], tw * cd);
    }
    const double ysum = block_sum(yd);
    __syncthreads();
    for (int q = threadIdx.x; q < k * kKmD; q += blockDim.x)
        if (s_acc[q] != 0.0f) atomicAdd(&Cbd[q], s_acc[q]);
    if (threadIdx.x == 0) atomicAdd(ydot_acc, ysum);
}

__global__ void kmeans_fwd_rev_init_kernel(float* Cbd, int kd, int accumulate, double* ydot_acc) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kd; q += gridDim.x * blockDim.x)
        if (!accumulate) Cbd[q] = 0.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ydot_acc = 0.0;
}

__global__ void kmeans_fwd_rev_finish_kernel(const double* ydot_acc, float* ydot_out) { *ydot_out = (float)*ydot_acc; }

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

inline int grid_for_n(int64_t n, int per_thread) {
    const int64_t g = (n + (int64_t)kJBlock * per_thread - 1) / ((int64_t)kJBlock * per_thread);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, kJMaxBlocks));
}

// workspace layouts
struct JvpReduceLayout {
    size_t red, off_scr, off_part, total;
};
JvpReduceLayout jvp_reduce_layout(adpar_opdesc d) {
    JvpReduceLayout L;
    L.red = reduce_workspace_size(d);
    L.off_scr = round_up(L.red, 256);
    L.off_part = L.off_scr + 256;  // y (8) | argidx (8) | aux (48)
    L.total = round_up(L.off_part + kJMaxBlocks * sizeof(double), 256);
    return L;
}

struct JvpHistLayout {
    size_t hist, off_hs, off_arg, off_aux, off_S, total;
};
JvpHistLayout jvp_hist_layout(adpar_opdesc d, int64_t m) {
    JvpHistLayout L;
    L.hist = hist_workspace_size(d, m);
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    L.off_hs = round_up(L.hist, 256);
    L.off_arg = round_up(L.off_hs + mm * 8, 256);
    L.off_aux = round_up(L.off_arg + mm * 8, 256);
    L.off_S = round_up(L.off_aux + mm * sizeof(adpar_prod_aux), 256);
    L.total = round_up(L.off_S + mm * 8, 256);
    return L;
}

}  // namespace

size_t jvp_reduce_workspace_size(adpar_opdesc d) {
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return (size_t)-1;
    if (reduce_workspace_size(d) == (size_t)-1) return (size_t)-1;
    return jvp_reduce_layout(d).total;
}

size_t jvp_hist_workspace_size(adpar_opdesc d, int64_t m) {
    if (m < 0 || hist_workspace_size(d, m) == (size_t)-1) return (size_t)-1;
    return jvp_hist_layout(d, m).total;
}

size_t kmeans_fwd_rev_workspace_size(int64_t N, int64_t k) {
    if (N < 0 || k < 0) return (size_t)-1;
    return round_up(kmeans_workspace_size(k), 256) + round_up((size_t)std::max<int64_t>(N, 1) * 4, 256) + 256;
}

}  // namespace adpar

// ------------------------------------------------------------ C ABI
using namespace adpar;

extern "C" int adpar_jvp_reduce(adpar_opdesc d, int64_t n, const void* a, const void* adot, void* y_out,
                                void* ydot_out, adpar_jvp_aux* ydot_aux, void* work, size_t work_bytes,
                                void* stream) {
    if (n < 0 || d.width != 1) return ADPAR_ERR_INVALID;
    if (d.op != ADPAR_OP_ADD && d.op != ADPAR_OP_MUL && d.op != ADPAR_OP_MIN && d.op != ADPAR_OP_MAX)
        return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (!ydot_out || (n > 0 && !adot)) return ADPAR_ERR_INVALID;
    if (n > 0 && !a && (d.op != ADPAR_OP_ADD || y_out)) return ADPAR_ERR_INVALID;
    if ((a && !aligned16(a)) || (adot && !aligned16(adot))) return ADPAR_ERR_ALIGN;
    const JvpReduceLayout L = jvp_reduce_layout(d);
    if (!work || work_bytes < L.total || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    char* w = static_cast<char*>(work);
    void* scr_y = w + L.off_scr;
    int64_t* scr_arg = reinterpret_cast<int64_t*>(w + L.off_scr + 8);
    adpar_prod_aux* scr_aux = reinterpret_cast<adpar_prod_aux*>(w + L.off_scr + 16);
    double* parts = reinterpret_cast<double*>(w + L.off_part);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = ADPAR_OK;
    // the recomputed forward sweep (and y when asked for)
    if (d.op != ADPAR_OP_ADD || y_out)
        st = adpar_reduce(d, n, a, y_out ? y_out : scr_y, scr_arg, d.op == ADPAR_OP_MUL ? scr_aux : nullptr, work,
                          L.red, stream);
    if (st != ADPAR_OK) return st;
    const bool f64 = d.dtype == ADPAR_F64;
    int nparts = 0;
    if (d.op == ADPAR_OP_ADD || d.op == ADPAR_OP_MUL) {
        nparts = grid_for_n(n, 8);
        if (d.op == ADPAR_OP_ADD) {
            if (f64) jvp_partial_sum_kernel<double, 0><<<nparts, kJBlock, 0, s>>>(n, nullptr, (const double*)adot, parts);
            else jvp_partial_sum_kernel<float, 0><<<nparts, kJBlock, 0, s>>>(n, nullptr, (const float*)adot, parts);
        } else {
            if (f64)
                jvp_partial_sum_kernel<double, 1><<<nparts, kJBlock, 0, s>>>(n, (const double*)a, (const double*)adot,
                                                                             parts);
            else
                jvp_partial_sum_kernel<float, 1><<<nparts, kJBlock, 0, s>>>(n, (const float*)a, (const float*)adot,
                                                                            parts);
        }
    }
    if (f64)
        jvp_reduce_finalize_kernel<double><<<1, kJBlock, 0, s>>>(d.op, n, (const double*)adot, parts, nparts, scr_aux,
                                                                 scr_arg, (double*)ydot_out, ydot_aux);
    else
        jvp_reduce_finalize_kernel<float><<<1, kJBlock, 0, s>>>(d.op, n, (const float*)adot, parts, nparts, scr_aux,
                                                                scr_arg, (float*)ydot_out, ydot_aux);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_jvp_hist(adpar_opdesc d, int64_t n, int64_t m, const void* vals, const void* vdot,
                              const void* inds, int itype, void* hs_out, void* hsdot_out, adpar_jvp_aux* hsdot_aux,
                              void* work, size_t work_bytes, void* stream) {
    if (n < 0 || m < 0 || d.width != 1) return ADPAR_ERR_INVALID;
    if (d.op != ADPAR_OP_ADD && d.op != ADPAR_OP_MUL && d.op != ADPAR_OP_MIN && d.op != ADPAR_OP_MAX)
        return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if ((m > 0 && !hsdot_out) || (n > 0 && (!vdot || !inds))) return ADPAR_ERR_INVALID;
    if (n > 0 && !vals && (d.op != ADPAR_OP_ADD || hs_out)) return ADPAR_ERR_INVALID;
    if (hsdot_aux && d.op != ADPAR_OP_MUL) return ADPAR_ERR_UNSUPPORTED;
    if ((vals && !aligned16(vals)) || (vdot && !aligned16(vdot)) || (inds && !aligned16(inds)))
        return ADPAR_ERR_ALIGN;
    const JvpHistLayout L = jvp_hist_layout(d, m);
    if (!work || work_bytes < L.total || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    if (m == 0) return ADPAR_OK;
    char* w = static_cast<char*>(work);
    void* scr_hs = w + L.off_hs;
    int64_t* scr_arg = reinterpret_cast<int64_t*>(w + L.off_arg);
    adpar_prod_aux* scr_aux = reinterpret_cast<adpar_prod_aux*>(w + L.off_aux);
    double* S = reinterpret_cast<double*>(w + L.off_S);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool f64 = d.dtype == ADPAR_F64;
    const int gm = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 4096));
    int st = ADPAR_OK;
    if (d.op == ADPAR_OP_ADD) {
        // linear: the tangent is the same reduce_by_index of the tangents
        if (hs_out) st = adpar_hist(d, n, m, vals, inds, itype, hs_out, nullptr, nullptr, work, L.hist, stream);
        if (st == ADPAR_OK) st = adpar_hist(d, n, m, vdot, inds, itype, hsdot_out, nullptr, nullptr, work, L.hist, stream);
        return st;
    }
    if (d.op == ADPAR_OP_MIN || d.op == ADPAR_OP_MAX) {
        st = adpar_hist(d, n, m, vals, inds, itype, hs_out ? hs_out : scr_hs, scr_arg, nullptr, work, L.hist, stream);
        if (st != ADPAR_OK) return st;
        if (f64) jvp_hist_gather_kernel<double><<<gm, 256, 0, s>>>(m, scr_arg, (const double*)vdot, (double*)hsdot_out);
        else jvp_hist_gather_kernel<float><<<gm, 256, 0, s>>>(m, scr_arg, (const float*)vdot, (float*)hsdot_out);
        return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
    }
    // *: per-bin zero count, lowest zero and scaled product, then S_b
    st = adpar_hist(d, n, m, vals, inds, itype, hs_out ? hs_out : scr_hs, nullptr, scr_aux, work, L.hist, stream);
    if (st != ADPAR_OK) return st;
    jvp_zero_f64_kernel<<<gm, 256, 0, s>>>(S, m);
    if (n > 0) {
        const bool priv = m <= kPrivBins;
        const int g = priv ? std::min(grid_for_n(n, 16), 4 * sm_count()) : grid_for_n(n, 4);
#define ADPAR_JVP_RATIO(T, I)                                                                             \
    do {                                                                                                  \
        if (priv) jvp_hist_ratio_kernel<T, I, true><<<g, kJBlock, 0, s>>>(n, m, (const T*)vals,           \
                                                                          (const T*)vdot, (const I*)inds, S); \
        else jvp_hist_ratio_kernel<T, I, false><<<g, kJBlock, 0, s>>>(n, m, (const T*)vals,               \
                                                                      (const T*)vdot, (const I*)inds, S);     \
    } while (0)
        if (f64) {
            if (itype == ADPAR_I32) ADPAR_JVP_RATIO(double, int32_t); else ADPAR_JVP_RATIO(double, int64_t);
        } else {
            if (itype == ADPAR_I32) ADPAR_JVP_RATIO(float, int32_t); else ADPAR_JVP_RATIO(float, int64_t);
        }
#undef ADPAR_JVP_RATIO
    }
    if (f64)
        jvp_hist_prod_finalize_kernel<double><<<gm, 256, 0, s>>>(m, scr_aux, S, (const double*)vdot, (double*)hsdot_out,
                                                                  hsdot_aux);
    else
        jvp_hist_prod_finalize_kernel<float><<<gm, 256, 0, s>>>(m, scr_aux, S, (const float*)vdot, (float*)hsdot_out,
                                                                 hsdot_aux);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_jvp_scatter(int dtype, int64_t n, int64_t m, const void* is, int itype, const void* vsdot,
                                 void* ysdot_inout, void* stream) {
    // scatter is linear in (xs, vs): its tangent is the scatter of the tangents
    return adpar_scatter(dtype, n, m, is, itype, vsdot, ysdot_inout, nullptr, stream);
}

extern "C" int adpar_jvp_map_acc(int gfun, int dtype, int64_t nj, int64_t na, int width, const void* as,
                                 const void* is, int itype, const void* ws, const void* asdot, const void* wsdot,
                                 void* xsdot, void* stream) {
    if (nj < 0 || na < 0 || width < 1) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_GATHER && gfun != ADPAR_G_SCALE && gfun != ADPAR_G_SQDIST_ROW) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_SQDIST_ROW && width != 1) return ADPAR_ERR_INVALID;
    if (dtype != ADPAR_F32 && dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if (nj == 0) return ADPAR_OK;
    if (!is || !xsdot || (na > 0 && !asdot)) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_GATHER && !ws) return ADPAR_ERR_INVALID;
    if (gfun == ADPAR_G_SCALE && wsdot && !as) return ADPAR_ERR_INVALID;
    if (gfun == ADPAR_G_SQDIST_ROW && !as) return ADPAR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nj + 255) / 256, 8 * (int64_t)sm_count()));
#define ADPAR_JVP_MAP(T, I)                                                                                     \
    jvp_map_acc_kernel<T, I><<<g, 256, 0, s>>>(gfun, nj, na, width, (const T*)as, (const I*)is, (const T*)ws, \
                                               (const T*)asdot, (const T*)wsdot, (T*)xsdot)
    if (dtype == ADPAR_F64) {
        if (itype == ADPAR_I32) ADPAR_JVP_MAP(double, int32_t); else ADPAR_JVP_MAP(double, int64_t);
    } else {
        if (itype == ADPAR_I32) ADPAR_JVP_MAP(float, int32_t); else ADPAR_JVP_MAP(float, int64_t);
    }
#undef ADPAR_JVP_MAP
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_kmeans_fwd_rev(int64_t N, int d, int k, const float* X, const float* C, const float* Cdot,
                                    const float* ybar, float* ydot_out, float* Cbardot, uint32_t flags, void* work,
                                    size_t work_bytes, void* stream) {
    if (N < 0 || d != kKmD || k < 32 || k > kKmMaxK || (k % 32) != 0) return ADPAR_ERR_INVALID;
    if (!C || !Cdot || !ybar || !Cbardot || (N > 0 && !X)) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    const size_t kw = round_up(kmeans_workspace_size(k), 256);
    const size_t need = kmeans_fwd_rev_workspace_size(N, k);
    if (!work || work_bytes < need || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    char* w = static_cast<char*>(work);
    int32_t* argmin = reinterpret_cast<int32_t*>(w + kw);
    double* yacc = reinterpret_cast<double*>(w + kw + round_up((size_t)std::max<int64_t>(N, 1) * 4, 256));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the VJP kernel's forward part: the certified argmin of every point
    if (N > 0) {
        const int st = adpar_kmeans_vjp(N, d, k, X, C, nullptr, nullptr, argmin, nullptr, 0, work, kw, stream);
        if (st != ADPAR_OK) return st;
    }
    kmeans_fwd_rev_init_kernel<<<(k * kKmD + 255) / 256, 256, 0, s>>>(Cbardot, k * kKmD,
                                                                      (flags & ADPAR_ACCUMULATE) ? 1 : 0, yacc);
    if (N > 0) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((N + 7) / 8, 4 * (int64_t)sm_count()));
        kmeans_fwd_rev_kernel<<<g, 256, 0, s>>>(N, k, X, C, Cdot, argmin, ybar, Cbardot, yacc);
    }
    if (ydot_out) kmeans_fwd_rev_finish_kernel<<<1, 1, 0, s>>>(yacc, ydot_out);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}
