// VJP of scatter (Sec. 5.3) and of map with a free array (Sec. 5.4).
//
// scatter:  ys = scatter xs is vs  (is free of duplicates).  The return
//   sweep gathers vsbar[j] += ysbar[is_j], then zeroes ysbar[is_j], which
//   turns ysbar into xsbar in place, and optionally restores
//   ys[is_j] = xs_saved[j].  Work is O(m), not O(n): the same thread reads
//   and then zeroes ysbar[is_j], and no other thread touches that element.
//
// map_acc:  xs[j] = g(as[is_j, :], ws[j, :]).  Every read of the free array
//   as becomes an accumulation into asbar at the same index (the
//   accumulators of Sec. 5.4, atomic adds on the GPU as in Sec. 6); ws is
//   an ordinary mapped input.  When asbar fits in shared memory each block
//   accumulates privately and flushes once with vector atomics (the
//   reduction form that Sec. 6.1 turns accumulators into).
#include <algorithm>

#include "common.cuh"

namespace adpar {
namespace {

constexpr int kBlk = 256;

template <class I>
__device__ __forceinline__ int64_t ldi(const I* p, int64_t j) {
    return (int64_t)__ldcs(p + j);
}

// Four indices per thread per step: the four random reads (and then the
// four random zeroing writes) are independent, so each thread keeps four
// scattered accesses in flight instead of one dependent chain.
template <class T, class I>
__global__ void __launch_bounds__(kBlk) scatter_vjp_kernel(int64_t n, int64_t m, const I* is, T* ysbar,
                                                          T* vsbar, T* ys, const T* xs_saved, int accumulate) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t j0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; j0 < m; j0 += stride) {
        const int cnt = (int)(m - j0 < 4 ? m - j0 : 4);
        int64_t k[4];
        bool in[4];
        T g[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            k[u] = u < cnt ? ldi(is, j0 + u) : -1;
            in[u] = k[u] >= 0 && k[u] < n;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) g[u] = in[u] ? ysbar[k[u]] : T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (in[u]) {
                ysbar[k[u]] = T(0);
                if (ys) ys[k[u]] = __ldcs(xs_saved + j0 + u);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (u >= cnt) break;
            if (accumulate) {
                if (in[u]) vsbar[j0 + u] += g[u];
            } else {
                __stcs(vsbar + j0 + u, g[u]);
            }
        }
    }
}

// ------------------------------------------------------------- map_acc
template <class T>
struct MapAccArgs {
    int g;
    int64_t nj, na;
    int width;
    const T* as;
    const void* is;
    const T* ws;
    const T* xsbar;
    T* asbar;
    T* wsbar;
    int acc_w;
    int priv;  // asbar (na * width values) is privatised in shared memory
};

template <class T>
__device__ __forceinline__ void acc_add(T* p, T v) {
    atomicAdd(p, v);
}

template <class T, class I>
__global__ void __launch_bounds__(kBlk) map_acc_kernel(MapAccArgs<T> A) {
    extern __shared__ unsigned char smem_raw[];
    T* sh = reinterpret_cast<T*>(smem_raw);
    const int64_t tot = A.na * A.width;
    if (A.priv) {
        for (int64_t q = threadIdx.x; q < tot; q += blockDim.x) sh[q] = T(0);
        __syncthreads();
    }
    T* dst = A.priv ? sh : A.asbar;
    const I* is = static_cast<const I*>(A.is);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < A.nj; j += stride) {
        const int64_t i = ldi(is, j);
        const bool in = i >= 0 && i < A.na;
        const T xb = __ldcs(A.xsbar + j);
        if (A.g == ADPAR_G_GATHER) {
            if (in) acc_add(dst + i, xb);
        } else if (A.g == ADPAR_G_SCALE) {
            const T w = __ldcs(A.ws + j);
            T wb = T(0);
            if (in) {
                acc_add(dst + i, w * xb);
                wb = __ldg(A.as + i) * xb;
            }
            if (A.wsbar) {
                if (A.acc_w) A.wsbar[j] += wb;
                else A.wsbar[j] = wb;
            }
        } else {  // SQDIST_ROW, rows of `width`
            for (int k = 0; k < A.width; ++k) {
                const T w = A.ws[j * A.width + k];
                T wb = T(0);
                if (in) {
                    const T diff = w - __ldg(A.as + i * A.width + k);
                    acc_add(dst + i * A.width + k, T(-2) * diff * xb);
                    wb = T(2) * diff * xb;
                }
                if (A.wsbar) {
                    if (A.acc_w) A.wsbar[j * A.width + k] += wb;
                    else A.wsbar[j * A.width + k] = wb;
                }
            }
        }
    }
    if (A.priv) {
        __syncthreads();
        for (int64_t q = threadIdx.x; q < tot; q += blockDim.x)
            if (sh[q] != T(0)) atomicAdd(A.asbar + q, sh[q]);
    }
}

// primal of scatter (Sec. 5.3's forward sweep): xs_saved[j] = ys[is_j]
// (optional), then ys[is_j] = vs[j], in place
template <class T, class I>
__global__ void __launch_bounds__(kBlk) scatter_fwd_kernel(int64_t n, int64_t m, const I* is, const T* vs, T* ys,
                                                          T* xs_saved) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += stride) {
        const int64_t k = ldi(is, j);
        if (k < 0 || k >= n) {
            if (xs_saved) xs_saved[j] = T(0);
            continue;
        }
        if (xs_saved) xs_saved[j] = ys[k];
        ys[k] = __ldcs(vs + j);
    }
}

// primal of map: xs[j] = g(as[is_j, :], ws[j, :]) (0 for an index out of range)
template <class T, class I>
__global__ void __launch_bounds__(kBlk) map_fwd_kernel(int g, int64_t nj, int64_t na, int width, const T* as,
                                                      const I* is, const T* ws, T* xs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nj; j += stride) {
        const int64_t i = ldi(is, j);
        T x = T(0);
        if (i >= 0 && i < na) {
            if (g == ADPAR_G_GATHER) {
                x = __ldg(as + i);
            } else if (g == ADPAR_G_SCALE) {
                x = __ldg(as + i) * ws[j];
            } else {
                for (int k = 0; k < width; ++k) {
                    const T d = ws[j * width + k] - __ldg(as + i * width + k);
                    x += d * d;
                }
            }
        }
        xs[j] = x;
    }
}

template <class T>
__global__ void zero_kernel(T* p, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) p[i] = T(0);
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 132;
}

constexpr size_t kPrivBytes = 48 * 1024;

}  // namespace
}  // namespace adpar

extern "C" int adpar_vjp_scatter(int dtype, int64_t n, int64_t m, const void* is, int itype,
                                 void* ysbar_inout, void* vsbar, void* ys_restore, const void* xs_saved,
                                 uint32_t flags, void* stream) {
    using namespace adpar;
    if (n < 0 || m < 0) return ADPAR_ERR_INVALID;
    if (dtype != ADPAR_F32 && dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)(ADPAR_ACCUMULATE | ADPAR_SCATTER_RESTORE)) return ADPAR_ERR_UNSUPPORTED;
    const bool restore = (flags & ADPAR_SCATTER_RESTORE) != 0;
    if (m > 0 && (!is || !vsbar || !ysbar_inout)) return ADPAR_ERR_INVALID;
    if (restore && m > 0 && (!ys_restore || !xs_saved)) return ADPAR_ERR_INVALID;
    const void* ptrs[] = {is, ysbar_inout, vsbar, ys_restore, xs_saved};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    if (m == 0) return ADPAR_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m / 4 + kBlk) / kBlk, (int64_t)sm_count() * 8));
    const int acc = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    void* ys = restore ? ys_restore : nullptr;
#define ADPAR_SCATTER(T, I)                                                                               \
    scatter_vjp_kernel<T, I><<<grid, kBlk, 0, s>>>(n, m, static_cast<const I*>(is), static_cast<T*>(ysbar_inout), \
                                                   static_cast<T*>(vsbar), static_cast<T*>(ys),              \
                                                   static_cast<const T*>(xs_saved), acc)
    if (dtype == ADPAR_F32) {
        if (itype == ADPAR_I32) ADPAR_SCATTER(float, int32_t); else ADPAR_SCATTER(float, int64_t);
    } else {
        if (itype == ADPAR_I32) ADPAR_SCATTER(double, int32_t); else ADPAR_SCATTER(double, int64_t);
    }
#undef ADPAR_SCATTER
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_vjp_map_acc(int gfun, int dtype, int64_t nj, int64_t na, int width, const void* as,
                                 const void* is, int itype, const void* ws, const void* xsbar, void* asbar,
                                 void* wsbar, uint32_t flags, void* work, size_t work_bytes, void* stream) {
    using namespace adpar;
    (void)work;
    (void)work_bytes;
    if (nj < 0 || na < 0 || width < 1) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_GATHER && gfun != ADPAR_G_SCALE && gfun != ADPAR_G_SQDIST_ROW) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_SQDIST_ROW && width != 1) return ADPAR_ERR_INVALID;
    if (dtype != ADPAR_F32 && dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    if (nj > 0 && (!is || !xsbar || !asbar)) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_GATHER && nj > 0 && (!ws || !as)) return ADPAR_ERR_INVALID;
    const void* ptrs[] = {as, is, ws, xsbar, asbar, wsbar};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool acc = (flags & ADPAR_ACCUMULATE) != 0;
    const size_t esz = dtype == ADPAR_F64 ? 8 : 4;
    const int64_t tot = na * width;
    const int sms = sm_count();
    // asbar is an accumulator: without ADPAR_ACCUMULATE it starts from zero
    if (!acc && tot > 0) {
        const int gz = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, (int64_t)sms * 8));
        if (dtype == ADPAR_F32) zero_kernel<float><<<gz, 256, 0, s>>>(static_cast<float*>(asbar), tot);
        else zero_kernel<double><<<gz, 256, 0, s>>>(static_cast<double*>(asbar), tot);
    }
    if (nj == 0) return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
    const bool priv = (size_t)tot * esz <= kPrivBytes;
    const size_t shm = priv ? (size_t)tot * esz : 0;
    const int64_t blocks = priv ? std::min<int64_t>((nj + kBlk * 16 - 1) / (kBlk * 16), (int64_t)sms * 2)
                                : std::min<int64_t>((nj + kBlk - 1) / kBlk, (int64_t)sms * 8);
    const int grid = (int)std::max<int64_t>(1, blocks);
#define ADPAR_MAPACC(T, I)                                                                   \
    do {                                                                                     \
        MapAccArgs<T> A{gfun, nj, na, width, static_cast<const T*>(as), is,                  \
                        static_cast<const T*>(ws), static_cast<const T*>(xsbar),             \
                        static_cast<T*>(asbar), static_cast<T*>(wsbar), acc ? 1 : 0, priv ? 1 : 0}; \
        map_acc_kernel<T, I><<<grid, kBlk, shm, s>>>(A);                                     \
    } while (0)
    if (dtype == ADPAR_F32) {
        if (itype == ADPAR_I32) ADPAR_MAPACC(float, int32_t); else ADPAR_MAPACC(float, int64_t);
    } else {
        if (itype == ADPAR_I32) ADPAR_MAPACC(double, int32_t); else ADPAR_MAPACC(double, int64_t);
    }
#undef ADPAR_MAPACC
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_scatter(int dtype, int64_t n, int64_t m, const void* is, int itype, const void* vs,
                             void* ys_inout, void* xs_saved_out, void* stream) {
    using namespace adpar;
    if (n < 0 || m < 0) return ADPAR_ERR_INVALID;
    if (dtype != ADPAR_F32 && dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if (m > 0 && (!is || !vs || !ys_inout)) return ADPAR_ERR_INVALID;
    const void* ptrs[] = {is, vs, ys_inout, xs_saved_out};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    if (m == 0) return ADPAR_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m + kBlk - 1) / kBlk, (int64_t)sm_count() * 8));
#define ADPAR_SCAT_FWD(T, I)                                                                                   \
    scatter_fwd_kernel<T, I><<<grid, kBlk, 0, s>>>(n, m, static_cast<const I*>(is), static_cast<const T*>(vs), \
                                                   static_cast<T*>(ys_inout), static_cast<T*>(xs_saved_out))
    if (dtype == ADPAR_F32) {
        if (itype == ADPAR_I32) ADPAR_SCAT_FWD(float, int32_t); else ADPAR_SCAT_FWD(float, int64_t);
    } else {
        if (itype == ADPAR_I32) ADPAR_SCAT_FWD(double, int32_t); else ADPAR_SCAT_FWD(double, int64_t);
    }
#undef ADPAR_SCAT_FWD
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_map_acc(int gfun, int dtype, int64_t nj, int64_t na, int width, const void* as,
                             const void* is, int itype, const void* ws, void* xs_out, void* stream) {
    using namespace adpar;
    if (nj < 0 || na < 0 || width < 1) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_GATHER && gfun != ADPAR_G_SCALE && gfun != ADPAR_G_SQDIST_ROW) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_SQDIST_ROW && width != 1) return ADPAR_ERR_INVALID;
    if (dtype != ADPAR_F32 && dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if (nj > 0 && (!is || !xs_out || !as)) return ADPAR_ERR_INVALID;
    if (gfun != ADPAR_G_GATHER && nj > 0 && !ws) return ADPAR_ERR_INVALID;
    const void* ptrs[] = {as, is, ws, xs_out};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    if (nj == 0) return ADPAR_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nj + kBlk - 1) / kBlk, (int64_t)sm_count() * 8));
#define ADPAR_MAP_FWD(T, I)                                                                                    \
    map_fwd_kernel<T, I><<<grid, kBlk, 0, s>>>(gfun, nj, na, width, static_cast<const T*>(as),                  \
                                               static_cast<const I*>(is), static_cast<const T*>(ws),            \
                                               static_cast<T*>(xs_out))
    if (dtype == ADPAR_F32) {
        if (itype == ADPAR_I32) ADPAR_MAP_FWD(float, int32_t); else ADPAR_MAP_FWD(float, int64_t);
    } else {
        if (itype == ADPAR_I32) ADPAR_MAP_FWD(double, int32_t); else ADPAR_MAP_FWD(double, int64_t);
    }
#undef ADPAR_MAP_FWD
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}
