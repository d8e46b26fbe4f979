// VJP of reduce_by_index (Sec. 5.1.2) for +, min, max and *.
//
// The primal is the semantic loop  hs[inds_i] (.)= vals_i  with indices
// outside [0, m) ignored.  Following Sec. 5.1.2, the return sweep is the
// reduce rule of Sec. 5.1.1 per bin with ybar replaced by hsbar[inds_i]:
//   +        valsbar_i = hsbar[inds_i]: one gather pass, no recompute.
//   min/max  recompute per bin the extremum and its LOWEST index, then
//            valsbar[argidx_b] = hsbar_b and 0 elsewhere.
//   *        recompute per bin (zero count, lowest zero index, scaled
//            product of the nonzeros), then the three cases per element.
//
// Recompute pass (min/max/*): a grid-stride loop whose per-block bin state
// for the bin range [0, H) lives in shared memory (H = min(m, capacity));
// bins at or above H go straight to global atomics (L2).  Low bin ids are
// the hot ones of rank-ordered skewed data such as Zipf, so their
// contention stays on-chip.  The extremum of a bin is one 64-bit word:
//   max: (orderkey(v) << 32) | ~i   under atomicMax,
//   min: (orderkey(v) << 32) |  i   under atomicMin,
// where orderkey maps FP32 bits monotonically to unsigned (+0 and -0 equal),
// so ties resolve to the lowest index exactly.  FP64 values take two
// passes: the extremum key (64-bit atomic), then the lowest index holding it.
#include <algorithm>
#include <math_constants.h>

#include "common.cuh"
#include "prod.cuh"
#include "scan_ops.cuh"

namespace adpar {
namespace {

constexpr int kHistBlock = 512;
constexpr int kHistSmemKeys = 8192;  // 64 KB of 64-bit bin words per block

__device__ __forceinline__ uint32_t orderkey_f32(float f) {
    uint32_t u = __float_as_uint(f);
    if (u == 0x80000000u) u = 0u;  // -0 == +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_orderkey_f32(uint32_t k) {
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}
__device__ __forceinline__ unsigned long long orderkey_f64(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    if (u == 0x8000000000000000ull) u = 0ull;
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_orderkey_f64(unsigned long long k) {
    const unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

template <class I>
__device__ __forceinline__ int64_t ld_index(const I* p, int64_t i) {
    return (int64_t)__ldcs(p + i);
}

struct HistArgs {
    int op;
    int64_t n, m;
    const void* vals;
    const void* inds;
    const void* hsbar;
    void* valsbar;
    void* hs_out;
    int64_t* argidx_out;
    adpar_prod_aux* bin_aux;
    int8_t* vsign;
    int accumulate;
    int logdomain;
    int primal_only;  // forward operator only: valsbar is not touched
    WsHeader* hdr;
    unsigned long long* key;  // [m] extremum words (min/max), FP64 pass-1 keys
    unsigned long long* idx;  // [m] lowest index (FP64 min/max pass 2)
    double* pm;               // [m] * : mantissa of the nonzero product
    long long* pe;            // [m] * : its exponent
    unsigned int* pz;         // [m] * : zero count
    long long* pf;            // [m] * : lowest zero index
    struct BinQ* binq;        // [m] * with FP32 values: per-bin factor of the adjoint
    int q62;                  // * with FP32 values: pm holds the fixed-point mantissa
    // * : per-block partial states of the shared-memory bins [0, hw), merged
    // by hist_prod_merge_kernel ([blocks][hw] each)
    int64_t hw;
    unsigned long long* part_m;
    long long* part_e;
    long long* part_f;
    unsigned* part_z;
};

// Per-bin factor of the * adjoint for FP32 values (value domain): (qm, qe)
// with P_nz * hsbar_b = qm * 2^qe, qm an FP32 mantissa (0.5 <= |qm| < 1),
// and `sel`: -1 = the bin has no zero (every element gets P_nz/v_i * hsbar),
// an index = the bin's only zero (that element gets P_nz * hsbar), -2 =
// nothing (two or more zeros, or hsbar_b = 0).
struct alignas(16) BinQ {
    float qm;
    int qe;
    long long sel;
};

__global__ void hist_init_kernel(HistArgs A, unsigned long long key_empty) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t0 < 64) reinterpret_cast<uint32_t*>(A.hdr)[t0] = 0u;
    for (int64_t b = t0; b < A.m; b += stride) {
        if (A.key) A.key[b] = key_empty;
        if (A.idx) A.idx[b] = 0xffffffffffffffffull;
        if (A.pm) {  // the neutral product: fixed point 2^62 * 2^-62, or 0.5 * 2^1
            if (A.q62) reinterpret_cast<unsigned long long*>(A.pm)[b] = 1ull << 62;
            else A.pm[b] = 0.5;
            A.pe[b] = A.q62 ? 0 : 1;
            A.pz[b] = 0u;
            A.pf[b] = INT64_MAX;
        }
    }
}

// ------------------------------------------------------------------ +
// valsbar_i = hsbar[inds_i] (in range) -- the whole VJP is this gather.
template <class T, class I>
__global__ void __launch_bounds__(kHistBlock) hist_add_vjp_kernel(HistArgs A) {
    const I* inds = static_cast<const I*>(A.inds);
    const T* hsbar = static_cast<const T*>(A.hsbar);
    T* vb = static_cast<T*>(A.valsbar);
    constexpr int V = 4;  // 4 elements per thread step
    const int64_t nv = A.n / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += stride) {
        T o[V];
        int64_t b[V];
#pragma unroll
        for (int j = 0; j < V; ++j) b[j] = ld_index(inds, v * V + j);
#pragma unroll
        for (int j = 0; j < V; ++j) o[j] = (b[j] >= 0 && b[j] < A.m) ? __ldg(hsbar + b[j]) : T(0);
        if (A.accumulate) {
#pragma unroll
            for (int j = 0; j < V; ++j) o[j] += vb[v * V + j];
        }
        if constexpr (sizeof(T) == 4) {
            __stcs(reinterpret_cast<float4*>(vb + v * V), make_float4(o[0], o[1], o[2], o[3]));
        } else {
            __stcs(reinterpret_cast<double2*>(vb + v * V), make_double2(o[0], o[1]));
            __stcs(reinterpret_cast<double2*>(vb + v * V + 2), make_double2(o[2], o[3]));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < A.n - nv * V) {
        const int64_t i = nv * V + threadIdx.x;
        const int64_t b = ld_index(inds, i);
        const T o = (b >= 0 && b < A.m) ? hsbar[b] : T(0);
        vb[i] = A.accumulate ? vb[i] + o : o;
    }
}

// primal of + (only when hs_out is asked for): hs[b] += vals_i
template <class T, class I>
__global__ void __launch_bounds__(kHistBlock) hist_add_primal_kernel(HistArgs A) {
    extern __shared__ unsigned char smem_raw[];
    T* sh = reinterpret_cast<T*>(smem_raw);
    const int H = (int)std::min<int64_t>(A.m, kHistSmemKeys);
    for (int b = threadIdx.x; b < H; b += blockDim.x) sh[b] = T(0);
    __syncthreads();
    const I* inds = static_cast<const I*>(A.inds);
    const T* vals = static_cast<const T*>(A.vals);
    T* hs = static_cast<T*>(A.hs_out);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int64_t b = ld_index(inds, i);
        if (b < 0 || b >= A.m) continue;
        const T v = __ldcs(vals + i);
        if (b < H) atomicAdd(sh + b, v);
        else atomicAdd(hs + b, v);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < H; b += blockDim.x)
        if (sh[b] != T(0)) atomicAdd(hs + b, sh[b]);
}

__global__ void fill_zero_kernel(void* p, int64_t nbytes) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nv = nbytes / 16;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += stride)
        reinterpret_cast<uint4*>(p)[v] = make_uint4(0, 0, 0, 0);
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nbytes - nv * 16) static_cast<unsigned char*>(p)[nv * 16 + t] = 0;
}

// ------------------------------------------------------------ min / max
// FP32: one recompute pass with packed words; fuses the zero fill of valsbar.
template <class I, bool MAX>
__global__ void __launch_bounds__(kHistBlock) hist_arg_f32_kernel(HistArgs A) {
    extern __shared__ unsigned char smem_raw[];
    unsigned long long* sh = reinterpret_cast<unsigned long long*>(smem_raw);
    const unsigned long long empty = MAX ? 0ull : 0xffffffffffffffffull;
    const int H = (int)std::min<int64_t>(A.m, kHistSmemKeys);
    for (int b = threadIdx.x; b < H; b += blockDim.x) sh[b] = empty;
    __syncthreads();
    const I* inds = static_cast<const I*>(A.inds);
    const float* vals = static_cast<const float*>(A.vals);
    float* vb = static_cast<float*>(A.valsbar);
    const bool fill = !A.accumulate && !A.primal_only;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int64_t b = ld_index(inds, i);
        if (fill) __stcs(vb + i, 0.0f);
        if (b < 0 || b >= A.m) continue;
        const uint32_t k = orderkey_f32(__ldcs(vals + i));
        const unsigned long long w = ((unsigned long long)k << 32) |
                                     (MAX ? (unsigned long long)(~(uint32_t)i) : (unsigned long long)(uint32_t)i);
        if (b < H) {
            if (MAX) atomicMax(sh + b, w); else atomicMin(sh + b, w);
        } else {
            if (MAX) atomicMax(A.key + b, w); else atomicMin(A.key + b, w);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < H; b += blockDim.x) {
        const unsigned long long w = sh[b];
        if (w != empty) {
            if (MAX) atomicMax(A.key + b, w); else atomicMin(A.key + b, w);
        }
    }
}

// FP64, pass 1: extremum key per bin (+ zero fill of valsbar)
template <class I, bool MAX>
__global__ void __launch_bounds__(kHistBlock) hist_arg_f64_key_kernel(HistArgs A) {
    const I* inds = static_cast<const I*>(A.inds);
    const double* vals = static_cast<const double*>(A.vals);
    double* vb = static_cast<double*>(A.valsbar);
    const bool fill = !A.accumulate && !A.primal_only;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int64_t b = ld_index(inds, i);
        if (fill) vb[i] = 0.0;
        if (b < 0 || b >= A.m) continue;
        const unsigned long long k = orderkey_f64(vals[i]);
        if (MAX) atomicMax(A.key + b, k); else atomicMin(A.key + b, k);
    }
}
// FP64, pass 2: lowest index whose value equals the bin's extremum
template <class I>
__global__ void __launch_bounds__(kHistBlock) hist_arg_f64_idx_kernel(HistArgs A) {
    const I* inds = static_cast<const I*>(A.inds);
    const double* vals = static_cast<const double*>(A.vals);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int64_t b = ld_index(inds, i);
        if (b < 0 || b >= A.m) continue;
        if (orderkey_f64(vals[i]) == A.key[b]) atomicMin(A.idx + b, (unsigned long long)i);
    }
}

// per bin: valsbar[argidx_b] (+)= hsbar_b; hs_out, argidx_out
template <class T, bool MAX>
__global__ void hist_arg_finish_kernel(HistArgs A) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const T* hsbar = static_cast<const T*>(A.hsbar);
    T* vb = static_cast<T*>(A.valsbar);
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < A.m; b += stride) {
        int64_t arg = -1;
        T val = MAX ? -pos_inf<T>() : pos_inf<T>();
        if constexpr (sizeof(T) == 4) {
            const unsigned long long w = A.key[b];
            const unsigned long long empty = MAX ? 0ull : 0xffffffffffffffffull;
            if (w != empty) {
                const uint32_t lo = (uint32_t)w;
                arg = (int64_t)(MAX ? (uint32_t)~lo : lo);
                val = (T)from_orderkey_f32((uint32_t)(w >> 32));
            }
        } else {
            const unsigned long long ix = A.idx[b];
            if (ix != 0xffffffffffffffffull) {
                arg = (int64_t)ix;
                val = (T)from_orderkey_f64(A.key[b]);
            }
        }
        if (arg >= 0 && !A.primal_only) vb[arg] = A.accumulate ? vb[arg] + hsbar[b] : hsbar[b];
        if (A.hs_out) static_cast<T*>(A.hs_out)[b] = val;
        if (A.argidx_out) A.argidx_out[b] = arg;
    }
}

// ------------------------------------------------------------------ *
// pm *= mi under a CAS loop (global bins, FP64 values).  When the mantissa
// drops below 2^-823 it is scaled up by 2^900 through its exponent bits and
// the exponent counter takes -900 (both exact); the check reads the IEEE
// exponent field, so the loop does one FP64 multiply per attempt.
__device__ __forceinline__ void mul_into(double* pm, long long* pe, double mi, long long ei) {
    atomicAdd(reinterpret_cast<unsigned long long*>(pe), (unsigned long long)ei);
    unsigned long long* p = reinterpret_cast<unsigned long long*>(pm);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(p), assumed;
    long long shift;
    do {
        assumed = old;
        long long nb = __double_as_longlong(__longlong_as_double((long long)assumed) * mi);
        shift = 0;
        if (((nb >> 52) & 0x7ff) < 200) {  // below 2^-823 (products of mantissas are never 0)
            nb += 900LL << 52;
            shift = -900;
        }
        old = atomicCAS(p, assumed, (unsigned long long)nb);
    } while (old != assumed);
    if (shift) atomicAdd(reinterpret_cast<unsigned long long*>(pe), (unsigned long long)shift);
}

// global CAS: *pM = *pM * mv (fixed point); the exponent gets ev + the increment
__device__ __forceinline__ void q62_mul24_into(unsigned long long* pM, long long* pE, unsigned mv, int ev) {
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(pM), assumed, nb;
    int de;
    do {
        assumed = old;
        nb = q62_mul24(assumed, mv, de);
        old = atomicCAS(pM, assumed, nb);
    } while (old != assumed);
    atomicAdd(reinterpret_cast<unsigned long long*>(pE), (unsigned long long)(long long)(ev + de));
}

// A bin's recomputed state, for either representation.
template <class T>
__device__ __forceinline__ void read_bin(const HistArgs& A, int64_t b, double& mm, int64_t& e, unsigned& nz) {
    const unsigned z = A.pz[b];
    if constexpr (sizeof(T) == 4) {
        nz = z & 0x7fffffffu;
        q62_to_pow2(reinterpret_cast<const unsigned long long*>(A.pm)[b], A.pe[b], z >> 31, mm, e);
    } else {
        nz = z;
        int64_t ee;
        split_pow2(A.pm[b], mm, ee);
        e = A.pe[b] + ee;
    }
}

// Bin tiers of the * recompute:
//   [0, H)       warp-private copies: lanes of a warp that hit the same bin
//                are serialised into rounds (__match_any_sync picks one
//                leader per bin per round), so every update is a plain
//                read-modify-write of shared memory, however skewed;
//   [H, H + H2)  one block-shared copy updated with shared-memory CAS;
//   the rest     global CAS (L2).
// Rank-ordered skewed data (Zipf) keeps its hot bins in the first tiers.
// FP32 values use the fixed-point state above in every tier; FP64 values
// an FP64 mantissa in [0.5, 1) and an integer exponent.
constexpr int kProdWarpBins = 256;
constexpr int kProdBlockBins = 2048;
constexpr int kProdBlock = 256;
constexpr int kProdMaxGrid = 1024;  // rows of the partial-state arrays

// One warp-private bin: mantissa (fixed point, or FP64 bits), exponent and
// zero count (with the sign parity in bit 31 for fixed point), read and
// written as one 16-byte word.
struct alignas(16) WBin {
    unsigned long long M;
    int E;
    unsigned Z;
};

template <class T, class I>
__global__ void __launch_bounds__(kProdBlock, 4) hist_prod_kernel(HistArgs A) {
    extern __shared__ unsigned char smem_raw[];
    constexpr bool kQ = sizeof(T) == 4;
    constexpr int NW = kProdBlock / 32;
    const int H = (int)std::min<int64_t>(A.m, kProdWarpBins);
    WBin* wb = reinterpret_cast<WBin*>(smem_raw);              // [NW][H]
    long long* wf = reinterpret_cast<long long*>(wb + NW * H);  // [NW][H] lowest zero index
    const int H2 = (int)std::max<int64_t>(0, std::min<int64_t>(A.m - H, kProdBlockBins));
    unsigned long long* bm = reinterpret_cast<unsigned long long*>(wf + NW * H);  // [H2] block-shared tier
    long long* be = reinterpret_cast<long long*>(bm + H2);
    long long* bf = be + H2;
    unsigned int* bz = reinterpret_cast<unsigned int*>(bf + H2);
    const unsigned long long one = kQ ? kQ62One : (unsigned long long)__double_as_longlong(0.5);
    const int e_one = kQ ? 0 : 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < NW * H; q += blockDim.x) {
        wb[q] = WBin{one, e_one, 0u};
        wf[q] = INT64_MAX;
    }
    for (int q = threadIdx.x; q < H2; q += blockDim.x) {
        bm[q] = one;
        be[q] = e_one;
        bf[q] = INT64_MAX;
        bz[q] = 0u;
    }
    __syncthreads();
    WBin* myb = wb + warp * H;
    long long* myf = wf + warp * H;
    unsigned long long* gM = reinterpret_cast<unsigned long long*>(A.pm);
    // FP32 values: each lane keeps the nonzero factors of bins [0, kHot) in
    // registers (the hottest bins of rank-ordered skewed data), so they take
    // no part in the warp's serialised rounds; merged once at the end
    constexpr int kHot = kQ ? 8 : 0;
    const int hot = (int)std::min<int64_t>(A.m, kHot);
    unsigned long long cM[kHot > 0 ? kHot : 1];
    int cE[kHot > 0 ? kHot : 1];
    unsigned cS = 0;  // sign parities, bit k for bin k
#pragma unroll
    for (int k = 0; k < kHot; ++k) {
        cM[k] = kQ62One;
        cE[k] = 0;
    }
    const I* inds = static_cast<const I*>(A.inds);
    const T* vals = static_cast<const T*>(A.vals);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (A.n + stride - 1) / stride;  // same trip count in every lane
    for (int64_t it = 0; it < nround; ++it) {
        const int64_t i = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        int64_t b = -1;
        T v = T(0);
        if (i < A.n) {
            b = ld_index(inds, i);
            v = __ldcs(vals + i);
        }
        const bool zero = v == T(0);
        // the element's factor: fixed point (sg, mv, ev) or FP64 (mi, ei)
        unsigned sg = 0, mv = 0;
        int ev = 0;
        double mi = 0.5;
        int64_t ei = 1;
        const bool in = b >= 0 && b < A.m;
        if (in && !zero) {
            if constexpr (kQ) split_f32_int(v, sg, mv, ev);
            else split_pow2(v, mi, ei);
        }
        if (in && b >= H && b < H + H2) {  // warm bins: block-shared, shared-memory CAS
            const int q = (int)(b - H);
            if (zero) {
                atomicAdd(bz + q, 1u);
                atomicMin(bf + q, (long long)i);
            } else if constexpr (kQ) {
                q62_mul24_into(bm + q, be + q, mv, ev);
                if (sg) atomicXor(bz + q, 0x80000000u);
            } else {
                mul_into(reinterpret_cast<double*>(bm + q), be + q, mi, ei);
            }
        } else if (in && b >= H + H2) {  // cold bins: global atomics
            if (zero) {
                atomicAdd(A.pz + b, 1u);
                atomicMin(A.pf + b, (long long)i);
            } else if constexpr (kQ) {
                q62_mul24_into(gM + b, A.pe + b, mv, ev);
                if (sg) atomicXor(A.pz + b, 0x80000000u);
            } else {
                mul_into(A.pm + b, A.pe + b, mi, ei);
            }
        }
        bool pending = in && b < H;
        if constexpr (kHot > 0) {
            if (pending && !zero && b < hot) {
#pragma unroll
                for (int k = 0; k < kHot; ++k) {
                    if (b == k) {
                        int de;
                        cM[k] = q62_mul24(cM[k], mv, de);
                        cE[k] += ev + de;
                        cS ^= sg << k;
                    }
                }
                pending = false;
            }
        }
        const unsigned key = pending ? (unsigned)b : (0x80000000u | (unsigned)lane);
        while (__any_sync(0xffffffffu, pending)) {
            const unsigned grp = __match_any_sync(0xffffffffu, pending ? key : (0x80000000u | (unsigned)lane));
            const bool leader = pending && lane == __ffs(grp) - 1;
            if (leader) {
                WBin x = myb[b];
                if (zero) {
                    x.Z += 1;
                    if (i < myf[b]) myf[b] = i;
                } else if constexpr (kQ) {
                    int de;
                    x.M = q62_mul24(x.M, mv, de);
                    x.E += ev + de;
                    x.Z ^= sg << 31;
                } else {
                    double mm = __longlong_as_double((long long)x.M) * mi;
                    int64_t e2 = 0;
                    renorm(mm, e2);
                    x.M = (unsigned long long)__double_as_longlong(mm);
                    x.E += (int)(ei + e2);
                }
                myb[b] = x;
                pending = false;
            }
            __syncwarp();
        }
    }
    // the lanes' register bins: a shuffle tree per bin, then lane 0 folds
    // the warp's product into its shared-memory copy
    if constexpr (kHot > 0) {
#pragma unroll
        for (int k = 0; k < kHot; ++k) {
            unsigned long long M = cM[k];
            long long E = cE[k];
            unsigned sgn = (cS >> k) & 1u;
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const unsigned long long M2 = __shfl_xor_sync(0xffffffffu, M, off);
                const long long E2 = __shfl_xor_sync(0xffffffffu, E, off);
                int de;
                M = q62_mul(M, M2, de);
                E += E2 + de - 62;
                sgn ^= __shfl_xor_sync(0xffffffffu, sgn, off);
            }
            if (lane == 0 && k < hot) {
                WBin x = myb[k];
                int de;
                x.M = q62_mul(x.M, M, de);
                x.E += (int)(E + de - 62);
                x.Z ^= sgn << 31;
                myb[k] = x;
            }
        }
    }
    __syncthreads();
    // this block's state of the shared-memory bins goes to its partial row
    // (no global atomics); hist_prod_merge_kernel combines the rows
    const int64_t row = (int64_t)blockIdx.x * A.hw;
    for (int q = threadIdx.x; q < H; q += blockDim.x) {
        unsigned nz = 0, sign = 0;
        long long first = INT64_MAX;
        unsigned long long M;
        long long E;
        if constexpr (kQ) {
            M = kQ62One;
            E = 0;
        } else {
            M = (unsigned long long)__double_as_longlong(0.5);
            E = 1;
        }
        for (int w = 0; w < NW; ++w) {
            const WBin x = wb[w * H + q];
            nz += x.Z & 0x7fffffffu;
            sign ^= x.Z >> 31;
            first = std::min(first, wf[w * H + q]);
            if constexpr (kQ) {
                int de;
                M = q62_mul(M, x.M, de);
                E += x.E + de - 62;
            } else {
                double mm = __longlong_as_double((long long)M) * __longlong_as_double((long long)x.M);
                int64_t e2 = 0;
                renorm(mm, e2);
                M = (unsigned long long)__double_as_longlong(mm);
                E += x.E + e2;
            }
        }
        A.part_m[row + q] = M;
        A.part_e[row + q] = E;
        A.part_z[row + q] = nz | (sign << 31);
        A.part_f[row + q] = first;
    }
    for (int q = threadIdx.x; q < H2; q += blockDim.x) {
        A.part_m[row + H + q] = bm[q];
        A.part_e[row + H + q] = be[q];
        A.part_z[row + H + q] = bz[q];
        A.part_f[row + H + q] = bf[q];
    }
}

// Combines the per-block partial states of the shared-memory bins: one
// warp per bin, lanes take every 32nd block row, then a shuffle tree.  It is
// the only writer of these bins' global state.
template <class T>
__global__ void hist_prod_merge_kernel(HistArgs A, int rows) {
    constexpr bool kQ = sizeof(T) == 4;
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= A.hw) return;
    unsigned long long M = kQ ? kQ62One : (unsigned long long)__double_as_longlong(0.5);
    long long E = kQ ? 0 : 1;
    unsigned nz = 0, sign = 0;
    long long first = INT64_MAX;
    auto comb = [](unsigned long long& M1, long long& E1, unsigned long long M2, long long E2) {
        if constexpr (kQ) {
            int de;
            M1 = q62_mul(M1, M2, de);
            E1 += E2 + de - 62;
        } else {
            double mm = __longlong_as_double((long long)M1) * __longlong_as_double((long long)M2);
            int64_t e2 = 0;
            renorm(mm, e2);
            M1 = (unsigned long long)__double_as_longlong(mm);
            E1 += E2 + e2;
        }
    };
    for (int r = lane; r < rows; r += 32) {
        const int64_t k = (int64_t)r * A.hw + b;
        comb(M, E, A.part_m[k], A.part_e[k]);
        const unsigned z = A.part_z[k];
        nz += z & 0x7fffffffu;
        sign ^= z >> 31;
        first = std::min(first, A.part_f[k]);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const unsigned long long M2 = __shfl_xor_sync(0xffffffffu, M, off);
        const long long E2 = __shfl_xor_sync(0xffffffffu, E, off);
        comb(M, E, M2, E2);
        nz += __shfl_xor_sync(0xffffffffu, nz, off);
        sign ^= __shfl_xor_sync(0xffffffffu, sign, off);
        first = std::min(first, (long long)__shfl_xor_sync(0xffffffffu, first, off));
    }
    if (lane == 0) {
        A.pm[b] = __longlong_as_double((long long)M);  // the bits, in either representation
        A.pe[b] = E;
        A.pz[b] = kQ ? (nz | (sign << 31)) : nz;
        A.pf[b] = first;
    }
}

// per bin outputs of *: hs_out (product rounded to T) and aux
template <class T>
__global__ void hist_prod_bins_kernel(HistArgs A) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < A.m; b += stride) {
        double mm;
        int64_t e;
        unsigned nz;
        read_bin<T>(A, b, mm, e, nz);
        if (A.hs_out) static_cast<T*>(A.hs_out)[b] = nz ? T(0) : (T)ldexp_clamped(mm, e);
        if (A.bin_aux) {
            adpar_prod_aux x;
            x.nzero = nz;
            x.first_zero = nz ? A.pf[b] : -1;
            x.exp2 = e;
            x.mant = mm;
            x.log_abs_nz = log(fabs(mm)) + (double)e * 0.69314718055994530942;
            x.sign = mm > 0 ? 1 : -1;
            x.reserved = 0;
            A.bin_aux[b] = x;
        }
    }
}

// per element: the cases of Sec. 5.1.1 with ybar = hsbar[inds_i]
template <class T, class I>
__global__ void __launch_bounds__(kHistBlock) hist_prod_vjp_kernel(HistArgs A) {
    const I* inds = static_cast<const I*>(A.inds);
    const T* vals = static_cast<const T*>(A.vals);
    const T* hsbar = static_cast<const T*>(A.hsbar);
    T* vb = static_cast<T*>(A.valsbar);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int64_t b = ld_index(inds, i);
        const bool in = b >= 0 && b < A.m;
        double c = 0.0, lg = -CUDART_INF;
        int sg = 0;
        if (in) {
            const double yb = (double)hsbar[b];
            double mm;
            int64_t e;
            unsigned nz;
            read_bin<T>(A, b, mm, e, nz);
            if (yb != 0.0 && (nz == 0 || (nz == 1 && A.pf[b] == i))) {
                double ym;
                int64_t ye;
                split_pow2(yb, ym, ye);
                const int spy = (mm > 0 ? 1 : -1) * (yb > 0 ? 1 : -1);
                if (nz == 0) {
                    const double v = (double)vals[i];
                    if (A.logdomain) {
                        lg = log(fabs(mm)) + (double)e * 0.69314718055994530942 - log(fabs(v)) + log(fabs(yb));
                        sg = spy * (v > 0 ? 1 : -1);
                    } else {
                        double mi;
                        int64_t ei;
                        split_pow2(v, mi, ei);
                        c = scale_pow2(mm * ym * recip_mantissa(mi), e + ye - ei);
                    }
                } else {
                    if (A.logdomain) {
                        lg = log(fabs(mm)) + (double)e * 0.69314718055994530942 + log(fabs(yb));
                        sg = spy;
                    } else {
                        c = ldexp_clamped(mm * ym, e + ye);
                    }
                }
            }
        }
        if (A.logdomain) {
            vb[i] = (T)lg;
            if (A.vsign) A.vsign[i] = (int8_t)sg;
        } else if (A.accumulate) {
            if (in) vb[i] = (T)((double)vb[i] + c);
        } else {
            vb[i] = (T)c;
        }
    }
}

// per-bin factors of the FP32 value-domain adjoint (see BinQ)
template <class T>
__global__ void hist_prod_binq_kernel(HistArgs A) {
    const T* hsbar = static_cast<const T*>(A.hsbar);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < A.m; b += stride) {
        BinQ q;
        q.qm = 0.0f;
        q.qe = 0;
        q.sel = -2;
        const double yb = (double)hsbar[b];
        double mm;
        int64_t ee;
        unsigned nz;
        read_bin<T>(A, b, mm, ee, nz);
        if (yb != 0.0 && nz <= 1) {
            double ym, m2;
            int64_t ye, e2;
            split_pow2(yb, ym, ye);
            split_pow2(mm * ym, m2, e2);  // in [0.25, 1): one more split
            float qf = (float)m2;        // rounding may reach 1.0
            int64_t e = ee + ye + e2;
            if (fabsf(qf) >= 1.0f) {
                qf *= 0.5f;
                e += 1;
            }
            q.qm = qf;
            q.qe = (int)(e > (1 << 30) ? (1 << 30) : (e < -(1 << 30) ? -(1 << 30) : e));
            q.sel = nz == 0 ? -1 : A.pf[b];
        }
        A.binq[b] = q;
    }
}

// per element, FP32 values in the value domain: the three cases of
// Sec. 5.1.1 from the bin's factor, in FP32 arithmetic with the exponent
// kept apart (qm / m_v, then 2^(qe - e_v) applied to the exponent field)
template <class I>
__global__ void __launch_bounds__(kHistBlock) hist_prod_vjp_f32_kernel(HistArgs A) {
    const I* inds = static_cast<const I*>(A.inds);
    const float* vals = static_cast<const float*>(A.vals);
    float* vb = static_cast<float*>(A.valsbar);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int64_t b = ld_index(inds, i);
        const bool in = b >= 0 && b < A.m;
        float c = 0.0f;
        if (in) {
            const BinQ q = A.binq[b];
            if (q.sel == -1) {
                float mv;
                int ev;
                split_pow2_f32m(__ldcs(vals + i), mv, ev);
                c = scale_pow2f(q.qm * __frcp_rn(mv), (int64_t)q.qe - ev);
            } else if (q.sel == i) {
                c = scale_pow2f(q.qm, (int64_t)q.qe);
            }
        }
        if (A.accumulate) {
            if (in) vb[i] += c;
        } else {
            vb[i] = c;
        }
    }
}

// ------------------------------------------------------------ host side
struct HistLayout {
    size_t off_key, off_idx, off_pm, off_pe, off_pz, off_pf, off_binq, off_part_m, off_part_e, off_part_f,
        off_part_z, total;
};

HistLayout hist_layout(int op, int dtype, int64_t m) {
    HistLayout L{};
    size_t o = sizeof(WsHeader);
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    if (op == ADPAR_OP_MIN || op == ADPAR_OP_MAX) {
        L.off_key = o; o = round_up(o + mm * 8, 256);
        if (dtype == ADPAR_F64) { L.off_idx = o; o = round_up(o + mm * 8, 256); }
    } else if (op == ADPAR_OP_MUL) {
        L.off_pm = o; o = round_up(o + mm * 8, 256);
        L.off_pe = o; o = round_up(o + mm * 8, 256);
        L.off_pf = o; o = round_up(o + mm * 8, 256);
        L.off_pz = o; o = round_up(o + mm * 4, 256);
        if (dtype == ADPAR_F32) { L.off_binq = o; o = round_up(o + mm * sizeof(BinQ), 256); }
        const size_t hw = (size_t)std::min<int64_t>(m, kProdWarpBins + kProdBlockBins);
        const size_t np = hw * (size_t)kProdMaxGrid;
        L.off_part_m = o; o = round_up(o + np * 8, 256);
        L.off_part_e = o; o = round_up(o + np * 8, 256);
        L.off_part_f = o; o = round_up(o + np * 8, 256);
        L.off_part_z = o; o = round_up(o + np * 4, 256);
    }
    L.total = o;
    return L;
}

int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 132;
}

template <class T, class I>
int run_hist(HistArgs A, cudaStream_t s) {
    const int sms = num_sms();
    const int gridN = (int)std::max<int64_t>(1, std::min<int64_t>((A.n + kHistBlock - 1) / kHistBlock, (int64_t)sms * 4));
    const int gridM = (int)std::max<int64_t>(1, std::min<int64_t>((A.m + 255) / 256, (int64_t)sms * 8));
    const int op = A.op;
    if (op != ADPAR_OP_ADD) {
        const unsigned long long empty = op == ADPAR_OP_MAX ? 0ull : 0xffffffffffffffffull;
        hist_init_kernel<<<gridM, 256, 0, s>>>(A, empty);
    }
    switch (op) {
    case ADPAR_OP_ADD: {
        if (A.hs_out) {
            fill_zero_kernel<<<gridM, 256, 0, s>>>(A.hs_out, A.m * (int64_t)sizeof(T));
            const size_t sh = (size_t)std::min<int64_t>(A.m, kHistSmemKeys) * sizeof(T);
            hist_add_primal_kernel<T, I><<<gridN, kHistBlock, sh, s>>>(A);
        }
        if (A.primal_only) break;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((A.n / 4 + kHistBlock - 1) / kHistBlock, (int64_t)sms * 8));
        hist_add_vjp_kernel<T, I><<<g, kHistBlock, 0, s>>>(A);
        break;
    }
    case ADPAR_OP_MIN:
    case ADPAR_OP_MAX: {
        const bool mx = op == ADPAR_OP_MAX;
        if constexpr (sizeof(T) == 4) {
            const size_t sh = (size_t)std::min<int64_t>(A.m, kHistSmemKeys) * 8;
            if (mx) hist_arg_f32_kernel<I, true><<<gridN, kHistBlock, sh, s>>>(A);
            else hist_arg_f32_kernel<I, false><<<gridN, kHistBlock, sh, s>>>(A);
        } else {
            if (mx) hist_arg_f64_key_kernel<I, true><<<gridN, kHistBlock, 0, s>>>(A);
            else hist_arg_f64_key_kernel<I, false><<<gridN, kHistBlock, 0, s>>>(A);
            hist_arg_f64_idx_kernel<I><<<gridN, kHistBlock, 0, s>>>(A);
        }
        if (mx) hist_arg_finish_kernel<T, true><<<gridM, 256, 0, s>>>(A);
        else hist_arg_finish_kernel<T, false><<<gridM, 256, 0, s>>>(A);
        break;
    }
    case ADPAR_OP_MUL: {
        const int64_t h1 = std::min<int64_t>(A.m, kProdWarpBins);
        const int64_t h2 = std::max<int64_t>(0, std::min<int64_t>(A.m - h1, kProdBlockBins));
        const size_t sh = (size_t)h1 * 24 * (kProdBlock / 32) + (size_t)h2 * 28;
        const int gridP = (int)std::max<int64_t>(
            1, std::min<int64_t>((A.n + kProdBlock - 1) / kProdBlock, std::min<int64_t>(sms * 4, kProdMaxGrid)));
        A.hw = h1 + h2;
        hist_prod_kernel<T, I><<<gridP, kProdBlock, sh, s>>>(A);
        if (A.hw > 0) hist_prod_merge_kernel<T><<<(unsigned)((A.hw * 32 + 255) / 256), 256, 0, s>>>(A, gridP);
        if (A.hs_out || A.bin_aux) hist_prod_bins_kernel<T><<<gridM, 256, 0, s>>>(A);
        if (A.primal_only) break;
        if (sizeof(T) == 4 && !A.logdomain) {
            hist_prod_binq_kernel<T><<<gridM, 256, 0, s>>>(A);
            hist_prod_vjp_f32_kernel<I><<<gridN, kHistBlock, 0, s>>>(A);
        } else {
            hist_prod_vjp_kernel<T, I><<<gridN, kHistBlock, 0, s>>>(A);
        }
        break;
    }
    default:
        return ADPAR_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

constexpr int kMaxDev = 64;
bool smem_configured[kMaxDev] = {};

template <class T, class I>
void configure_smem() {
    // the recompute kernels use up to 64 KB of dynamic shared memory
    cudaFuncSetAttribute(hist_add_primal_kernel<T, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(hist_prod_kernel<T, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    if constexpr (sizeof(T) == 4) {
        cudaFuncSetAttribute(hist_arg_f32_kernel<I, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
        cudaFuncSetAttribute(hist_arg_f32_kernel<I, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    }
}

}  // namespace

size_t hist_workspace_size(adpar_opdesc d, int64_t m) {
    if (m < 0 || (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64)) return (size_t)-1;
    if (d.op != ADPAR_OP_ADD && d.op != ADPAR_OP_MUL && d.op != ADPAR_OP_MIN && d.op != ADPAR_OP_MAX)
        return (size_t)-1;
    return hist_layout(d.op, d.dtype, m).total;
}

}  // namespace adpar

namespace adpar {
namespace {
int hist_impl(adpar_opdesc d, int64_t n, int64_t m, const void* vals, const void* inds, int itype,
              const void* hsbar, void* valsbar, void* hs_out, int64_t* argidx_out, adpar_prod_aux* bin_aux_out,
              int8_t* valsbar_sign, uint32_t flags, void* work, size_t work_bytes, void* stream,
              bool primal_only) {
    if (n < 0 || m < 0 || d.width != 1) return ADPAR_ERR_INVALID;
    if (d.op != ADPAR_OP_ADD && d.op != ADPAR_OP_MUL && d.op != ADPAR_OP_MIN && d.op != ADPAR_OP_MAX)
        return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)(ADPAR_ACCUMULATE | ADPAR_PROD_LOGDOMAIN)) return ADPAR_ERR_UNSUPPORTED;
    const bool logd = (flags & ADPAR_PROD_LOGDOMAIN) != 0;
    if (logd && (d.op != ADPAR_OP_MUL || (flags & ADPAR_ACCUMULATE))) return ADPAR_ERR_UNSUPPORTED;
    if (valsbar_sign && !logd) return ADPAR_ERR_INVALID;
    if ((d.op == ADPAR_OP_MIN || d.op == ADPAR_OP_MAX) && d.dtype == ADPAR_F32 && n > 0xffffffffLL)
        return ADPAR_ERR_UNSUPPORTED;  // the packed word holds a 32-bit index
    if (n > 0 && (!inds || (!valsbar && !primal_only))) return ADPAR_ERR_INVALID;
    if (n > 0 && m > 0 && !hsbar && !primal_only) return ADPAR_ERR_INVALID;
    if (primal_only && m > 0 && !hs_out) return ADPAR_ERR_INVALID;
    if (n > 0 && !vals && (d.op != ADPAR_OP_ADD || hs_out)) return ADPAR_ERR_INVALID;
    const void* ptrs[] = {vals, inds, hsbar, valsbar, hs_out};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    const HistLayout L = hist_layout(d.op, d.dtype, m);
    if (!work || work_bytes < L.total || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    if (n == 0 && m == 0) return ADPAR_OK;
    HistArgs A{};
    A.op = d.op;
    A.n = n;
    A.m = m;
    A.vals = vals;
    A.inds = inds;
    A.hsbar = hsbar;
    A.valsbar = valsbar;
    A.hs_out = hs_out;
    A.argidx_out = argidx_out;
    A.bin_aux = bin_aux_out;
    A.vsign = valsbar_sign;
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    A.logdomain = logd ? 1 : 0;
    A.primal_only = primal_only ? 1 : 0;
    char* w = static_cast<char*>(work);
    A.hdr = reinterpret_cast<WsHeader*>(w);
    if (L.off_key) A.key = reinterpret_cast<unsigned long long*>(w + L.off_key);
    if (L.off_idx) A.idx = reinterpret_cast<unsigned long long*>(w + L.off_idx);
    if (L.off_binq) A.binq = reinterpret_cast<BinQ*>(w + L.off_binq);
    if (L.off_part_m) {
        A.part_m = reinterpret_cast<unsigned long long*>(w + L.off_part_m);
        A.part_e = reinterpret_cast<long long*>(w + L.off_part_e);
        A.part_f = reinterpret_cast<long long*>(w + L.off_part_f);
        A.part_z = reinterpret_cast<unsigned*>(w + L.off_part_z);
    }
    A.q62 = (d.op == ADPAR_OP_MUL && d.dtype == ADPAR_F32) ? 1 : 0;
    if (L.off_pm) {
        A.pm = reinterpret_cast<double*>(w + L.off_pm);
        A.pe = reinterpret_cast<long long*>(w + L.off_pe);
        A.pz = reinterpret_cast<unsigned int*>(w + L.off_pz);
        A.pf = reinterpret_cast<long long*>(w + L.off_pf);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return ADPAR_ERR_CUDA;
    if (!smem_configured[dev]) {  // once per device (idempotent if two threads race here)
        configure_smem<float, int32_t>();
        configure_smem<float, int64_t>();
        configure_smem<double, int32_t>();
        configure_smem<double, int64_t>();
        smem_configured[dev] = true;
    }
    if (d.dtype == ADPAR_F32)
        return itype == ADPAR_I32 ? run_hist<float, int32_t>(A, s) : run_hist<float, int64_t>(A, s);
    return itype == ADPAR_I32 ? run_hist<double, int32_t>(A, s) : run_hist<double, int64_t>(A, s);
}
}  // namespace
}  // namespace adpar

extern "C" int adpar_vjp_hist(adpar_opdesc d, int64_t n, int64_t m, const void* vals, const void* inds,
                              int itype, const void* hsbar, void* valsbar, void* hs_out,
                              int64_t* argidx_out, adpar_prod_aux* bin_aux_out, int8_t* valsbar_sign,
                              uint32_t flags, void* work, size_t work_bytes, void* stream) {
    return adpar::hist_impl(d, n, m, vals, inds, itype, hsbar, valsbar, hs_out, argidx_out, bin_aux_out,
                            valsbar_sign, flags, work, work_bytes, stream, false);
}

extern "C" int adpar_hist(adpar_opdesc d, int64_t n, int64_t m, const void* vals, const void* inds, int itype,
                          void* hs_out, int64_t* argidx_out, adpar_prod_aux* bin_aux_out, void* work,
                          size_t work_bytes, void* stream) {
    return adpar::hist_impl(d, n, m, vals, inds, itype, nullptr, nullptr, hs_out, argidx_out, bin_aux_out,
                            nullptr, 0u, work, work_bytes, stream, true);
}
