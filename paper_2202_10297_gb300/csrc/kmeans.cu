// k-means cost and its gradient in C, the nested-parallel program of
// Sec. 7.4 with squared distances:
//   loss = sum_i min_k ||x_i - c_k||^2,
//   Cbar[k] = 2 ybar (cnt_k c_k - sum_{i: argmin_i = k} x_i).
// Its VJP is the min-reduce rule of Sec. 5.1.1 (the adjoint goes to the
// argmin only) followed by the accumulator of Sec. 5.4 on the free array C,
// which Sec. 6.1 turns into a reduction; here that reduction is a per-block
// histogram of rows (counts and row sums per centroid) in shared memory.
//
// One persistent kernel, one CTA per SM, 18 warps:
//   warp 0     TMEM allocation and release; TMA producer: X tiles of 128
//              rows x 32 FP32 (128-byte rows, 128-byte swizzle) into a
//              4-stage ring; C (k x 32) once.
//   warp 1     MMA issuer: acc = X_tile C^T - |c|^2 / 2 with tcgen05.mma
//              kind::tf32 (M = 128, N = k, K = 32 in four steps of 8, then
//              one more K step with A rows (1, 1, 0, ..) and B rows holding
//              -|c_k|^2 / 2 split into two TF32 parts) into one of two TMEM
//              accumulators (2 x 256 columns).  The distance is
//              |x|^2 - 2 acc_k, so the argmin is the argmax of acc.
//   warps 2-17 epilogue, two groups of 8 warps taking alternate tiles (group
//              p reads accumulator p and synchronises on its own named
//              barrier), tiles handed out by a global ticket through the
//              producer.  In a group, two threads per row (warp w reads the
//              TMEM lanes of quarter w % 4, and every other 32-column chunk):
//              a tcgen05.ld.red pass (the load's own max reduction, sm_103a)
//              for the largest acc_k; the row's maximum from its two
//              threads; a second pass listing every centroid within the
//              TF32 error bound of it (one compare per value), before the
//              accumulator is released.  Then, with warp w of the group
//              taking 16 rows, 8 at a time, four adjacent lanes per row (8
//              coordinates each): the candidates' distances recomputed in
//              FP32; if two remain within the FP32 bound, FP64 (the oracle's
//              own arithmetic) decides, ties to the lowest k; the loss term
//              (the argmin's distance) and, for the gradient, the row added
//              into shared-memory row sums.
// Every mbarrier wait is bounded; a timeout is recorded in the workspace
// and the kernel drains its copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <math_constants.h>

#include <algorithm>

#include "common.cuh"
#include "tc.cuh"

namespace adpar {
namespace {

constexpr int KM_THREADS = 576;  // warps 0-1 roles, 2-17 epilogue
constexpr int KM_EPI = 512;      // epilogue threads
constexpr int KM_PG = 2;         // epilogue groups, taking alternate tiles
constexpr int KM_PG_THREADS = KM_EPI / KM_PG;
constexpr int KM_TPR = 2;        // threads per row in a group's scan passes
constexpr int KM_STAGES = 4;
constexpr int KM_D = 32;
constexpr int KM_KMAX = 256;
constexpr int KM_TILE = 128;
constexpr uint32_t KM_X_BYTES = KM_TILE * KM_D * 4;  // 16 KB
constexpr int KM_SLOTS = 4;                    // candidate slots per scanning thread
constexpr int KM_MAXCAND = KM_TPR * KM_SLOTS;  // per row

// shared memory layout (offsets from a 1024-aligned base)
constexpr uint32_t OFF_C = 0;                                           // 32 KB
constexpr uint32_t OFF_X = OFF_C + KM_KMAX * KM_D * 4;                  // 4 x 16 KB
constexpr int KM_SUM_LD = KM_D + 1;  // row-sum stride: rows of other centroids on other banks
// the |c|^2 term as one more K step of 8: A rows (1, 1, 0, ..), B rows
// (h_k, l_k, 0, ..) with h_k + l_k = -|c_k|^2 / 2, in the same swizzled layout
constexpr uint32_t OFF_AX = OFF_X + KM_STAGES * KM_X_BYTES;             // 16 KB
constexpr uint32_t OFF_BX = OFF_AX + KM_TILE * 128;                     // 32 KB
constexpr uint32_t OFF_SUM = OFF_BX + KM_KMAX * 128;                    // 33 KB
constexpr uint32_t OFF_CNT = OFF_SUM + KM_KMAX * KM_SUM_LD * 4;         // 1 KB
constexpr uint32_t OFF_CN2 = OFF_CNT + KM_KMAX * 4;                     // 1 KB
// per epilogue group:
constexpr uint32_t OFF_CAND = OFF_CN2 + KM_KMAX * 4;                    // 8 KB: [2][128][8] candidate slots
constexpr uint32_t OFF_MAX = OFF_CAND + KM_PG * KM_TILE * KM_MAXCAND * 4;  // 2 KB: [2][2][128] partial row maxima
constexpr uint32_t OFF_NC = OFF_MAX + KM_PG * KM_TPR * KM_TILE * 4;     // 2 KB: [2][128][2] candidate counts
constexpr uint32_t OFF_XN = OFF_NC + KM_PG * KM_TILE * KM_TPR * 4;      // 2 KB: [2][2][128] partial |x|^2
constexpr uint32_t OFF_BAR = OFF_XN + KM_PG * KM_TPR * KM_TILE * 4;     // barriers
constexpr uint32_t NBAR = 2 * KM_STAGES + 5;
constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
constexpr uint32_t KM_SMEM = OFF_MISC + 64 + 1024;  // + alignment slack
static_assert(OFF_X % 1024 == 0 && KM_X_BYTES % 1024 == 0 && OFF_AX % 1024 == 0 && OFF_BX % 1024 == 0,
              "swizzled tiles need 1024-byte alignment");
static_assert(KM_SMEM <= 227 * 1024, "shared memory of one CTA");

struct KmArgs {
    int64_t N;
    int k;
    const float* X;
    const float* C;
    const float* ybar;
    float* loss_out;
    int32_t* argmin_out;
    float* Cbar;
    int accumulate;
    int64_t ntiles;
    WsHeader* hdr;
    double* loss_acc;
    float* gsum;  // [k * 32]
    float* gcnt;  // [k]
};

// element j of row r of a 128-byte-swizzled tile (rows of 32 FP32)
__device__ __forceinline__ float sw_elem(const float* tile, int r, int j) {
    const int chunk = (j >> 2) ^ (r & 7);
    return tile[r * 32 + chunk * 4 + (j & 3)];
}
// ||x - c_kc||^2 in FP32 for one row: each of four adjacent lanes sums the
// squares of its 8 coordinates (x0, x1: the row's chunks 2 g, 2 g + 1), then
// two butterfly steps add the partial sums, so that the four lanes hold the
// same value.  All lanes of the warp call it.
__device__ __forceinline__ float cand_dist_f32(const float4& x0, const float4& x1, const float* sC, int kc, int g) {
    const float* crow = sC + kc * KM_D;
    const float4 c0 = *reinterpret_cast<const float4*>(crow + (((2 * g) ^ (kc & 7)) * 4));
    const float4 c1 = *reinterpret_cast<const float4*>(crow + (((2 * g + 1) ^ (kc & 7)) * 4));
    // two chains of four (chunk 2 g, chunk 2 g + 1), then their sum
    float d, s = 0.f, u = 0.f;
    d = x0.x - c0.x; s = fmaf(d, d, s);
    d = x1.x - c1.x; u = fmaf(d, d, u);
    d = x0.y - c0.y; s = fmaf(d, d, s);
    d = x1.y - c1.y; u = fmaf(d, d, u);
    d = x0.z - c0.z; s = fmaf(d, d, s);
    d = x1.z - c1.z; u = fmaf(d, d, u);
    d = x0.w - c0.w; s = fmaf(d, d, s);
    d = x1.w - c1.w; u = fmaf(d, d, u);
    s += u;
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    return s;
}

// the oracle's FP64 arithmetic: s += (x - c)^2 with no fused multiply-add
__device__ __noinline__ double exact_f64(const float* xt, int r, const float* sC, int kc) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const double d = __dsub_rn((double)sw_elem(xt, r, j), (double)sw_elem(sC, kc, j));
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    return s;
}

// N == 0: the empty sum
__global__ void km_empty_kernel(float* loss_out, float* Cbar, int kd, int accumulate) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && loss_out) *loss_out = 0.f;
    if (Cbar && !accumulate)
        for (int q = t; q < kd; q += gridDim.x * blockDim.x) Cbar[q] = 0.f;
}

// The 16 epilogue warps (warps 2-17) form two groups of 8 (256 threads)
// that take alternate tiles, group p synchronising on named barrier 1 + p.
// epi_any is a barrier that also ORs a predicate over the group, so a
// decision to stop is taken by all of its threads together.
__device__ __forceinline__ void epi_sync(int pg) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + pg), "r"(KM_PG_THREADS) : "memory");
}
__device__ __forceinline__ bool epi_any(int pg, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred o, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(1 + pg), "r"(KM_PG_THREADS)
        : "memory");
    return r != 0;
}

__global__ void km_init_kernel(KmArgs A) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 64) reinterpret_cast<uint32_t*>(A.hdr)[t] = 0u;
    if (t == 0) *A.loss_acc = 0.0;
    for (int q = t; q < A.k * KM_D; q += gridDim.x * blockDim.x) A.gsum[q] = 0.f;
    for (int q = t; q < A.k; q += gridDim.x * blockDim.x) A.gcnt[q] = 0.f;
}

__global__ void __launch_bounds__(KM_THREADS, 1)
    kmeans_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmC, KmArgs A) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment by an offset into the shared array, so that every
    // access below stays a shared-memory access (a round trip through an
    // integer would leave the compiler generic loads, stores and atomics)
    unsigned char* base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    float* sC = reinterpret_cast<float*>(base + OFF_C);
    float* sX = reinterpret_cast<float*>(base + OFF_X);
    float* s_sum = reinterpret_cast<float*>(base + OFF_SUM);
    float* s_cnt = reinterpret_cast<float*>(base + OFF_CNT);
    float* s_cn2 = reinterpret_cast<float*>(base + OFF_CN2);
    int* s_cand = reinterpret_cast<int*>(base + OFF_CAND);
    float* s_max = reinterpret_cast<float*>(base + OFF_MAX);
    float* sAX = reinterpret_cast<float*>(base + OFF_AX);
    float* sBX = reinterpret_cast<float*>(base + OFF_BX);
    int* s_ncnt = reinterpret_cast<int*>(base + OFF_NC);
    float* s_xn = reinterpret_cast<float*>(base + OFF_XN);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + OFF_BAR);
    uint64_t* x_full = bars;
    uint64_t* x_empty = bars + KM_STAGES;
    uint64_t* t_full = bars + 2 * KM_STAGES;
    uint64_t* t_empty = bars + 2 * KM_STAGES + 2;
    uint64_t* c_bar = bars + 2 * KM_STAGES + 4;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(base + OFF_MISC);
    volatile int* s_abort = reinterpret_cast<volatile int*>(base + OFF_MISC + 4);
    volatile int* s_never = reinterpret_cast<volatile int*>(base + OFF_MISC + 12);  // stays 0
    float* s_cmax = reinterpret_cast<float*>(base + OFF_MISC + 8);
    // the tile in each X stage (-1: no more tiles), written by the producer
    // before the stage's x_full phase completes
    volatile int* s_tile = reinterpret_cast<volatile int*>(base + OFF_MISC + 16);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = A.k;
    const bool want_grad = A.Cbar != nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < KM_STAGES; ++s) {
            tc::mbar_init(&x_full[s], 1);
            tc::mbar_init(&x_empty[s], KM_PG_THREADS / 32);  // one arrival per warp of a group
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&t_full[b], 1);
            tc::mbar_init(&t_empty[b], 1);  // one arrival after the epilogue barrier
        }
        tc::mbar_init(c_bar, 1);
        *s_abort = 0;
        *s_never = 0;
        tc::fence_mbar_init();
        tc::tma_prefetch_desc(&tmX);
        tc::tma_prefetch_desc(&tmC);
    }
    for (int q = threadIdx.x; q < k * KM_SUM_LD; q += KM_THREADS) s_sum[q] = 0.f;
    float cm = 0.f;
    for (int c = threadIdx.x; c < k; c += KM_THREADS) {
        float s = 0.f;
        for (int j = 0; j < KM_D; ++j) {
            const float v = __ldg(A.C + c * KM_D + j);
            s = fmaf(v, v, s);
        }
        s_cn2[c] = s;
        s_cnt[c] = 0.f;
        cm = fmaxf(cm, s);
        // -|c|^2 / 2 = h + l: h keeps the 10 mantissa bits TF32 reads, l
        // (exact in FP32) the rest, of which TF32 keeps 10 more
        const float hv = -0.5f * s;
        const float h = __uint_as_float(__float_as_uint(hv) & 0xFFFFE000u);
        sBX[c * KM_D + ((0 ^ (c & 7)) << 2) + 0] = h;
        sBX[c * KM_D + ((0 ^ (c & 7)) << 2) + 1] = hv - h;
    }
    // the rest of the two extra operands: A rows (1, 1, 0, ..), B rows of
    // zeros past the first two elements (and past k)
    for (int q = threadIdx.x; q < KM_TILE * KM_D; q += KM_THREADS) {
        const int r = q / KM_D, j = q % KM_D;  // logical element j of row r
        sAX[r * KM_D + (((j >> 2) ^ (r & 7)) << 2) + (j & 3)] = j < 2 ? 1.f : 0.f;
    }
    for (int q = threadIdx.x; q < KM_KMAX * KM_D; q += KM_THREADS) {
        const int r = q / KM_D, j = q % KM_D;
        if (j >= 2 || r >= k) sBX[r * KM_D + (((j >> 2) ^ (r & 7)) << 2) + (j & 3)] = 0.f;
    }
    tc::fence_proxy_async();  // generic-proxy writes, read by the tensor core
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, off));
    if (threadIdx.x == 0) *s_cmax = 0.f;
    if (warp == 0) {
        tc::tmem_alloc(s_tmem, 512);
        tc::fence_before_sync();
    }
    __syncthreads();
    if (lane == 0) atomicMax(reinterpret_cast<int*>(s_cmax), __float_as_int(cm));  // cm >= 0
    tc::fence_after_sync();
    __syncthreads();
    const uint32_t tmem = *s_tmem;
    const float cmax = sqrtf(*s_cmax);

    int issued = 0, committed = 0;
    if (warp == 0) {
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(c_bar, (uint32_t)(k * KM_D * 4));
            tc::tma_load_2d(sC, &tmC, 0, 0, c_bar);
            // tiles by a global ticket (CTAs ran at different speeds: static
            // shares left the slowest SMs 40% behind the median); once the
            // tickets run out, one end marker for each epilogue group
            int ended = 0;
            for (int i = 0; ended < KM_PG; ++i) {
                const int s = i % KM_STAGES;
                if (i >= KM_STAGES && !tc::mbar_wait(&x_empty[s], ((i / KM_STAGES) - 1) & 1, s_abort)) {
                    *s_abort = 1;
                    break;
                }
                int64_t t = ended ? A.ntiles : (int64_t)atomicAdd(&A.hdr->ticket[0], 1u);
                if (t >= A.ntiles) {
                    s_tile[s] = -1;
                    tc::mbar_arrive(&x_full[s]);  // no copy: the phase completes at once
                    ++ended;
                } else {
                    s_tile[s] = (int)t;
                    tc::mbar_arrive_expect_tx(&x_full[s], KM_X_BYTES);
                    tc::tma_load_2d(sX + s * (KM_X_BYTES / 4), &tmX, 0, (int)(t * KM_TILE), &x_full[s]);
                }
                issued = i + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32_m128((uint32_t)k);
            const uint64_t bdesc = tc::desc_sw128_kmajor(tc::smem_u32(sC));
            const uint64_t axdesc = tc::desc_sw128_kmajor(tc::smem_u32(sAX));
            const uint64_t bxdesc = tc::desc_sw128_kmajor(tc::smem_u32(sBX));
            if (!tc::mbar_wait(c_bar, 0, s_abort)) *s_abort = 1;
            for (int i = 0; !*s_abort; ++i) {
                const int s = i % KM_STAGES, b = i & 1;
                if (!tc::mbar_wait(&x_full[s], (i / KM_STAGES) & 1, s_abort)) { *s_abort = 1; break; }
                if (s_tile[s] < 0) break;  // no more tiles
                if (i >= 2 && !tc::mbar_wait(&t_empty[b], ((i >> 1) - 1) & 1, s_abort)) { *s_abort = 1; break; }
                tc::fence_after_sync();
                const uint64_t adesc = tc::desc_sw128_kmajor(tc::smem_u32(sX + s * (KM_X_BYTES / 4)));
#pragma unroll
                for (int kk = 0; kk < KM_D / 8; ++kk)  // K step of 8 TF32 = 32 bytes = +2 in the address field
                    tc::mma_tf32(tmem + (uint32_t)(b * 256), adesc + 2 * kk, bdesc + 2 * kk, idesc, kk > 0);
                // + (-|c_k|^2 / 2): the accumulator holds x.c_k - |c_k|^2 / 2
                tc::mma_tf32(tmem + (uint32_t)(b * 256), axdesc, bxdesc, idesc, 1u);
                tc::mma_commit(&t_full[b]);
                committed = i + 1;
            }
        }
    } else if (warp >= 2) {
        // 16 epilogue warps in two groups; group pg takes the tiles i with
        // i % 2 == pg, in accumulator pg.  Warp w reads the TMEM lanes of
        // quarter w % 4; the two warps of a group on a quarter split the
        // 32-column chunks (q % 2 == grp)
        const int ew = warp - 2;
        const int pg = ew >> 3, gw = ew & 7;
        const int quarter = warp & 3, grp = gw >> 2;
        const int r = quarter * 32 + lane;  // row of the tile == TMEM lane
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const int nq = k / 32;
        float* g_max = s_max + pg * KM_TPR * KM_TILE;
        float* g_xn = s_xn + pg * KM_TPR * KM_TILE;
        int* g_ncnt = s_ncnt + pg * KM_TILE * KM_TPR;
        int* g_cand = s_cand + pg * KM_TILE * KM_MAXCAND;
        // loss: FP32 sum with Neumaier's compensation of the FP32-certified
        // distances, FP64 sum of those FP64 decided (FP64 instructions, on a
        // GB300 one warp instruction per 16 cycles per SM, stay off the
        // per-row path)
        float lsum = 0.f, lcomp = 0.f;
        double loss64 = 0.0;
        if (!tc::mbar_wait(c_bar, 0, s_abort)) *s_abort = 1;
        for (int i = pg;; i += KM_PG) {
            const int s = i % KM_STAGES, b = pg;
            // the stage's tile (or the end marker), then the accumulator.  A
            // wait that gives up, or the end marker, makes the warp skip its
            // reads of the accumulator; the first barrier of the tile then
            // takes every thread of the group out together
            const bool okx = __all_sync(0xffffffffu, tc::mbar_wait(&x_full[s], (i / KM_STAGES) & 1, s_abort));
            const int64_t t = s_tile[s];
            const bool more = okx && t >= 0;
            const bool ok = more && __all_sync(0xffffffffu, tc::mbar_wait(&t_full[b], (i >> 1) & 1, s_abort));
            if (!okx || (more && !ok)) *s_abort = 1;
            tc::fence_after_sync();
            const float* xt = sX + s * (KM_X_BYTES / 4);
            {
                // this thread's half of |x|^2 (coordinates 16 grp .. 16 grp + 15)
                float xp = 0.f;
#pragma unroll
                for (int c = 4 * grp; c < 4 * grp + 4; ++c) {
                    const float4 v = *reinterpret_cast<const float4*>(xt + r * 32 + ((c ^ (r & 7)) * 4));
                    xp = fmaf(v.x, v.x, xp);
                    xp = fmaf(v.y, v.y, xp);
                    xp = fmaf(v.z, v.z, xp);
                    xp = fmaf(v.w, v.w, xp);
                }
                g_xn[grp * KM_TILE + r] = xp;
            }
            const uint32_t tb = tmem + lane_base + (uint32_t)(b * 256);

            // pass 1: the largest x.c_k - |c_k|^2 / 2 (the smallest distance)
            // of this thread's chunks, from the TMEM load's own max reduction
            float m1 = -CUDART_INF_F;
            for (int q = grp; ok && q < nq; q += KM_TPR) {
                uint32_t va[32];
                float cm;
                __syncwarp();
                tc::tmem_ld32_max(tb + (uint32_t)(q * 32), va, &cm);
                tc::tmem_ld_wait();
                m1 = fmaxf(m1, cm);
            }
            g_max[grp * KM_TILE + r] = m1;
            if (epi_any(pg, !ok)) break;  // every thread of the group leaves together
            float amax = g_max[r], xn2 = g_xn[r];
#pragma unroll
            for (int g = 1; g < KM_TPR; ++g) {
                amax = fmaxf(amax, g_max[g * KM_TILE + r]);
                xn2 += g_xn[g * KM_TILE + r];
            }
            const float xn = sqrtf(xn2);
            // the distance is |x|^2 - 2 acc_k.  |acc~_k - acc_k| <= |S~ - S| +
            // rounding <= 2^-9 |x| |c_k| (TF32 keeps 10 mantissa bits of each
            // operand of S = x.c_k) plus FP32 terms, the norm term within
            // 2^-21 |c_k|^2; the true argmin is within twice that of the
            // computed maximum, and tol is 4x that bound
            const float tol = 8.0e-3f * xn * cmax + 1.0e-5f * (cmax * cmax + xn * cmax) + 1e-20f;
            const float thr = amax - tol;
            // pass 2: candidates, every column within tol of the row's maximum
            // (this thread's first KM_SLOTS in its own slots; a count above
            // KM_SLOTS sends the row to the all-centroids path)
            int ncnt = 0;
            int* slots = g_cand + r * KM_MAXCAND + grp * KM_SLOTS;
            for (int q = grp; q < nq; q += KM_TPR) {
                uint32_t va[32];
                __syncwarp();
                tc::tmem_ld32(tb + (uint32_t)(q * 32), va);
                tc::tmem_ld_wait();
                // four independent OR chains (one long chain waits on itself)
                uint32_t mk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int j = 0; j < 32; ++j) mk[j & 3] |= (__uint_as_float(va[j]) >= thr ? 1u : 0u) << j;
                uint32_t mask = (mk[0] | mk[1]) | (mk[2] | mk[3]);
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    if (ncnt < KM_SLOTS) slots[ncnt] = q * 32 + j;
                    ++ncnt;
                }
            }
            g_ncnt[r * KM_TPR + grp] = ncnt;
            // every thread of the group has read the accumulator past this barrier
            tc::fence_before_sync();
            epi_sync(pg);
            if (gw == 0 && lane == 0) tc::mbar_arrive(&t_empty[b]);

            // certification, loss and row sums: warp gw takes rows 16 gw ..
            // 16 gw + 15, 8 at a time, four adjacent lanes per row, lane g of
            // a row the coordinates 8 g .. 8 g + 7
#pragma unroll 1
            for (int rd = 0; rd < 2; ++rd) {
                const int rc = gw * 16 + rd * 8 + (lane >> 2), g = lane & 3;
                const float* xrow = xt + rc * KM_D;
                const float4 x0 = *reinterpret_cast<const float4*>(xrow + (((2 * g) ^ (rc & 7)) * 4));
                const float4 x1 = *reinterpret_cast<const float4*>(xrow + (((2 * g + 1) ^ (rc & 7)) * 4));
                // the row's candidates: scanning thread 0's first min(count,
                // KM_SLOTS) slots, then thread 1's; a count above KM_SLOTS
                // makes every centroid a candidate
                const int2 cn = *reinterpret_cast<const int2*>(g_ncnt + rc * KM_TPR);
                const bool ovf = max(cn.x, cn.y) > KM_SLOTS;
                const int p1 = min(cn.x, KM_SLOTS);
                const int cnt = ovf ? k : p1 + min(cn.y, KM_SLOTS);
                const int* rslots = g_cand + rc * KM_MAXCAND;
                auto cand_at = [&](int c) -> int {
                    if (ovf) return c;
                    return c < p1 ? rslots[c] : rslots[KM_SLOTS + c - p1];
                };
                int cmax_w = cnt;
#pragma unroll
                for (int off = 4; off < 32; off <<= 1) cmax_w = max(cmax_w, __shfl_xor_sync(0xffffffffu, cmax_w, off));
                // FP32 distances of the candidates (a sum of four 8-term
                // partial sums), two at a time; the smallest, its centroid,
                // the second smallest
                float emin = CUDART_INF_F, e2 = CUDART_INF_F;
                int kmin = 0;
                auto take = [&](float e, int kc) {
                    if (e < emin) {
                        e2 = emin;
                        emin = e;
                        kmin = kc;
                    } else if (e < e2) {
                        e2 = e;
                    }
                };
                for (int c = 0; c < cmax_w; c += 2) {
                    const bool h0 = c < cnt, h1 = c + 1 < cnt;
                    const int k0 = h0 ? cand_at(c) : 0;
                    const int k1 = h1 ? cand_at(c + 1) : 0;
                    const float e0 = cand_dist_f32(x0, x1, sC, k0, g);
                    const float e1 = cand_dist_f32(x0, x1, sC, k1, g);
                    if (h0) take(e0, k0);
                    if (h1) take(e1, k1);
                }
                // FP32 separates the smallest when no other candidate is
                // within the FP32 bound of it; else FP64 (the oracle's own
                // arithmetic) decides among those within it, ties to the lowest k
                const float u32 = emin + 4.0e-6f * emin + 1e-30f;
                const bool need64 = e2 - 4.0e-6f * e2 <= u32;
                int best = kmin;
                const int64_t row = t * KM_TILE + rc;
                if (__any_sync(0xffffffffu, need64)) {
                    double bd = CUDART_INF;
                    int bk = k;
                    for (int c = 0; c < cmax_w; ++c) {
                        const bool has = c < cnt;
                        const int kc = has ? cand_at(c) : 0;
                        const float e = cand_dist_f32(x0, x1, sC, kc, g);
                        if (need64 && has && g == 0 && e - 4.0e-6f * e <= u32) {
                            const double d = exact_f64(xt, rc, sC, kc);
                            if (d < bd || (d == bd && kc < bk)) { bd = d; bk = kc; }
                        }
                    }
                    bk = __shfl_sync(0xffffffffu, bk, lane & ~3);
                    bd = __shfl_sync(0xffffffffu, bd, lane & ~3);
                    if (need64) {
                        best = bk;
                        if (g == 0 && row < A.N) loss64 += bd;  // FP64 only on this rare path
                    }
                }
                if (row < A.N) {
                    if (g == 0) {
                        if (!need64) {
                            const float ts = lsum + emin;  // emin >= 0
                            lcomp += lsum >= emin ? (lsum - ts) + emin : (emin - ts) + lsum;
                            lsum = ts;
                        }
                        if (A.argmin_out) A.argmin_out[row] = best;
                    }
                    if (want_grad) {
                        // (a row at a time with lanes = its 32 coordinates,
                        // conflict-free, measured slower: 0.225 -> 0.250 ms)
                        float* srow = s_sum + best * KM_SUM_LD + 8 * g;
                        atomicAdd(srow + 0, x0.x);
                        atomicAdd(srow + 1, x0.y);
                        atomicAdd(srow + 2, x0.z);
                        atomicAdd(srow + 3, x0.w);
                        atomicAdd(srow + 4, x1.x);
                        atomicAdd(srow + 5, x1.y);
                        atomicAdd(srow + 6, x1.z);
                        atomicAdd(srow + 7, x1.w);
                        if (g == 0) atomicAdd(&s_cnt[best], 1.f);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&x_empty[s]);  // the X stage may be refilled now
        }
        // loss: warp reduce, then one double atomic per warp
        double loss_local = (double)lsum + (double)lcomp + loss64;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) loss_local += __shfl_xor_sync(0xffffffffu, loss_local, off);
        if (lane == 0 && loss_local != 0.0) atomicAdd(A.loss_acc, loss_local);
    }

    // drain: no TMA copy or MMA may be in flight when the CTA leaves
    if (warp == 0 && lane == 0) {
        for (int j = std::max(0, issued - KM_STAGES); j < issued; ++j)
            tc::mbar_wait(&x_full[j % KM_STAGES], (j / KM_STAGES) & 1, s_never, 1u << 20);
        tc::mbar_wait(c_bar, 0, s_never, 1u << 20);
    }
    if (warp == 1 && lane == 0) {
        for (int j = std::max(0, committed - 2); j < committed; ++j)
            tc::mbar_wait(&t_full[j & 1], (j >> 1) & 1, s_never, 1u << 20);
    }
    __syncthreads();
    if (*s_abort && threadIdx.x == 0) record_status(A.hdr, ADPAR_ERR_TIMEOUT);

    if (want_grad) {
        for (int q = threadIdx.x; q < k * KM_D; q += KM_THREADS)
            if (s_sum[(q / KM_D) * KM_SUM_LD + q % KM_D] != 0.f)
                atomicAdd(&A.gsum[q], s_sum[(q / KM_D) * KM_SUM_LD + q % KM_D]);
        for (int q = threadIdx.x; q < k; q += KM_THREADS)
            if (s_cnt[q] != 0.f) atomicAdd(&A.gcnt[q], s_cnt[q]);
    }
    // the last CTA to finish writes the loss and Cbar
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&A.hdr->done[0], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0 && A.loss_out) *A.loss_out = (float)ld_cg(A.loss_acc);
        if (want_grad) {
            const float yb2 = 2.f * (A.ybar ? *A.ybar : 1.f);
            for (int q = threadIdx.x; q < k * KM_D; q += KM_THREADS) {
                const int kc = q / KM_D;
                const float g = yb2 * (ld_cg(&A.gcnt[kc]) * __ldg(A.C + q) - ld_cg(&A.gsum[q]));
                A.Cbar[q] = A.accumulate ? A.Cbar[q] + g : g;
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// rows x 32 FP32, row stride 128 bytes, box of box_rows rows, 128-byte swizzle
bool make_map(CUtensorMap* m, const float* ptr, int64_t rows, uint32_t box_rows) {
    EncodeTiledFn f = encode_fn();
    if (!f) return false;
    cuuint64_t dims[2] = {(cuuint64_t)KM_D, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(KM_D * 4)};
    cuuint32_t box[2] = {(cuuint32_t)KM_D, box_rows};
    cuuint32_t es[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kMaxDev = 64;
bool km_configured[kMaxDev] = {};

// Hessian diagonal in C from the counts a gradient call left in the
// workspace: d^2 loss / dc_kj^2 = 2 ybar cnt_k (argmins held fixed).
__global__ void km_hessdiag_kernel(int kd, const float* ybar, const float* gcnt, float* H, int accumulate) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kd) return;
    const float h = 2.f * *ybar * gcnt[q / KM_D];
    H[q] = accumulate ? H[q] + h : h;
}

}  // namespace

size_t kmeans_workspace_size(int64_t k) {
    if (k <= 0 || k > KM_KMAX) return (size_t)-1;
    return sizeof(WsHeader) + 256 + round_up((size_t)k * KM_D * 4, 256) + round_up((size_t)k * 4, 256);
}

}  // namespace adpar

extern "C" int adpar_kmeans_vjp(int64_t N, int d, int k, const float* X, const float* C, const float* ybar,
                                float* loss_out, int32_t* argmin_out, float* Cbar, uint32_t flags, void* work,
                                size_t work_bytes, void* stream) {
    using namespace adpar;
    if (N < 0 || d <= 0 || k <= 0) return ADPAR_ERR_INVALID;
    if (d != KM_D || k > KM_KMAX || k % 32 != 0) return ADPAR_ERR_UNSUPPORTED;
    if (N > 0 && (!X || !C)) return ADPAR_ERR_INVALID;
    if (Cbar && !ybar) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    const void* ptrs[] = {X, C, Cbar, argmin_out};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    const size_t need = kmeans_workspace_size(k);
    if (!work || work_bytes < need || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    if (N >= (int64_t(1) << 31) - KM_TILE) return ADPAR_ERR_UNSUPPORTED;  // 32-bit TMA row coordinate
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return ADPAR_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!km_configured[dev]) {
        if (cudaFuncSetAttribute(kmeans_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KM_SMEM) !=
            cudaSuccess)
            return ADPAR_ERR_CUDA;
        km_configured[dev] = true;
    }
    KmArgs A{};
    A.N = N;
    A.k = k;
    A.X = X;
    A.C = C;
    A.ybar = ybar;
    A.loss_out = loss_out;
    A.argmin_out = argmin_out;
    A.Cbar = Cbar;
    A.accumulate = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    A.ntiles = (N + KM_TILE - 1) / KM_TILE;
    char* w = static_cast<char*>(work);
    A.hdr = reinterpret_cast<WsHeader*>(w);
    A.loss_acc = reinterpret_cast<double*>(w + sizeof(WsHeader));
    A.gsum = reinterpret_cast<float*>(w + sizeof(WsHeader) + 256);
    A.gcnt = reinterpret_cast<float*>(w + sizeof(WsHeader) + 256 + round_up((size_t)k * KM_D * 4, 256));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    km_init_kernel<<<8, 256, 0, s>>>(A);
    if (N == 0) {
        // empty sum: loss 0, Cbar = 2 ybar (0 * c - 0) = 0 (accumulate: unchanged)
        km_empty_kernel<<<1, 256, 0, s>>>(loss_out, Cbar, k * KM_D, A.accumulate);
        return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
    }
    CUtensorMap tmX, tmC;
    if (!make_map(&tmX, X, N, KM_TILE) || !make_map(&tmC, C, k, (uint32_t)k)) return ADPAR_ERR_CUDA;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.ntiles, sms));
    kmeans_kernel<<<grid, KM_THREADS, KM_SMEM, s>>>(tmX, tmC, A);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

extern "C" int adpar_kmeans_hessdiag(int k, const float* ybar, const void* work, size_t work_bytes, float* Hdiag,
                                     uint32_t flags, void* stream) {
    using namespace adpar;
    if (k <= 0 || !ybar || !Hdiag) return ADPAR_ERR_INVALID;
    if (k > KM_KMAX || k % 32 != 0) return ADPAR_ERR_UNSUPPORTED;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    const size_t need = kmeans_workspace_size(k);
    if (!work || work_bytes < need || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    const char* w = static_cast<const char*>(work);
    const float* gcnt =
        reinterpret_cast<const float*>(w + sizeof(WsHeader) + 256 + round_up((size_t)k * KM_D * 4, 256));
    const int kd = k * KM_D;
    km_hessdiag_kernel<<<(kd + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        kd, ybar, gcnt, Hdiag, (flags & ADPAR_ACCUMULATE) ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}
