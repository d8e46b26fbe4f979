// Batched VJPs: many independent instances of uneven length, each a
// product-reduce VJP (Sec. 5.1.1) followed by a linear-recurrence scan VJP
// (Sec. 5.2), in ONE persistent launch that a CUDA graph can capture.
//
// Work items.  Segment s of length L has R = ceil(L / RT) reduce tiles and
// S = ceil(L / ST) scan tiles, and contributes, in this order,
//   R product-reduce tiles, S primal-scan tiles (left to right),
//   S adjoint-scan tiles (right to left), R product-map tiles.
// Items are numbered segment after segment and handed out by one global
// atomic ticket.  An item only ever waits on items with smaller numbers of
// its own segment (the look-back predecessors, the primal carries, the
// finished product), which were handed out earlier to blocks that are
// running, so the schedule cannot deadlock, and every wait is bounded.
// Small segments are one tile of each kind; no look-back happens there.
//
// The scan tiles run the linear recurrence on per-thread runs
// (batch_runs.cuh: a forward tile stores its runs' carries, a reverse tile
// re-forms the primal from them); the product tiles re-run the forward
// sweep as a (zero count, lowest zero, scaled product) reduction per tile
// whose last tile to finish combines the partials and raises the segment's
// flag.
#include <algorithm>
#include <cstring>
#include <vector>

#include "batch_runs.cuh"
#include "prod.cuh"
#include "scan_tiles.cuh"

namespace adpar {
namespace {

struct BatchPlanHeader {
    int64_t nseg;
    int64_t total_items;
    int64_t ws_bytes;
    int64_t seg_off;   // byte offset of the segment array in the plan
    int64_t meta_off;  // byte offset of the SegMeta array in the plan
    int32_t variant;
    int32_t order;
    int32_t ctas_per_sm;
    int32_t reserved;
};

struct SegMeta {
    int64_t item_base;  // first item number of the segment
    int64_t state_off;  // byte offset of its state in the workspace
    int32_t red_tiles;
    int32_t scan_tiles;
};

// reduce/map tile of the compiled variants (RT elements); the scan tiles
// are brun_tile<T>() elements in every variant
struct VariantShape {
    int rt;
};
constexpr VariantShape kVariants[] = {{8192}, {16384}, {4096}};
constexpr int kNumVariants = 3;

// per-segment state layout (bytes from state_off)
struct StateLayout {
    int64_t partials, counter, final_state, p_agg, p_incl, r_agg, r_incl, done, carA, carB, prod, total;
};

__host__ __device__ inline int64_t al16(int64_t x) { return (x + 15) & ~int64_t(15); }

__host__ __device__ inline StateLayout state_layout(int dtype, int red, int scan) {
    const int wp = dtype == ADPAR_F64 ? 4 : 2;  // 64-bit words of a primal (A, B) state
    const int wr = dtype == ADPAR_F64 ? 6 : 3;  // of a lin_o (c, dA, dB) state
    const int64_t es = dtype == ADPAR_F64 ? 8 : 4;
    const int64_t runs = (int64_t)scan * kBNT;
    StateLayout L;
    int64_t o = 0;
    L.partials = o; o = al16(o + (int64_t)red * (int64_t)sizeof(ProdStateQ));
    L.counter = o; o = al16(o + 16);
    L.final_state = o; o = al16(o + (int64_t)sizeof(ProdState));
    L.p_agg = o; o = al16(o + (int64_t)scan * wp * 8);
    L.p_incl = o; o = al16(o + (int64_t)scan * wp * 8);
    L.r_agg = o; o = al16(o + (int64_t)scan * wr * 8);
    L.r_incl = o; o = al16(o + (int64_t)scan * wr * 8);
    L.done = o; o = al16(o + (int64_t)scan * 4);
    L.carA = o; o = al16(o + runs * es);
    L.carB = o; o = al16(o + runs * es);
    L.prod = o; o = al16(o + runs * es);
    L.total = o;
    return L;
}

template <class S>
__device__ __forceinline__ S block_reduce_256(S v, S (*comb)(const S&, const S&), S* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = comb(v, shfl_down_s(v, off));
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = s_warp[lane < 8 ? lane : 0];
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            S o = shfl_down_s(v, off);
            if (lane + off < 8) v = comb(v, o);
        }
    }
    return v;  // valid in thread 0
}

__device__ ProdStateQ prod_comb(const ProdStateQ& x, const ProdStateQ& y) { return ProdStateQ::comb(x, y); }

// product reduce tile r of a segment
template <class T>
__device__ void prod_reduce_tile(const adpar_batch_segment& sg, char* st, const StateLayout& L, int red, int r,
                                 int RT, WsHeader* hdr) {
    __shared__ ProdStateQ s_warp[8];
    __shared__ int s_last;
    const T* x = static_cast<const T*>(sg.x);
    const int64_t lo = (int64_t)r * RT, hi = std::min<int64_t>(sg.len, lo + RT);
    range_prefetch_l2(x, lo, hi);
    ProdStateQ ps = ProdStateQ::id();  // fixed-point products: no FP64 per element
    constexpr int V = Vec16<T>::N;
    for (int64_t i = lo + threadIdx.x * V; i < hi; i += 256 * V) {
        if (i + V <= hi) {
            Vec16<T> v = ld_vec(x + i);
#pragma unroll
            for (int j = 0; j < V; ++j) ps.push(v.v[j], i + j);
        } else {
            for (int64_t j = i; j < hi; ++j) ps.push(x[j], j);
        }
    }
    ProdStateQ bs = block_reduce_256<ProdStateQ>(ps, prod_comb, s_warp);
    ProdStateQ* partials = reinterpret_cast<ProdStateQ*>(st + L.partials);
    unsigned int* counter = reinterpret_cast<unsigned int*>(st + L.counter);
    if (threadIdx.x == 0) {
        partials[r] = bs;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == (unsigned)(red - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ProdStateQ totq = ProdStateQ::id();
    for (int q = threadIdx.x; q < red; q += 256) totq = ProdStateQ::comb(totq, ld_cg(partials + q));
    __syncthreads();
    totq = block_reduce_256<ProdStateQ>(totq, prod_comb, s_warp);
    if (threadIdx.x == 0) {
        const ProdState tot = totq.to_state();
        *reinterpret_cast<ProdState*>(st + L.final_state) = tot;
        if (sg.aux) {
            adpar_prod_aux a;
            a.nzero = tot.nz;
            a.first_zero = tot.nz > 0 ? tot.first : -1;
            a.exp2 = tot.e;
            a.mant = tot.m;
            a.log_abs_nz = log(fabs(tot.m)) + (double)tot.e * 0.69314718055994530942;
            a.sign = tot.m > 0 ? 1 : -1;
            a.reserved = 0;
            *sg.aux = a;
        }
        __threadfence();
        st_release_u32(counter + 1, 1u);  // the segment's product is final
    }
}

// product map tile r: the three cases of Sec. 5.1.1
template <class T>
__device__ void prod_map_tile(const adpar_batch_segment& sg, char* st, const StateLayout& L, int r, int RT,
                              WsHeader* hdr) {
    __shared__ ProdState s_fin;
    unsigned int* counter = reinterpret_cast<unsigned int*>(st + L.counter);
    range_prefetch_l2(static_cast<const T*>(sg.x), (int64_t)r * RT, std::min<int64_t>(sg.len, (int64_t)r * RT + RT));
    if (threadIdx.x == 0) {
        if (wait_flag(counter + 1, hdr) != 0u) s_fin = ld_cg(reinterpret_cast<const ProdState*>(st + L.final_state));
        else s_fin = ProdState::id();
    }
    __syncthreads();
    const T* x = static_cast<const T*>(sg.x);
    T* xb = static_cast<T*>(sg.xbar);
    const int64_t lo = (int64_t)r * RT, hi = std::min<int64_t>(sg.len, lo + RT);
    const ProdState f = s_fin;
    const double yb = sg.ybar_prod;
    double ym = 0.0;
    int64_t ye = 0;
    if (yb != 0.0) split_pow2(yb, ym, ye);
    const double kq = f.m * ym;     // mantissa of p * ybar
    const float qf = (float)kq;
    for (int64_t i = lo + threadIdx.x; i < hi; i += 256) {
        double c = 0.0;
        if (yb != 0.0) {
            if (f.nz == 0) {
                if constexpr (sizeof(T) == 4) {  // FP32 output: FP32 arithmetic suffices
                    float mf;
                    int ef;
                    split_pow2_f32m(static_cast<const float*>(sg.x)[i], mf, ef);
                    xb[i] = scale_pow2f(qf * __frcp_rn(mf), f.e + ye - ef);
                    continue;
                } else {
                    double mi;
                    int64_t ei;
                    split_pow2((double)x[i], mi, ei);
                    c = scale_pow2(quot_mantissa(kq, mi), f.e + ye - ei);
                }
            } else if (f.nz == 1 && i == f.first) {
                c = ldexp_clamped(f.m * ym, f.e + ye);
            }
        }
        xb[i] = (T)c;
    }
}

// linear-recurrence tile j of a segment: forward (adjoint false, left to
// right) or reverse (right to left), on per-thread runs
template <class T>
__device__ void linrec_tile(const adpar_batch_segment& sg, char* st, const StateLayout& L, int scan_tiles,
                            int64_t j, bool adjoint, unsigned char* smem, WsHeader* hdr) {
    BRunState S;
    S.p_agg = reinterpret_cast<unsigned long long*>(st + L.p_agg);
    S.p_incl = reinterpret_cast<unsigned long long*>(st + L.p_incl);
    S.r_agg = reinterpret_cast<unsigned long long*>(st + L.r_agg);
    S.r_incl = reinterpret_cast<unsigned long long*>(st + L.r_incl);
    S.done = reinterpret_cast<uint32_t*>(st + L.done);
    S.carA = st + L.carA;
    S.carB = st + L.carB;
    S.prod = st + L.prod;
    const T* a = static_cast<const T*>(sg.a);
    const T* b = static_cast<const T*>(sg.b);
    if (adjoint)
        brun_rev_tile<T>(a, b, static_cast<const T*>(sg.ybar_a), static_cast<const T*>(sg.ybar_b),
                         static_cast<T*>(sg.abar), static_cast<T*>(sg.bbar), sg.len, S, scan_tiles, j, smem, hdr);
    else
        brun_fwd_tile<T>(a, b, sg.len, S, j, smem, hdr);
}

__global__ void batch_init_kernel(char* ws, int64_t bytes) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n16 = bytes / 16;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride)
        reinterpret_cast<uint4*>(ws)[i] = make_uint4(0, 0, 0, 0);
}

template <int RT>
__global__ void __launch_bounds__(256) batch_kernel(const char* plan, char* ws) {
    extern __shared__ __align__(16) unsigned char s_dyn[];  // kBRunSmem: the scan tiles' arrays
    const BatchPlanHeader* H = reinterpret_cast<const BatchPlanHeader*>(plan);
    const adpar_batch_segment* segs = reinterpret_cast<const adpar_batch_segment*>(plan + H->seg_off);
    const SegMeta* meta = reinterpret_cast<const SegMeta*>(plan + H->meta_off);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    const int64_t nseg = H->nseg, total = H->total_items;
    __shared__ uint32_t s_item;
    __shared__ int s_stop;
    __shared__ int64_t s_seg;
    // thread 0's segment of the CTA's last item: tickets only grow, so the
    // next item's segment is found from there (usually the same segment: no
    // load at all; else a galloping search forward), instead of a binary
    // search of 12 dependent loads per item
    int64_t seg = 0, seg_next = nseg > 1 ? meta[1].item_base : INT64_MAX;
    while (true) {
        __syncthreads();  // consecutive items reuse the static shared memory
        if (threadIdx.x == 0) {
            s_item = atomicAdd(&hdr->ticket[0], 1u);
            s_stop = ((int64_t)s_item >= total) || gave_up(hdr);
            const int64_t q = s_item;
            if (!s_stop && q >= seg_next) {
                // the last s with item_base <= q lies in (seg, nseg)
                int64_t lo = seg + 1, step = 1;
                while (lo + step < nseg && meta[lo + step].item_base <= q) {
                    lo += step;
                    step <<= 1;
                }
                int64_t hi = std::min<int64_t>(nseg - 1, lo + step - 1);
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (meta[mid].item_base <= q) lo = mid;
                    else hi = mid - 1;
                }
                seg = lo;
                seg_next = seg + 1 < nseg ? meta[seg + 1].item_base : INT64_MAX;
            }
            s_seg = seg;
        }
        __syncthreads();
        if (s_stop) break;
        const int64_t q = s_item;
        const int64_t lo = s_seg;
        const SegMeta m = meta[lo];
        const adpar_batch_segment sg = segs[lo];
        const StateLayout L = state_layout(sg.dtype, m.red_tiles, m.scan_tiles);
        char* st = ws + m.state_off;
        int64_t j = q - m.item_base;
        const bool f64 = sg.dtype == ADPAR_F64;
        if (j < m.red_tiles) {
            if (f64) prod_reduce_tile<double>(sg, st, L, m.red_tiles, (int)j, RT, hdr);
            else prod_reduce_tile<float>(sg, st, L, m.red_tiles, (int)j, RT, hdr);
            continue;
        }
        j -= m.red_tiles;
        if (j < m.scan_tiles) {
            if (f64) linrec_tile<double>(sg, st, L, m.scan_tiles, j, false, s_dyn, hdr);
            else linrec_tile<float>(sg, st, L, m.scan_tiles, j, false, s_dyn, hdr);
            continue;
        }
        j -= m.scan_tiles;
        if (j < m.scan_tiles) {
            if (f64) linrec_tile<double>(sg, st, L, m.scan_tiles, j, true, s_dyn, hdr);
            else linrec_tile<float>(sg, st, L, m.scan_tiles, j, true, s_dyn, hdr);
            continue;
        }
        j -= m.scan_tiles;
        if (f64) prod_map_tile<double>(sg, st, L, (int)j, RT, hdr);
        else prod_map_tile<float>(sg, st, L, (int)j, RT, hdr);
    }
}

typedef void (*BatchKernel)(const char*, char*);
BatchKernel kernel_of(int v) {
    switch (v) {
    case 0: return batch_kernel<8192>;
    case 1: return batch_kernel<16384>;
    case 2: return batch_kernel<4096>;
    }
    return nullptr;
}

size_t plan_bytes(int64_t nseg) {
    return round_up(sizeof(BatchPlanHeader), 64) + round_up((size_t)nseg * sizeof(adpar_batch_segment), 64) +
           round_up((size_t)nseg * sizeof(SegMeta), 64);
}

}  // namespace
}  // namespace adpar

extern "C" size_t adpar_batch_plan_bytes(int nseg) {
    return nseg < 0 ? (size_t)-1 : adpar::plan_bytes(nseg);
}

extern "C" int adpar_batch_plan(const adpar_batch_segment* segs, int nseg, const adpar_batch_config* cfg,
                                void* plan_host, size_t plan_bytes_avail, size_t* work_bytes_out) {
    using namespace adpar;
    static_assert(sizeof(adpar_batch_segment) == 96, "segment descriptor is 96 bytes");
    if (nseg < 0 || (nseg > 0 && !segs) || !plan_host || !work_bytes_out) return ADPAR_ERR_INVALID;
    adpar_batch_config c{0, 2, 1, 0};
    if (cfg) c = *cfg;
    if (c.variant < 0 || c.variant >= kNumVariants || c.ctas_per_sm < 1 || c.ctas_per_sm > 8 || c.order < 0 ||
        c.order > 1)
        return ADPAR_ERR_INVALID;
    const size_t need = plan_bytes(nseg);
    if (plan_bytes_avail < need) return ADPAR_ERR_WORKSPACE;
    for (int s = 0; s < nseg; ++s) {
        const adpar_batch_segment& g = segs[s];
        if (g.len < 0 || (g.dtype != ADPAR_F32 && g.dtype != ADPAR_F64)) return ADPAR_ERR_INVALID;
        if (g.len > 0 && (!g.x || !g.xbar || !g.a || !g.b || !g.ybar_a || !g.ybar_b || !g.abar || !g.bbar))
            return ADPAR_ERR_INVALID;
        const void* ptrs[] = {g.x, g.xbar, g.a, g.b, g.ybar_a, g.ybar_b, g.abar, g.bbar};
        for (const void* p : ptrs)
            if (p && !aligned16(p)) return ADPAR_ERR_ALIGN;
    }
    const VariantShape V = kVariants[c.variant];
    // scheduling order: as given, or the longest (most bytes) first so the
    // tail of the launch is made of short segments
    std::vector<int> order(nseg);
    for (int s = 0; s < nseg; ++s) order[s] = s;
    if (c.order == 1)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const int64_t wx = segs[x].len * (segs[x].dtype == ADPAR_F64 ? 2 : 1);
            const int64_t wy = segs[y].len * (segs[y].dtype == ADPAR_F64 ? 2 : 1);
            return wx > wy;
        });
    char* P = static_cast<char*>(plan_host);
    std::memset(P, 0, need);
    BatchPlanHeader* H = reinterpret_cast<BatchPlanHeader*>(P);
    H->nseg = nseg;
    H->seg_off = (int64_t)round_up(sizeof(BatchPlanHeader), 64);
    H->meta_off = H->seg_off + (int64_t)round_up((size_t)nseg * sizeof(adpar_batch_segment), 64);
    H->variant = c.variant;
    H->order = c.order;
    H->ctas_per_sm = c.ctas_per_sm;
    adpar_batch_segment* S = reinterpret_cast<adpar_batch_segment*>(P + H->seg_off);
    SegMeta* M = reinterpret_cast<SegMeta*>(P + H->meta_off);
    int64_t items = 0, state = (int64_t)sizeof(WsHeader);
    for (int q = 0; q < nseg; ++q) {
        const adpar_batch_segment& g = segs[order[q]];
        const int st = g.dtype == ADPAR_F64 ? brun_tile<double>() : brun_tile<float>();
        const int64_t red = std::max<int64_t>(1, (g.len + V.rt - 1) / V.rt);
        const int64_t scan = std::max<int64_t>(1, (g.len + st - 1) / st);
        if (red > INT32_MAX || scan > INT32_MAX) return ADPAR_ERR_UNSUPPORTED;
        S[q] = g;
        M[q].item_base = items;
        M[q].red_tiles = (int32_t)red;
        M[q].scan_tiles = (int32_t)scan;
        M[q].state_off = state;
        items += 2 * red + 2 * scan;
        state += state_layout(g.dtype, (int)red, (int)scan).total;
    }
    if (items > (int64_t)UINT32_MAX - ((int64_t)1 << 20)) return ADPAR_ERR_UNSUPPORTED;  // 32-bit tickets
    H->total_items = items;
    H->ws_bytes = (int64_t)round_up((size_t)state, 256);
    *work_bytes_out = (size_t)H->ws_bytes;
    return ADPAR_OK;
}

extern "C" int adpar_vjp_batch(const void* plan_host, const void* plan_dev, void* work, size_t work_bytes,
                               void* stream) {
    using namespace adpar;
    if (!plan_host || !plan_dev) return ADPAR_ERR_INVALID;
    const BatchPlanHeader* H = static_cast<const BatchPlanHeader*>(plan_host);
    if (H->variant < 0 || H->variant >= kNumVariants) return ADPAR_ERR_INVALID;
    if (!work || work_bytes < (size_t)H->ws_bytes || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    if (H->nseg == 0) return ADPAR_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADPAR_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ib = (int)std::max<int64_t>(1, std::min<int64_t>((H->ws_bytes / 16 + 255) / 256, (int64_t)sms * 4));
    batch_init_kernel<<<ib, 256, 0, s>>>(static_cast<char*>(work), H->ws_bytes);
    static bool configured[64][kNumVariants] = {};
    if (dev < 0 || dev >= 64) return ADPAR_ERR_CUDA;
    if (!configured[dev][H->variant]) {
        if (cudaFuncSetAttribute(kernel_of(H->variant), cudaFuncAttributeMaxDynamicSharedMemorySize, kBRunSmem) !=
            cudaSuccess)
            return ADPAR_ERR_CUDA;
        configured[dev][H->variant] = true;
    }
    const int64_t grid = std::min<int64_t>((int64_t)sms * H->ctas_per_sm, H->total_items);
    kernel_of(H->variant)<<<(unsigned)std::max<int64_t>(1, grid), 256, kBRunSmem, s>>>(
        static_cast<const char*>(plan_dev), static_cast<char*>(work));
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}
