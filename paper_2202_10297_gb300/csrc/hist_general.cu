// reduce_by_index VJP by the GENERAL rule of Sec. 5.1.2, for every operator
// of scan_ops.cuh (LINREC, which has no special rule, included).
//
//   hs[k] = (.) over the elements i with inds_i = k, in increasing i,
//   a_bar_i (+)= d(l_i (.) a_i (.) r_i)/d a_i ^T hs_bar[inds_i],
// where l_i and r_i combine the elements of i's bin before and after i.
// Those are per-bin ("multi-") scans; as Sec. 5.1.2 proposes they come from
// sorting the elements by bin and running a forward and a reverse
// irregular-segmented scan over the sorted sequence.
//
// Sort: least-significant-digit radix passes of up to 8 bits of the bin
// number, each three kernels (digit counts per block, a scan of the counts
// per digit, a stable scatter that ranks each tile by digit, stages it in
// shared memory in digit order and writes every digit's run contiguously).
// The values travel with their keys, so every read of a and b is
// coalesced, and each pass records where every element went.  Elements
// whose index is outside [0, m) leave in the first pass.
// Segmented scans: a segmented scan is a plain scan of (state, flag) pairs,
//   forward  (x1,f1) + (x2,f2) = f2 ? (x2,f2) : (x1 (.) x2, f1)
// with f = "a bin starts here", and its mirror image for the reverse scan
// with f = "a bin ends here".  Both are single-pass look-back scans over
// tiles; the forward one keeps only each tile's carry, the reverse one
// re-forms l inside the tile from that carry, applies the map and writes
// the adjoints in sorted order.
// Return: the recorded destinations of the passes, read backwards, gather
// the adjoints back to the original order (each inverse pass has the
// access pattern of a radix pass, and the last one writes the caller's
// arrays coalesced), instead of one random store per element.
#include <algorithm>

#include "common.cuh"
#include "scan_engine.cuh"
#include "scan_ops.cuh"

namespace adpar {
namespace {

constexpr int kSortBlock = 256;
constexpr int kSortNW = kSortBlock / 32;
// elements per thread and tile of the scatter (a tile is staged in static
// shared memory: fewer for FP64 pairs)
template <class T, int W>
constexpr int sort_items() {
    return sizeof(T) == 8 && W == 2 ? 6 : 8;
}
constexpr int kChunkAlign = kSortBlock * 24;  // a multiple of every tile
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortMaxGrid = 2048;
constexpr int kSegBlock = 256;
constexpr int kSegV = 4;  // consecutive elements per thread and chunk
constexpr int kSegK = 2;  // chunks per tile
constexpr int kSegTile = kSegK * kSegBlock * kSegV;
constexpr uint32_t kNoKey = 0xffffffffu;  // above every bin number (m < 2^31)

// ------------------------------------------------------------ radix sort
template <class T>
struct SortPass {
    int64_t n, m;          // all elements; bins
    const void* inds;      // first pass: the caller's indices
    const uint32_t* kin;   // later passes: keys and values
    const T* ain;
    const T* bin;
    uint32_t* kout;
    T* aout;
    T* bout;
    uint32_t* dest;        // [input length] where each input element went (kNoKey: left the sort)
    uint32_t* cnt;         // [2^bits][G] digit counts per block, then their exclusive scan
    uint32_t* rowtot;      // [2^bits] elements per digit
    const uint32_t* nsorted;  // in-range elements (set by the first pass)
    int shift, bits, G;
};

// Block c of a pass covers [c * len_c, (c + 1) * len_c) of its input, a
// whole number of tiles.
__device__ __forceinline__ int64_t block_chunk(int64_t len, int G) {
    const int64_t c = (len + G - 1) / G;
    return (c + kChunkAlign - 1) / kChunkAlign * kChunkAlign;
}

// Exclusive scan of one value per thread over a block of kSortBlock.
__device__ __forceinline__ uint32_t block_excl_u32(uint32_t x, uint32_t* s_w, uint32_t* total = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < kSortNW; ++w) {
            const uint32_t t = s_w[w];
            s_w[w] = run;
            run += t;
        }
        s_w[kSortNW] = run;
    }
    __syncthreads();
    const uint32_t r = s_w[warp] + inc - x;
    if (total) *total = s_w[kSortNW];
    __syncthreads();
    return r;
}

template <class I, class T, bool FIRST>
__device__ __forceinline__ bool sort_key(const SortPass<T>& P, int64_t i, uint32_t& key) {
    if constexpr (FIRST) {
        const int64_t ix = (int64_t)static_cast<const I*>(P.inds)[i];
        key = (uint32_t)ix;
        return ix >= 0 && ix < P.m;
    } else {
        key = P.kin[i];
        return true;
    }
}

template <class I, class T, bool FIRST>
__global__ void __launch_bounds__(kSortBlock) hg_count_kernel(SortPass<T> P) {
    __shared__ uint32_t h[kSortNW][kRadix];
    const int warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < kSortNW * kRadix; q += kSortBlock) (&h[0][0])[q] = 0u;
    __syncthreads();
    const int64_t len = FIRST ? P.n : (int64_t)*P.nsorted;
    const int64_t bc = block_chunk(len, P.G);
    const int64_t lo = (int64_t)blockIdx.x * bc;
    const int64_t hi = lo + bc < len ? lo + bc : len;
    const uint32_t dmask = (1u << P.bits) - 1u;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kSortBlock) {
        uint32_t key;
        if (sort_key<I, T, FIRST>(P, i, key)) atomicAdd(&h[warp][(key >> P.shift) & dmask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < (1 << P.bits); d += kSortBlock) {
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < kSortNW; ++w) t += h[w][d];
        P.cnt[(int64_t)d * P.G + blockIdx.x] = t;
    }
}

// Block d turns row d of the counts into its exclusive scan over the
// blocks and records the row total (the first pass also sums the totals
// into the in-range element count).
__global__ void __launch_bounds__(kSortBlock) hg_scan_counts_kernel(uint32_t* cnt, uint32_t* rowtot, int G,
                                                                    uint32_t* nsorted) {
    constexpr int E = 8;
    __shared__ uint32_t s_w[kSortNW + 1];
    uint32_t* row = cnt + (int64_t)blockIdx.x * G;
    uint32_t run = 0;
    for (int base = 0; base < G; base += kSortBlock * E) {
        uint32_t v[E];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int q = base + threadIdx.x * E + j;
            v[j] = q < G ? row[q] : 0u;
            s += v[j];
        }
        uint32_t tot;
        uint32_t ex = run + block_excl_u32(s, s_w, &tot);
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int q = base + threadIdx.x * E + j;
            if (q < G) row[q] = ex;
            ex += v[j];
        }
        run += tot;
    }
    if (threadIdx.x == 0) {
        rowtot[blockIdx.x] = run;
        if (nsorted) atomicAdd(nsorted, run);
    }
}

// Stable scatter of one pass.  A block takes its chunk tile by tile (warp
// w holds the tile's elements [w*256, (w+1)*256), 32 consecutive ones per
// item).  Every element gets its rank among the equal digits before it in
// the tile (the lanes of equal digit from one ballot per digit bit, per-warp
// digit counts, their scan over the warps
// and the digits), which is its place in the tile sorted by digit; the tile
// is staged in that order in shared memory and written out so that each
// digit's run lands contiguously after the block's previous run of that
// digit.  Blocks and tiles are in input order and the counts were scanned
// over the blocks digit by digit, so equal digits keep their input order.
template <class I, class T, int W, bool FIRST>
__global__ void __launch_bounds__(kSortBlock) hg_scatter_kernel(SortPass<T> P) {
    constexpr int kSortItems = sort_items<T, W>();
    constexpr int kSortTile = kSortBlock * kSortItems;
    __shared__ uint32_t s_cnt[kSortNW][kRadix];
    __shared__ uint32_t s_off[kRadix];    // the block's next global position per digit
    __shared__ uint32_t s_start[kRadix];  // the digit's first place in the sorted tile
    __shared__ uint32_t s_w[kSortNW + 1];
    __shared__ uint32_t s_key[kSortTile];
    __shared__ T s_a[kSortTile];
    __shared__ T s_b[W == 2 ? kSortTile : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = 1 << P.bits;
    const uint32_t dmask = (uint32_t)R - 1u;
    {
        const uint32_t rt = threadIdx.x < R ? P.rowtot[threadIdx.x] : 0u;
        const uint32_t ex = block_excl_u32(rt, s_w);
        if (threadIdx.x < R) s_off[threadIdx.x] = ex + P.cnt[(int64_t)threadIdx.x * P.G + blockIdx.x];
    }
    const int64_t len = FIRST ? P.n : (int64_t)*P.nsorted;
    const int64_t bc = block_chunk(len, P.G);
    const int64_t lo = (int64_t)blockIdx.x * bc;
    const int64_t hi = lo + bc < len ? lo + bc : len;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t t0 = lo; t0 < hi; t0 += kSortTile) {
        for (int q = threadIdx.x; q < kSortNW * kRadix; q += kSortBlock) (&s_cnt[0][0])[q] = 0u;
        __syncthreads();
        uint32_t key[kSortItems], rk[kSortItems];
        T va[kSortItems], vb[kSortItems];
        bool ok[kSortItems];
#pragma unroll
        for (int u = 0; u < kSortItems; ++u) {
            const int64_t i = t0 + warp * (32 * kSortItems) + u * 32 + lane;
            ok[u] = false;
            key[u] = 0u;
            va[u] = T(0);
            vb[u] = T(0);
            if (i < hi) {  // values loaded beside the key, not after its range test
                ok[u] = sort_key<I, T, FIRST>(P, i, key[u]);
                va[u] = __ldcs(P.ain + i);
                if constexpr (W == 2) vb[u] = __ldcs(P.bin + i);
            }
        }
#pragma unroll
        for (int u = 0; u < kSortItems; ++u) {
            const uint32_t d = (key[u] >> P.shift) & dmask;
            // the lanes holding the same digit: one ballot per digit bit
            uint32_t peers = __ballot_sync(0xffffffffu, ok[u]);
            for (int b = 0; b < P.bits; ++b) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            const uint32_t base = ok[u] ? s_cnt[warp][d] : 0u;
            __syncwarp();
            if (ok[u] && (peers & lt) == 0u) s_cnt[warp][d] = base + __popc(peers);  // the lowest peer
            __syncwarp();
            rk[u] = base + __popc(peers & lt);
        }
        __syncthreads();
        // per digit: exclusive over the warps, then over the digits
        uint32_t tot = 0;
        if (threadIdx.x < R) {
#pragma unroll
            for (int w = 0; w < kSortNW; ++w) {
                const uint32_t c = s_cnt[w][threadIdx.x];
                s_cnt[w][threadIdx.x] = tot;
                tot += c;
            }
        }
        uint32_t nvalid;
        const uint32_t st = block_excl_u32(tot, s_w, &nvalid);
        if (threadIdx.x < R) s_start[threadIdx.x] = st;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kSortItems; ++u) {
            const int64_t i = t0 + warp * (32 * kSortItems) + u * 32 + lane;
            if (i >= hi) continue;
            if (!ok[u]) {
                P.dest[i] = kNoKey;
                continue;
            }
            const uint32_t d = (key[u] >> P.shift) & dmask;
            const uint32_t within = s_cnt[warp][d] + rk[u];
            const uint32_t lpos = s_start[d] + within;
            P.dest[i] = s_off[d] + within;
            s_key[lpos] = key[u];
            s_a[lpos] = va[u];
            if constexpr (W == 2) s_b[lpos] = vb[u];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < (int)nvalid; q += kSortBlock) {
            const uint32_t k = s_key[q];
            const uint32_t d = (k >> P.shift) & dmask;
            const uint32_t pos = s_off[d] + (uint32_t)q - s_start[d];
            P.kout[pos] = k;
            P.aout[pos] = s_a[q];
            if constexpr (W == 2) P.bout[pos] = s_b[q];
        }
        __syncthreads();
        if (threadIdx.x < R) s_off[threadIdx.x] += tot;
    }
}

// Inverse of one pass: out[i] = in[dest[i]] over the pass's input order.
// The first pass's inverse writes the caller's adjoints (0 or unchanged
// for an element that left the sort, += with accumulation).
template <class T, int W, bool FIRST>
__global__ void __launch_bounds__(kSortBlock) hg_unsort_kernel(int64_t n, const uint32_t* nsorted,
                                                               const uint32_t* dest, const T* ia, const T* ib,
                                                               T* oa, T* ob, int accumulate) {
    const int64_t len = FIRST ? n : (int64_t)*nsorted;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; i0 < len; i0 += stride) {
        uint32_t d[4];
        if (i0 + 4 <= len) {
            const uint4 x = __ldcs(reinterpret_cast<const uint4*>(dest + i0));
            d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) d[j] = i0 + j < len ? dest[i0 + j] : kNoKey;
        }
        T va[4], vb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            va[j] = d[j] != kNoKey ? ia[d[j]] : T(0);
            vb[j] = (W == 2 && d[j] != kNoKey) ? ib[d[j]] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = i0 + j;
            if (i >= len) break;
            if (FIRST && accumulate) {
                if (d[j] != kNoKey) {
                    oa[i] += va[j];
                    if constexpr (W == 2) ob[i] += vb[j];
                }
            } else {
                oa[i] = va[j];
                if constexpr (W == 2) ob[i] = vb[j];
            }
        }
    }
}

// ------------------------------------------------------ segmented scans
template <class Op>
struct SegS {
    typename Op::P x;
    uint32_t f;
};

template <class Op>
__device__ __forceinline__ SegS<Op> seg_id() {
    return SegS<Op>{Op::pid(), 0u};
}

// forward: f = a bin starts inside the right operand
template <class Op>
__device__ __forceinline__ SegS<Op> seg_fcomb(const SegS<Op>& l, const SegS<Op>& r) {
    return r.f ? r : SegS<Op>{Op::pcomb(l.x, r.x), l.f};
}

// reverse: e holds later elements, l earlier ones; f = a bin ends inside
template <class Op>
__device__ __forceinline__ SegS<Op> seg_rcomb(const SegS<Op>& e, const SegS<Op>& l) {
    return l.f ? l : SegS<Op>{Op::pcomb(l.x, e.x), e.f};
}

template <class Op, class T>
struct SegArgs {
    const uint32_t* keys;  // sorted bin numbers
    const T* a;            // sorted values
    const T* b;
    const uint32_t* nsorted;
    int64_t tiles;
    SegS<Op>* carry;       // [tiles] forward state before each tile
    unsigned long long* fA;
    unsigned long long* fI;
    unsigned long long* rA;
    unsigned long long* rI;
    WsHeader* hdr;
    const T* hsbar_a;
    const T* hsbar_b;
    T* oa;                 // [n] adjoints in sorted order
    T* ob;
    T* hs_a;
    T* hs_b;
};

__device__ __forceinline__ void ld_keys(const uint32_t* p, int64_t e, int64_t n, uint32_t (&o)[kSegV]) {
    if (e + kSegV <= n) {
        const uint4 x = __ldcs(reinterpret_cast<const uint4*>(p + e));
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    } else {
#pragma unroll
        for (int j = 0; j < kSegV; ++j) o[j] = e + j < n ? p[e + j] : kNoKey;
    }
}

template <class T>
__device__ __forceinline__ void ld_vals(const T* p, int64_t e, int64_t n, T pad, T (&o)[kSegV]) {
    constexpr int VV = Vec16<T>::N;
    if (e + kSegV <= n) {
#pragma unroll
        for (int q = 0; q < kSegV / VV; ++q) {
            const Vec16<T> x = ld_vec_stream(p + e + q * VV);
#pragma unroll
            for (int j = 0; j < VV; ++j) o[q * VV + j] = x.v[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < kSegV; ++j) o[j] = e + j < n ? p[e + j] : pad;
    }
}

template <class T>
__device__ __forceinline__ void st_vals(T* p, int64_t e, int64_t n, const T (&v)[kSegV]) {
    constexpr int VV = Vec16<T>::N;
    if (e + kSegV <= n) {
#pragma unroll
        for (int q = 0; q < kSegV / VV; ++q) {
            Vec16<T> x;
#pragma unroll
            for (int j = 0; j < VV; ++j) x.v[j] = v[q * VV + j];
            st_vec(p + e + q * VV, x);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kSegV; ++j)
            if (e + j < n) p[e + j] = v[j];
    }
}

// Forward pass: each tile's forward segmented state before its first
// element (the carry), by look-back.
template <class Op, class T>
__global__ void __launch_bounds__(kSegBlock) hg_seg_fwd_kernel(SegArgs<Op, T> A) {
    using S = SegS<Op>;
    constexpr int NW = kSegBlock / 32, K = kSegK, V = kSegV;
    __shared__ uint32_t s_tile;
    __shared__ S s_tot[K * NW];
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[0], 1u);
    __syncthreads();
    const int64_t t = s_tile;
    const int64_t ns = (int64_t)*A.nsorted;
    const int64_t base = t * kSegTile;
    S agg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kSegBlock * V + threadIdx.x * V;
        uint32_t kk[V];
        T av[V], bv[V];
        ld_keys(A.keys, e, ns, kk);
        ld_vals(A.a, e, ns, Op::pad_a(), av);
        if constexpr (Op::kWidth == 2) ld_vals(A.b, e, ns, T(0), bv);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[j] = T(0);
        }
        uint32_t prev = (e > 0 && e - 1 < ns) ? A.keys[e - 1] : kNoKey;
        S acc = seg_id<Op>();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (e + j < ns) acc = seg_fcomb<Op>(acc, S{Op::pelem(av[j], bv[j]), kk[j] != prev ? 1u : 0u});
            prev = kk[j];
        }
        agg[k] = acc;
    }
    auto fc = [](const S& l, const S& r) { return seg_fcomb<Op>(l, r); };
    S wex[K];
    const S total = block_scan_part1<S, false, K, NW>(agg, wex, s_tot, seg_id<Op>(), fc);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<S> st{A.fA, A.fI};
        const S pre = lookback(t, st, total, seg_id<Op>(), fc, A.hdr);
        if ((threadIdx.x & 31) == 0) A.carry[t] = pre;
    }
}

// Reverse pass: tiles right to left.  l comes from the tile's carry and a
// forward block scan, r from a reverse block scan and a look-back over the
// tiles to the right; then the map of Sec. 5.1.2 and, at the first element
// of every bin, hs[bin] = a_first (.) r_first.
template <class Op, class T>
__global__ void __launch_bounds__(kSegBlock) hg_seg_bwd_kernel(SegArgs<Op, T> A) {
    using S = SegS<Op>;
    using P = typename Op::P;
    constexpr int NW = kSegBlock / 32, K = kSegK, V = kSegV, W = Op::kWidth;
    __shared__ uint32_t s_tile;
    __shared__ S s_totF[K * NW];
    __shared__ S s_totR[K * NW];
    __shared__ S s_carry;
    __shared__ S s_suf;
    if (threadIdx.x == 0) s_tile = atomicAdd(&A.hdr->ticket[1], 1u);
    __syncthreads();
    const int64_t t_log = s_tile;
    const int64_t tile = A.tiles - 1 - t_log;
    const int64_t ns = (int64_t)*A.nsorted;
    const int64_t base = tile * kSegTile;
    if (threadIdx.x == 0) s_carry = A.carry[tile];

    uint32_t kk[K][V], kprev[K], knext[K];
    T av[K][V], bv[K][V];
    S aggF[K], aggR[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kSegBlock * V + threadIdx.x * V;
        ld_keys(A.keys, e, ns, kk[k]);
        ld_vals(A.a, e, ns, Op::pad_a(), av[k]);
        if constexpr (W == 2) ld_vals(A.b, e, ns, T(0), bv[k]);
        else {
#pragma unroll
            for (int j = 0; j < V; ++j) bv[k][j] = T(0);
        }
        kprev[k] = (e > 0 && e - 1 < ns) ? A.keys[e - 1] : kNoKey;
        knext[k] = (e + V < ns) ? A.keys[e + V] : kNoKey;
        S f = seg_id<Op>();
        uint32_t prev = kprev[k];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (e + j < ns) f = seg_fcomb<Op>(f, S{Op::pelem(av[k][j], bv[k][j]), kk[k][j] != prev ? 1u : 0u});
            prev = kk[k][j];
        }
        aggF[k] = f;
        S r = seg_id<Op>();
        uint32_t next = knext[k];
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {
            if (e + j < ns) r = seg_rcomb<Op>(r, S{Op::pelem(av[k][j], bv[k][j]), kk[k][j] != next ? 1u : 0u});
            next = kk[k][j];
        }
        aggR[k] = r;
    }
    auto fc = [](const S& l, const S& r) { return seg_fcomb<Op>(l, r); };
    auto rc = [](const S& e, const S& l) { return seg_rcomb<Op>(e, l); };
    S wexF[K], wexR[K];
    (void)block_scan_part1<S, false, K, NW>(aggF, wexF, s_totF, seg_id<Op>(), fc);
    const S totR = block_scan_part1<S, true, K, NW>(aggR, wexR, s_totR, seg_id<Op>(), rc);
    if ((threadIdx.x >> 5) == 0) {
        LookbackState<S> st{A.rA, A.rI};
        const S suf = lookback(t_log, st, totR, seg_id<Op>(), rc, A.hdr);
        if ((threadIdx.x & 31) == 0) s_suf = suf;
    }
    __syncthreads();

#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kSegBlock * V + threadIdx.x * V;
        if (e >= ns) continue;
        S lf = block_scan_excl<S, false, K, NW>(k, wexF, s_totF, s_carry, fc);
        P lx[V];
        uint32_t prev = kprev[k];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const bool head = kk[k][j] != prev;
            lx[j] = head ? Op::pid() : lf.x;
            lf = seg_fcomb<Op>(lf, S{Op::pelem(av[k][j], bv[k][j]), head ? 1u : 0u});
            prev = kk[k][j];
        }
        S rr = block_scan_excl<S, true, K, NW>(k, wexR, s_totR, s_suf, rc);
        uint32_t next = knext[k];
        T oa[V], ob[V];
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {
            const uint32_t key = kk[k][j];
            const bool tail = key != next;
            next = key;
            oa[j] = T(0);
            ob[j] = T(0);
            if (e + j >= ns) continue;
            const P rx = tail ? Op::pid() : rr.x;
            const T ya = A.hsbar_a[key];
            const T yb = W == 2 ? A.hsbar_b[key] : T(0);
            Op::mid_vjp(lx[j], av[k][j], bv[k][j], rx, ya, yb, oa[j], ob[j]);
            const bool head = j > 0 ? kk[k][j - 1] != key : kprev[k] != key;
            if (head && A.hs_a) {
                const P y = Op::pcomb(Op::pelem(av[k][j], bv[k][j]), rx);
                A.hs_a[key] = Op::out_a(y);
                if constexpr (W == 2) A.hs_b[key] = Op::out_b(y);
            }
            rr = seg_rcomb<Op>(rr, S{Op::pelem(av[k][j], bv[k][j]), tail ? 1u : 0u});
        }
        st_vals(A.oa, e, ns, oa);
        if constexpr (W == 2) st_vals(A.ob, e, ns, ob);
    }
}

// hs of a bin without elements is the neutral element
template <class Op, class T>
__global__ void hg_fill_kernel(int64_t m, T* hs_a, T* hs_b) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        hs_a[k] = Op::out_a(Op::pid());
        if constexpr (Op::kWidth == 2) hs_b[k] = Op::out_b(Op::pid());
    }
}

// ------------------------------------------------------------ host side
constexpr int kMaxPasses = 4;  // 31 key bits in passes of at most 8

struct HgLayout {
    size_t off_cnt, off_rowtot, off_k[2], off_a[2], off_b[2], off_dest[kMaxPasses], off_carry, off_slots;
    size_t slot_bytes, total;
    int64_t tiles;
};

int key_bits(int64_t m) {
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < m) ++bits;
    return bits;
}

template <class Op, class T>
HgLayout hg_layout(int64_t n, int64_t m) {
    using S = SegS<Op>;
    HgLayout L{};
    const size_t nn = (size_t)(n > 0 ? n : 1);
    size_t o = sizeof(WsHeader);
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = round_up(o + bytes, 256);
        return at;
    };
    L.off_cnt = take(sizeof(uint32_t) * kRadix * kSortMaxGrid);
    L.off_rowtot = take(sizeof(uint32_t) * kRadix);
    for (int q = 0; q < 2; ++q) {
        L.off_k[q] = take(sizeof(uint32_t) * nn);
        L.off_a[q] = take(sizeof(T) * nn);
        L.off_b[q] = Op::kWidth == 2 ? take(sizeof(T) * nn) : L.off_a[q];
    }
    const int passes = (key_bits(m) + kRadixBits - 1) / kRadixBits;
    for (int p = 0; p < passes; ++p) L.off_dest[p] = take(sizeof(uint32_t) * nn);
    L.tiles = (n + kSegTile - 1) / kSegTile;
    if (L.tiles < 1) L.tiles = 1;
    L.off_carry = take(sizeof(S) * (size_t)L.tiles);
    L.slot_bytes = 4 * sizeof(unsigned long long) * (size_t)lb_words<S>() * (size_t)L.tiles;
    L.off_slots = take(L.slot_bytes);
    L.total = o;
    return L;
}

int sms_now() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class Op, class T, class I>
int run_hist_general(int64_t n, int64_t m, const void* a, const void* b, const void* inds, const void* hsbar_a,
                     const void* hsbar_b, void* abar, void* bbar, void* hs_a, void* hs_b, uint32_t flags,
                     void* work, size_t work_bytes, cudaStream_t s) {
    using S = SegS<Op>;
    constexpr int W = Op::kWidth;
    const HgLayout L = hg_layout<Op, T>(n, m);
    if (work == nullptr || work_bytes < L.total || (reinterpret_cast<uintptr_t>(work) & 255u))
        return ADPAR_ERR_WORKSPACE;
    char* w = static_cast<char*>(work);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(w);
    if (cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s) != cudaSuccess) return ADPAR_ERR_CUDA;
    if (hs_a && m > 0) {
        const int blocks = (int)std::min<int64_t>((m + 255) / 256, 4096);
        hg_fill_kernel<Op, T><<<blocks, 256, 0, s>>>(m, static_cast<T*>(hs_a), static_cast<T*>(hs_b));
    }
    if (n == 0) return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
    if (cudaMemsetAsync(w + L.off_slots, 0, L.slot_bytes, s) != cudaSuccess) return ADPAR_ERR_CUDA;

    // key bits: bin numbers are below m (out-of-range elements leave in pass 0)
    const int bits = key_bits(m);
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const int dbits = (bits + passes - 1) / passes;
    // one wave of the scatter kernel: every block's chunk is in flight at once
    const int sms = sms_now();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hg_scatter_kernel<I, T, W, false>, kSortBlock, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int G = (int)std::max<int64_t>(
        1, std::min<int64_t>({(n + kChunkAlign - 1) / kChunkAlign, (int64_t)kSortMaxGrid, (int64_t)sms * per_sm}));
    uint32_t* nsorted = &hdr->done[0];
    SortPass<T> SP{};
    SP.n = n;
    SP.m = m;
    SP.inds = inds;
    SP.cnt = reinterpret_cast<uint32_t*>(w + L.off_cnt);
    SP.rowtot = reinterpret_cast<uint32_t*>(w + L.off_rowtot);
    SP.nsorted = nsorted;
    SP.G = G;
    for (int p = 0; p < passes; ++p) {
        const int src = p & 1, dst = (p + 1) & 1;
        SP.shift = p * dbits;
        SP.bits = std::min(dbits, bits - p * dbits);
        SP.kin = reinterpret_cast<const uint32_t*>(w + L.off_k[src]);
        SP.ain = p == 0 ? static_cast<const T*>(a) : reinterpret_cast<const T*>(w + L.off_a[src]);
        SP.bin = p == 0 ? static_cast<const T*>(b) : reinterpret_cast<const T*>(w + L.off_b[src]);
        SP.kout = reinterpret_cast<uint32_t*>(w + L.off_k[dst]);
        SP.aout = reinterpret_cast<T*>(w + L.off_a[dst]);
        SP.bout = reinterpret_cast<T*>(w + L.off_b[dst]);
        SP.dest = reinterpret_cast<uint32_t*>(w + L.off_dest[p]);
        if (p == 0) {
            hg_count_kernel<I, T, true><<<G, kSortBlock, 0, s>>>(SP);
            hg_scan_counts_kernel<<<1 << SP.bits, kSortBlock, 0, s>>>(SP.cnt, SP.rowtot, G, nsorted);
            hg_scatter_kernel<I, T, W, true><<<G, kSortBlock, 0, s>>>(SP);
        } else {
            hg_count_kernel<I, T, false><<<G, kSortBlock, 0, s>>>(SP);
            hg_scan_counts_kernel<<<1 << SP.bits, kSortBlock, 0, s>>>(SP.cnt, SP.rowtot, G, nullptr);
            hg_scatter_kernel<I, T, W, false><<<G, kSortBlock, 0, s>>>(SP);
        }
    }
    // the sorted data sit in buffer fin; the other buffer takes the
    // sorted-order adjoints, and the inverse passes alternate between them
    const int fin = passes & 1;
    const size_t wd = (size_t)lb_words<S>() * (size_t)L.tiles;
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(w + L.off_slots);
    SegArgs<Op, T> A{};
    A.keys = reinterpret_cast<const uint32_t*>(w + L.off_k[fin]);
    A.a = reinterpret_cast<const T*>(w + L.off_a[fin]);
    A.b = reinterpret_cast<const T*>(w + L.off_b[fin]);
    A.nsorted = nsorted;
    A.tiles = L.tiles;
    A.carry = reinterpret_cast<S*>(w + L.off_carry);
    A.fA = slots;
    A.fI = slots + wd;
    A.rA = slots + 2 * wd;
    A.rI = slots + 3 * wd;
    A.hdr = hdr;
    A.hsbar_a = static_cast<const T*>(hsbar_a);
    A.hsbar_b = static_cast<const T*>(hsbar_b);
    A.oa = reinterpret_cast<T*>(w + L.off_a[1 - fin]);
    A.ob = reinterpret_cast<T*>(w + L.off_b[1 - fin]);
    A.hs_a = static_cast<T*>(hs_a);
    A.hs_b = static_cast<T*>(hs_b);
    hg_seg_fwd_kernel<Op, T><<<(unsigned)L.tiles, kSegBlock, 0, s>>>(A);
    hg_seg_bwd_kernel<Op, T><<<(unsigned)L.tiles, kSegBlock, 0, s>>>(A);
    const int acc = (flags & ADPAR_ACCUMULATE) ? 1 : 0;
    const int ublocks = (int)std::max<int64_t>(1, std::min<int64_t>((n / 4 + kSortBlock) / kSortBlock,
                                                                       (int64_t)sms * 8));
    int cur = 1 - fin;
    for (int p = passes - 1; p >= 0; --p) {
        const uint32_t* dest = reinterpret_cast<const uint32_t*>(w + L.off_dest[p]);
        const T* ia = reinterpret_cast<const T*>(w + L.off_a[cur]);
        const T* ib = reinterpret_cast<const T*>(w + L.off_b[cur]);
        if (p == 0) {
            hg_unsort_kernel<T, W, true><<<ublocks, kSortBlock, 0, s>>>(n, nsorted, dest, ia, ib, static_cast<T*>(abar),
                                                                       static_cast<T*>(bbar), acc);
        } else {
            T* oa = reinterpret_cast<T*>(w + L.off_a[1 - cur]);
            T* ob = reinterpret_cast<T*>(w + L.off_b[1 - cur]);
            hg_unsort_kernel<T, W, false><<<ublocks, kSortBlock, 0, s>>>(n, nsorted, dest, ia, ib, oa, ob, acc);
            cur = 1 - cur;
        }
    }
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}

template <class T, class I>
int dispatch_hist_general(int op, int64_t n, int64_t m, const void* a, const void* b, const void* inds,
                          const void* ya, const void* yb, void* abar, void* bbar, void* hs_a, void* hs_b,
                          uint32_t flags, void* work, size_t wb, cudaStream_t s) {
    switch (op) {
    case ADPAR_OP_ADD:
        return run_hist_general<OpAdd<T>, T, I>(n, m, a, b, inds, ya, yb, abar, bbar, hs_a, hs_b, flags, work, wb, s);
    case ADPAR_OP_MUL:
        return run_hist_general<OpMul<T>, T, I>(n, m, a, b, inds, ya, yb, abar, bbar, hs_a, hs_b, flags, work, wb, s);
    case ADPAR_OP_MIN:
        return run_hist_general<OpMin<T>, T, I>(n, m, a, b, inds, ya, yb, abar, bbar, hs_a, hs_b, flags, work, wb, s);
    case ADPAR_OP_MAX:
        return run_hist_general<OpMax<T>, T, I>(n, m, a, b, inds, ya, yb, abar, bbar, hs_a, hs_b, flags, work, wb, s);
    case ADPAR_OP_LINREC:
        return run_hist_general<OpLinrec<T>, T, I>(n, m, a, b, inds, ya, yb, abar, bbar, hs_a, hs_b, flags, work, wb,
                                                   s);
    }
    return ADPAR_ERR_INVALID;
}

template <class T>
size_t layout_total(int op, int64_t n, int64_t m) {
    switch (op) {
    case ADPAR_OP_ADD: return hg_layout<OpAdd<T>, T>(n, m).total;
    case ADPAR_OP_MUL: return hg_layout<OpMul<T>, T>(n, m).total;
    case ADPAR_OP_MIN: return hg_layout<OpMin<T>, T>(n, m).total;
    case ADPAR_OP_MAX: return hg_layout<OpMax<T>, T>(n, m).total;
    case ADPAR_OP_LINREC: return hg_layout<OpLinrec<T>, T>(n, m).total;
    }
    return (size_t)-1;
}

}  // namespace

size_t hist_general_workspace_size(adpar_opdesc d, int64_t n, int64_t m) {
    if (n < 0 || m < 0 || d.op < ADPAR_OP_ADD || d.op > ADPAR_OP_LINREC) return (size_t)-1;
    if (d.dtype == ADPAR_F32) return layout_total<float>(d.op, n, m);
    if (d.dtype == ADPAR_F64) return layout_total<double>(d.op, n, m);
    return (size_t)-1;
}

}  // namespace adpar

extern "C" int adpar_vjp_hist_general(adpar_opdesc d, int64_t n, int64_t m, const void* a, const void* b,
                                      const void* inds, int itype, const void* hsbar_a, const void* hsbar_b,
                                      void* abar, void* bbar, void* hs_a, void* hs_b, uint32_t flags, void* work,
                                      size_t work_bytes, void* stream) {
    using namespace adpar;
    if (n < 0 || m < 0) return ADPAR_ERR_INVALID;
    if (d.op < ADPAR_OP_ADD || d.op > ADPAR_OP_LINREC) return ADPAR_ERR_INVALID;
    if (d.dtype != ADPAR_F32 && d.dtype != ADPAR_F64) return ADPAR_ERR_INVALID;
    if (itype != ADPAR_I32 && itype != ADPAR_I64) return ADPAR_ERR_INVALID;
    const int want_w = d.op == ADPAR_OP_LINREC ? 2 : 1;
    if (d.width != want_w) return ADPAR_ERR_INVALID;
    if (flags & ~(uint32_t)ADPAR_ACCUMULATE) return ADPAR_ERR_UNSUPPORTED;
    // positions and bin numbers travel as 32-bit words
    if (n >= (int64_t)0xffffffffu || m > ((int64_t)1 << 31)) return ADPAR_ERR_UNSUPPORTED;
    if (want_w == 2 && hs_a && !hs_b) return ADPAR_ERR_INVALID;
    if (hs_a == nullptr && hs_b != nullptr) return ADPAR_ERR_INVALID;
    if (n > 0) {
        if (!a || !inds || !abar || (m > 0 && !hsbar_a)) return ADPAR_ERR_INVALID;
        if (want_w == 2 && (!b || !bbar || (m > 0 && !hsbar_b))) return ADPAR_ERR_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.dtype == ADPAR_F32) {
        if (itype == ADPAR_I32)
            return dispatch_hist_general<float, int32_t>(d.op, n, m, a, b, inds, hsbar_a, hsbar_b, abar, bbar, hs_a,
                                                         hs_b, flags, work, work_bytes, s);
        return dispatch_hist_general<float, int64_t>(d.op, n, m, a, b, inds, hsbar_a, hsbar_b, abar, bbar, hs_a, hs_b,
                                                     flags, work, work_bytes, s);
    }
    if (itype == ADPAR_I32)
        return dispatch_hist_general<double, int32_t>(d.op, n, m, a, b, inds, hsbar_a, hsbar_b, abar, bbar, hs_a,
                                                      hs_b, flags, work, work_bytes, s);
    return dispatch_hist_general<double, int64_t>(d.op, n, m, a, b, inds, hsbar_a, hsbar_b, abar, bbar, hs_a, hs_b,
                                                  flags, work, work_bytes, s);
}
