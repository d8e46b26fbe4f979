// Device-side helpers shared by the adpar kernels: memory-order primitives
// for single-pass (decoupled look-back) scans, bounded waits that record a
// status instead of hanging, warp shuffles of small structs, and the
// workspace header.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/adpar.h"

namespace adpar {

constexpr int kWarp = 32;

// Bounded waits.  A wait polls at most kSpinLimit times with a short
// sleep in between (about a second in total), then records
// ADPAR_ERR_TIMEOUT in the workspace header and lets the kernel finish
// with whatever it has, so a broken dependency never hangs the GPU.
constexpr uint32_t kSpinLimit = 1u << 22;

// Workspace header (first 256 bytes of every workspace).
struct WsHeader {
    uint32_t status;       // ADPAR_OK or ADPAR_ERR_TIMEOUT
    uint32_t ticket[7];    // dynamic tile tickets, one per pass
    uint32_t done[8];      // "last block" counters
    uint8_t pad[256 - 64];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void record_status(WsHeader* h, uint32_t code) {
    atomicCAS(&h->status, (uint32_t)ADPAR_OK, code);
}

__device__ __forceinline__ bool gave_up(const WsHeader* h) {
    return *reinterpret_cast<const volatile uint32_t*>(&h->status) != (uint32_t)ADPAR_OK;
}

// Wait until *flag != 0; returns the flag value, or 0 after recording a
// timeout.  Once any wait of the call has timed out, every later wait
// returns at once, so a broken call ends in about one wait limit in total
// rather than one per tile.
__device__ __forceinline__ uint32_t wait_flag(const uint32_t* flag, WsHeader* h) {
    uint32_t f = ld_acquire_u32(flag);
    uint32_t it = 0;
    while (f == 0) {
        ++it;
        if (it > kSpinLimit || ((it & 255u) == 0 && gave_up(h))) {
            record_status(h, ADPAR_ERR_TIMEOUT);
            return 0;
        }
        __nanosleep(it < 64 ? 20 : 200);
        f = ld_acquire_u32(flag);
    }
    return f;
}

// L2-coherent (non-L1) loads of values published by other blocks.
template <class T>
__device__ __forceinline__ T ld_cg(const T* p) {
    static_assert(sizeof(T) % 4 == 0, "4-byte granules");
    constexpr int W = sizeof(T) / 4;
    union { T t; uint32_t w[W]; } u;
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int i = 0; i < W; ++i) u.w[i] = __ldcg(q + i);
    return u.t;
}

// Warp shuffles of any struct made of 4-byte granules.
template <class T>
__device__ __forceinline__ T shfl_up_s(T v, int off) {
    constexpr int W = sizeof(T) / 4;
    union { T t; uint32_t w[W]; } u;
    u.t = v;
#pragma unroll
    for (int i = 0; i < W; ++i) u.w[i] = __shfl_up_sync(0xffffffffu, u.w[i], off);
    return u.t;
}
template <class T>
__device__ __forceinline__ T shfl_down_s(T v, int off) {
    constexpr int W = sizeof(T) / 4;
    union { T t; uint32_t w[W]; } u;
    u.t = v;
#pragma unroll
    for (int i = 0; i < W; ++i) u.w[i] = __shfl_down_sync(0xffffffffu, u.w[i], off);
    return u.t;
}
template <class T>
__device__ __forceinline__ T shfl_idx_s(T v, int src) {
    constexpr int W = sizeof(T) / 4;
    union { T t; uint32_t w[W]; } u;
    u.t = v;
#pragma unroll
    for (int i = 0; i < W; ++i) u.w[i] = __shfl_sync(0xffffffffu, u.w[i], src);
    return u.t;
}

// 16-byte vector of T (4 floats or 2 doubles).
template <class T> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int N = 4;
    float v[4];
};
template <> struct Vec16<double> {
    static constexpr int N = 2;
    double v[2];
};

template <class T>
__device__ __forceinline__ Vec16<T> ld_vec(const T* p) {
    Vec16<T> r;
    if constexpr (sizeof(T) == 4) {
        float4 x = __ldg(reinterpret_cast<const float4*>(p));
        r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
    } else {
        double2 x = __ldg(reinterpret_cast<const double2*>(p));
        r.v[0] = x.x; r.v[1] = x.y;
    }
    return r;
}

// Streaming load (data read once: evict-first in L1/L2).
template <class T>
__device__ __forceinline__ Vec16<T> ld_vec_stream(const T* p) {
    Vec16<T> r;
    if constexpr (sizeof(T) == 4) {
        float4 x = __ldcs(reinterpret_cast<const float4*>(p));
        r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
    } else {
        double2 x = __ldcs(reinterpret_cast<const double2*>(p));
        r.v[0] = x.x; r.v[1] = x.y;
    }
    return r;
}

template <class T>
__device__ __forceinline__ void st_vec(T* p, const Vec16<T>& r) {
    if constexpr (sizeof(T) == 4) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
    } else {
        __stcs(reinterpret_cast<double2*>(p), make_double2(r.v[0], r.v[1]));
    }
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace adpar
