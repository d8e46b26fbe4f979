// Scaled products for the * rules of Sec. 5.1.1 (reduce and reduce_by_index).
//
// The forward sweep of the * rule is re-executed as a map-reduce of
// (number of zeros, lowest zero index, product of the nonzero elements).
// The product of the nonzeros leaves every floating-point range on
// realistic sizes (a product of 65536 values from U[0.5,1.5) is about
// 1e-1287), so it is carried as  p = m * 2^e  with an FP64 mantissa m in
// [0.5, 1) and a 64-bit exponent e.  The exponent split uses the bits of
// the IEEE-754 representation (no FP64 arithmetic), so each element costs
// one FP64 multiply.
#pragma once

#include <stdint.h>

namespace adpar {

// x != 0 finite:  x = m * 2^e, 0.5 <= |m| < 1 (subnormals included).
__device__ __forceinline__ void split_pow2(double x, double& m, int64_t& e) {
    long long bits = __double_as_longlong(x);
    int ex = (int)((bits >> 52) & 0x7ff);
    int adj = 0;
    if (ex == 0) {  // subnormal: scale into the normal range first
        x *= 18014398509481984.0;  // 2^54
        bits = __double_as_longlong(x);
        ex = (int)((bits >> 52) & 0x7ff);
        adj = -54;
    }
    bits = (bits & ~(0x7ffLL << 52)) | (1022LL << 52);
    m = __longlong_as_double(bits);
    e = (int64_t)(ex - 1022 + adj);
}

// Renormalise m (nonzero, normal) into [0.5, 1), moving its exponent into e.
__device__ __forceinline__ void renorm(double& m, int64_t& e) {
    long long bits = __double_as_longlong(m);
    const int ex = (int)((bits >> 52) & 0x7ff);
    bits = (bits & ~(0x7ffLL << 52)) | (1022LL << 52);
    m = __longlong_as_double(bits);
    e += (int64_t)(ex - 1022);
}

struct ProdState {
    double m;       // mantissa of the product of the nonzeros, [0.5, 1)
    int64_t e;      // its binary exponent
    int64_t nz;     // number of zeros
    int64_t first;  // lowest zero index (INT64_MAX when none)

    __device__ static ProdState id() { return {0.5, 1, 0, INT64_MAX}; }  // 0.5 * 2^1 = 1
    __device__ static ProdState comb(const ProdState& x, const ProdState& y) {
        ProdState r;
        r.m = x.m * y.m;
        r.e = x.e + y.e;
        renorm(r.m, r.e);
        r.nz = x.nz + y.nz;
        r.first = x.first < y.first ? x.first : y.first;
        return r;
    }
    __device__ void push(double a, int64_t i) {
        if (a == 0.0) {
            ++nz;
            if (i < first) first = i;
        } else {
            double mi;
            int64_t ei;
            split_pow2(a, mi, ei);
            m *= mi;
            e += ei;
            renorm(m, e);
        }
    }
};

// ldexp with the exponent clamped to a range where the result is already
// 0 or infinite, so that a 64-bit exponent never overflows the int argument.
__device__ __forceinline__ double ldexp_clamped(double x, int64_t e) {
    if (e < -2200) e = -2200;
    if (e > 2200) e = 2200;
    return ldexp(x, (int)e);
}

}  // namespace adpar
