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

// FP32 x != 0 finite:  x = m * 2^e, 0.5 <= |m| < 1, with m as an FP32 and
// as an FP64 (formed from the bits: no conversion instruction)
__device__ __forceinline__ void split_pow2_f32m(float x, float& m, int& e) {
    int bits = __float_as_int(x);
    int ex = (bits >> 23) & 0xff;
    int adj = 0;
    if (ex == 0) {  // subnormal
        x *= 16777216.0f;  // 2^24
        bits = __float_as_int(x);
        ex = (bits >> 23) & 0xff;
        adj = -24;
    }
    m = __int_as_float((bits & ~(0xff << 23)) | (126 << 23));
    e = ex - 126 + adj;
}
__device__ __forceinline__ void split_pow2_f32(float x, double& m, int64_t& e) {
    float mf;
    int ef;
    split_pow2_f32m(x, mf, ef);
    const int b = __float_as_int(mf);
    const unsigned long long sign = (unsigned long long)((unsigned)b & 0x80000000u) << 32;
    m = __longlong_as_double((long long)(sign | (1022ULL << 52) | ((unsigned long long)(b & 0x7fffff) << 29)));
    e = ef;
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

// x * 2^e for a normal x with |x| in [2^-4, 2^4): the exponent field is
// adjusted directly when the result is normal (exact); a result in the
// subnormal range is formed by one multiply by 2^-1000 (one rounding,
// correct); below that it is a signed zero, above it an infinity.
__device__ __forceinline__ double scale_pow2(double x, int64_t e) {
    const long long b = __double_as_longlong(x);
    const int64_t ex = ((b >> 52) & 0x7ff) + e;
    const long long sign = b & (long long)0x8000000000000000ULL;
    if (ex >= 1 && ex <= 2046) return __longlong_as_double((b & ~(0x7ffLL << 52)) | ((long long)ex << 52));
    if (ex > 2046) return __longlong_as_double(sign | (0x7ffLL << 52));
    if (ex < -60) return __longlong_as_double(sign);
    return __longlong_as_double((b & ~(0x7ffLL << 52)) | ((long long)(ex + 1000) << 52)) * 9.332636185032189e-302;
}
// the same for FP32 results (x a float in [2^-4, 2^4))
__device__ __forceinline__ float scale_pow2f(float x, int64_t e) {
    const int b = __float_as_int(x);
    const int64_t ex = ((b >> 23) & 0xff) + e;
    const int sign = b & (int)0x80000000u;
    if (ex >= 1 && ex <= 254) return __int_as_float((b & ~(0xff << 23)) | ((int)ex << 23));
    if (ex > 254) return __int_as_float(sign | (0xff << 23));
    if (ex < -30) return __int_as_float(sign);
    return __int_as_float((b & ~(0xff << 23)) | ((int)(ex + 100) << 23)) * 7.888609052210118e-31f;  // 2^-100
}

// 1 / m for a mantissa with 0.5 <= |m| < 1, by Newton-Raphson on
// f(r) = 1/r - |m|: the seed is the FP32 reciprocal of |m| truncated to 24
// bits (relative error below 2^-22), and each step  r <- r + r (1 - |m| r)
// squares the relative error, so two steps reach FP64 rounding (1-2 ulp).
// The sign of m is put back at the end.
__device__ __forceinline__ double recip_mantissa(double m) {
    const long long bm = __double_as_longlong(m);
    const long long sign = bm & (long long)0x8000000000000000ULL;
    const double am = __longlong_as_double(bm ^ sign);
    const float mf = __int_as_float(0x3F000000 | (int)((bm >> 29) & 0x7FFFFF));  // |m| truncated, in [0.5, 1)
    const float rf = __frcp_rn(mf);                                             // in (1, 2]
    const int br = __float_as_int(rf);
    // widen the float (exponent 127 or 128) to a double without a conversion instruction
    double r = __longlong_as_double(((long long)(((br >> 23) & 0xff) - 127 + 1023) << 52) |
                                    ((long long)(br & 0x7FFFFF) << 29));
    double e = fma(-am, r, 1.0);
    r = fma(r, e, r);
    e = fma(-am, r, 1.0);
    r = fma(r, e, r);
    return __longlong_as_double(__double_as_longlong(r) | sign);
}

}  // namespace adpar
