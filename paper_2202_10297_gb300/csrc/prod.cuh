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

// FP32 values: a product of nonzeros is kept in integer fixed point so
// that no FP64 instruction runs per element (GB300 issues FP64 at 1/64 of
// the FP32 rate).  A mantissa M in [2^62, 2^63) stands for
// M * 2^(E - 62); the sign is a parity bit (bit 31 of the zero counter).
// Each product is truncated to 63 significant bits, a relative error below
// 2^-61 per factor, so a product of 2^27 factors stays within 1e-10.
constexpr unsigned long long kQ62One = 1ull << 62;

// M * mv for a 24-bit mantissa mv in [2^23, 2^24); returns the new M and
// the exponent increment (23 or 24)
__device__ __forceinline__ unsigned long long q62_mul24(unsigned long long M, unsigned mv, int& de) {
    const unsigned long long hi = (unsigned long long)(unsigned)(M >> 32) * mv;  // < 2^55
    const unsigned long long lo = (unsigned long long)(unsigned)M * mv;          // < 2^56
    const unsigned long long t24 = (hi << 8) + (lo >> 24);
    if (t24 >= kQ62One) {
        de = 24;
        return t24;
    }
    de = 23;
    return (hi << 9) + (lo >> 23);
}
// M1 * M2; returns the new M and the exponent increment (62 or 63)
__device__ __forceinline__ unsigned long long q62_mul(unsigned long long M1, unsigned long long M2, int& de) {
    const unsigned long long hi = __umul64hi(M1, M2), lo = M1 * M2;  // product in [2^124, 2^126)
    if (hi >= (1ull << 61)) {
        de = 63;
        return (hi << 1) | (lo >> 63);
    }
    de = 62;
    return (hi << 2) | (lo >> 62);
}
// an FP32 value v != 0 as (sign, 24-bit mantissa, exponent): |v| = mv * 2^ev
__device__ __forceinline__ void split_f32_int(float v, unsigned& sg, unsigned& mv, int& ev) {
    int bits = __float_as_int(v);
    sg = (unsigned)bits >> 31;
    int ex = (bits >> 23) & 0xff;
    int adj = 0;
    if (ex == 0) {  // subnormal
        bits = __float_as_int(v * 16777216.0f);
        ex = (bits >> 23) & 0xff;
        adj = -24;
    }
    mv = (unsigned)(bits & 0x7fffff) | 0x800000u;
    ev = ex - 150 + adj;
}
// fixed-point state -> (FP64 mantissa in [0.5, 1) with the sign, exponent)
__device__ __forceinline__ void q62_to_pow2(unsigned long long M, long long E, unsigned sign, double& mm,
                                            int64_t& e) {
    // M has its top bit at 62: as a double, 1 <= M * 2^-62 < 2 (rounded to 53 bits)
    const double x = __longlong_as_double((long long)((1023ull << 52) | ((M << 2) >> 12)));
    split_pow2(sign ? -x : x, mm, e);
    e += E;
}

// (zero count, lowest zero index, product of the nonzeros) in the
// fixed-point form above, for FP32 values (24-bit mantissas) and FP64 values
// (53-bit mantissas, one 64x64-bit product per factor); to_state() gives the
// FP64 form.
struct ProdStateQ {
    unsigned long long M;  // [2^62, 2^63): the product is M * 2^(E - 62)
    long long E;
    long long nz;
    long long first;
    unsigned sign;  // parity of the negative factors

    __device__ static ProdStateQ id() { return {kQ62One, 0, 0, INT64_MAX, 0u}; }
    __device__ static ProdStateQ comb(const ProdStateQ& x, const ProdStateQ& y) {
        ProdStateQ r;
        int de;
        r.M = q62_mul(x.M, y.M, de);
        r.E = x.E + y.E + de - 62;
        r.nz = x.nz + y.nz;
        r.first = x.first < y.first ? x.first : y.first;
        r.sign = x.sign ^ y.sign;
        return r;
    }
    __device__ void push(float a, int64_t i) {
        if (a == 0.0f) {
            ++nz;
            if (i < first) first = i;
        } else {
            unsigned sg, mv;
            int ev, de;
            split_f32_int(a, sg, mv, ev);
            M = q62_mul24(M, mv, de);
            E += ev + de;
            sign ^= sg;
        }
    }
    __device__ void push(double a, int64_t i) {
        if (a == 0.0) {
            ++nz;
            if (i < first) first = i;
            return;
        }
        long long bits = __double_as_longlong(a);
        int ex = (int)((bits >> 52) & 0x7ff);
        int adj = 0;
        if (ex == 0) {  // subnormal
            bits = __double_as_longlong(a * 18014398509481984.0);  // 2^54
            ex = (int)((bits >> 52) & 0x7ff);
            adj = -54;
        }
        // |a| = m53 * 2^(ex - 1075), m53 in [2^52, 2^53): as fixed point
        // m53 * 2^10 stands for |a| with exponent ex - 1075 + 52
        const unsigned long long m = ((unsigned long long)(bits & 0xfffffffffffffLL) | (1ull << 52)) << 10;
        int de;
        M = q62_mul(M, m, de);
        E += (ex - 1075 + adj + 52) + de - 62;
        sign ^= (unsigned)((unsigned long long)bits >> 63);
    }
    __device__ ProdState to_state() const {
        ProdState s;
        q62_to_pow2(M, E, sign, s.m, s.e);
        s.nz = nz;
        s.first = first;
        return s;
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

// 1 / m for a mantissa with 0.5 <= |m| < 1 in integer arithmetic, so that
// no FP64 instruction runs (GB300 issues FP64 at 1/64 of the FP32 rate):
// the seed r0 is the FP32 reciprocal of |m| truncated to 24 bits (relative
// error below 2^-22); one Newton step r1 = r0 (2 - |m| r0) in 64-bit fixed
// point (r scaled by 2^62, |m| by 2^53, products by __umul64hi) squares the
// error, below 2^-44 relative; r1 never exceeds 1/|m|, so it fits.  The sign
// of m is put back at the end.
__device__ __forceinline__ double recip_mantissa(double m) {
    const unsigned long long bm = (unsigned long long)__double_as_longlong(m);
    const unsigned long long sign = bm & 0x8000000000000000ULL;
    const unsigned long long M = (bm & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);  // |m| * 2^53
    const float mf = __int_as_float(0x3F000000 | (int)((bm >> 29) & 0x7FFFFF));  // |m| truncated, in [0.5, 1)
    const unsigned br = __float_as_uint(__frcp_rn(mf));                          // in (1, 2]
    const int ex = (int)((br >> 23) & 0xff) - 127;                               // 0, or 1 for r0 = 2
    const unsigned long long R0 = (unsigned long long)((br & 0x7FFFFFu) | 0x800000u) << (39 + ex);  // r0 * 2^62
    // |m| r0 * 2^62 = M R0 / 2^53 (M R0 < 2^116)
    const unsigned long long mr = (__umul64hi(M, R0) << 11) | ((M * R0) >> 53);
    const unsigned long long d = (2ULL << 62) - mr;  // (2 - |m| r0) * 2^62
    const unsigned long long R1 = (__umul64hi(R0, d) << 2) | ((R0 * d) >> 62);  // r1 * 2^62, in [2^62, 2^63]
    const int lz = __clzll((long long)R1);  // 0 only for r1 = 2
    const unsigned long long mant = ((R1 << lz) >> 11) & 0xFFFFFFFFFFFFFULL;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(1024 - lz) << 52) | mant));
}

// k / m for mantissas with 0.25 <= |k| <= 1 and 0.5 <= |m| < 1: k times the
// integer reciprocal above (relative error below 2^-44), one FP64 multiply
__device__ __forceinline__ double quot_mantissa(double k, double m) { return k * recip_mantissa(m); }

}  // namespace adpar
