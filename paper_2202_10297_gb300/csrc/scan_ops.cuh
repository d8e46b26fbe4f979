// Associative operators for the scan and reduce rules (Sec. 5.1, 5.2).
//
// An operator (.) supplies, on its primal state P:
//   pid()            neutral element e
//   pcomb(l, r)      l (.) r, l earlier in the sequence
//   pelem(a, b)      the element built from the input arrays (b: LINREC)
//   pad_a()          an input value whose element is harmless as padding
//                    past the end of the data (its J_left is 1, see coef)
// and, for the return sweep of Sec. 5.2, with prev = rs_{i-1}:
//   coef(prev, a)    J_left(i) = d(prev (.) a_i)/d prev.  Every operator
//                    here has J_left = c * I, so c is one scalar even for
//                    the width-2 LINREC element (its J_left is a_i * I).
//   vjp_right(...)   J_right(i)^T rs_bar_i = the adjoint of as_i.
// and, for the general reduce rule of Sec. 5.1.1 (l = the elements before,
// r = the elements after, as states):
//   mid_vjp(l, a, b, r, yA, yB)  the adjoint of the element (a, b) in
//                    y = l (.) (a, b) (.) r, i.e. d(l (.) x (.) r)/dx^T ybar.
// and, for forward mode (JVP):
//   tcomb(l, tl, r, tr)  the tangent of l (.) r given the tangents tl, tr of
//                    l and r (a state of the same shape).
// kNeedPrimal says whether vjp_right reads prev; kCoefNeedsPrimal whether
// coef does (MIN/MAX: the tie rule compares against prev).  kCoefIsA says
// that J_left(i) is the element's own a_i (MUL, LINREC): then the product
// of the J_left factors over a run of elements is out_a of the run's
// primal prefix, which the return sweep reuses instead of re-multiplying;
// for these operators P is exactly (out_a, out_b) and pelem rebuilds it.
// To add an operator, write one more struct of this shape.
#pragma once

#include <math_constants.h>

namespace adpar {

template <class T> __device__ __forceinline__ T pos_inf();
template <> __device__ __forceinline__ float pos_inf<float>() { return CUDART_INF_F; }
template <> __device__ __forceinline__ double pos_inf<double>() { return CUDART_INF; }

template <class T>
struct ScalarP {
    T v;
};
template <class T>
struct PairP {
    T A, B;
};

template <class T>
struct OpAdd {
    static constexpr int kWidth = 1;
    static constexpr bool kNeedPrimal = false;
    static constexpr bool kCoefNeedsPrimal = false;
    static constexpr bool kCoefOne = true;
    static constexpr bool kCoefIsA = false;
    using P = ScalarP<T>;
    __device__ static P pid() { return {T(0)}; }
    __device__ static P pcomb(P l, P r) { return {l.v + r.v}; }
    __device__ static P pelem(T a, T) { return {a}; }
    __device__ static T pad_a() { return T(0); }
    __device__ static T coef(P, T) { return T(1); }
    __device__ static void vjp_right(P, T, T, T ra, T, T& oa, T&) { oa = ra; }
    __device__ static void mid_vjp(P, T, T, P, T ya, T, T& oa, T&) { oa = ya; }
    __device__ static P tcomb(P, P tl, P, P tr) { return {tl.v + tr.v}; }
    __device__ static T out_a(P p) { return p.v; }
    __device__ static T out_b(P) { return T(0); }
};

template <class T>
struct OpMul {
    static constexpr int kWidth = 1;
    static constexpr bool kNeedPrimal = true;
    static constexpr bool kCoefNeedsPrimal = false;
    static constexpr bool kCoefOne = false;
    static constexpr bool kCoefIsA = true;
    using P = ScalarP<T>;
    __device__ static P pid() { return {T(1)}; }
    __device__ static P pcomb(P l, P r) { return {l.v * r.v}; }
    __device__ static P pelem(T a, T) { return {a}; }
    __device__ static T pad_a() { return T(1); }
    __device__ static T coef(P, T a) { return a; }
    __device__ static void vjp_right(P prev, T, T, T ra, T, T& oa, T&) { oa = prev.v * ra; }
    // l a r: the product of all the others (no division, zeros are safe)
    __device__ static void mid_vjp(P l, T, T, P r, T ya, T, T& oa, T&) { oa = (l.v * r.v) * ya; }
    __device__ static P tcomb(P l, P tl, P r, P tr) { return {fma(tl.v, r.v, l.v * tr.v)}; }
    __device__ static T out_a(P p) { return p.v; }
    __device__ static T out_b(P) { return T(0); }
};

// max: ties keep the earlier element (J_left = [prev >= a], J_right = [a > prev]).
template <class T>
struct OpMax {
    static constexpr int kWidth = 1;
    static constexpr bool kNeedPrimal = true;
    static constexpr bool kCoefNeedsPrimal = true;
    static constexpr bool kCoefOne = false;
    static constexpr bool kCoefIsA = false;
    using P = ScalarP<T>;
    __device__ static P pid() { return {-pos_inf<T>()}; }
    __device__ static P pcomb(P l, P r) { return {r.v > l.v ? r.v : l.v}; }
    __device__ static P pelem(T a, T) { return {a}; }
    __device__ static T pad_a() { return -pos_inf<T>(); }
    __device__ static T coef(P prev, T a) { return prev.v >= a ? T(1) : T(0); }
    __device__ static void vjp_right(P prev, T a, T, T ra, T, T& oa, T&) {
        oa = a > prev.v ? ra : T(0);
    }
    // the extremum's lowest index: strictly above everything before it, at
    // least everything after it
    __device__ static void mid_vjp(P l, T a, T, P r, T ya, T, T& oa, T&) {
        oa = (a > l.v && a >= r.v) ? ya : T(0);
    }
    __device__ static P tcomb(P l, P tl, P r, P tr) { return r.v > l.v ? tr : tl; }  // ties: the earlier
    __device__ static T out_a(P p) { return p.v; }
    __device__ static T out_b(P) { return T(0); }
};

template <class T>
struct OpMin {
    static constexpr int kWidth = 1;
    static constexpr bool kNeedPrimal = true;
    static constexpr bool kCoefNeedsPrimal = true;
    static constexpr bool kCoefOne = false;
    static constexpr bool kCoefIsA = false;
    using P = ScalarP<T>;
    __device__ static P pid() { return {pos_inf<T>()}; }
    __device__ static P pcomb(P l, P r) { return {r.v < l.v ? r.v : l.v}; }
    __device__ static P pelem(T a, T) { return {a}; }
    __device__ static T pad_a() { return pos_inf<T>(); }
    __device__ static T coef(P prev, T a) { return prev.v <= a ? T(1) : T(0); }
    __device__ static void vjp_right(P prev, T a, T, T ra, T, T& oa, T&) {
        oa = a < prev.v ? ra : T(0);
    }
    __device__ static void mid_vjp(P l, T a, T, P r, T ya, T, T& oa, T&) {
        oa = (a < l.v && a <= r.v) ? ya : T(0);
    }
    __device__ static P tcomb(P l, P tl, P r, P tr) { return r.v < l.v ? tr : tl; }
    __device__ static T out_a(P p) { return p.v; }
    __device__ static T out_b(P) { return T(0); }
};

// Linear recurrence (a1,b1) (.) (a2,b2) = (a2*a1, a2*b1 + b2).
//   J_left(i)  = a_i * I
//   J_right(i) = [[A_{i-1}, 0], [B_{i-1}, 1]]  (rows A,B; columns a,b)
// so J_right^T rs_bar = (A_{i-1} rA + B_{i-1} rB, rB).
template <class T>
struct OpLinrec {
    static constexpr int kWidth = 2;
    static constexpr bool kNeedPrimal = true;
    static constexpr bool kCoefNeedsPrimal = false;
    static constexpr bool kCoefOne = false;
    static constexpr bool kCoefIsA = true;
    using P = PairP<T>;
    __device__ static P pid() { return {T(1), T(0)}; }
    __device__ static P pcomb(P l, P r) { return {r.A * l.A, fma(r.A, l.B, r.B)}; }
    __device__ static P pelem(T a, T b) { return {a, b}; }
    __device__ static T pad_a() { return T(1); }
    __device__ static T coef(P, T a) { return a; }
    __device__ static void vjp_right(P prev, T, T, T ra, T rb, T& oa, T& ob) {
        oa = fma(prev.A, ra, prev.B * rb);
        ob = rb;
    }
    // y = l (.) (a, b) (.) r = (rA a lA, rA (a lB + b) + rB):
    //   dy/da = (rA lA, rA lB),  dy/db = (0, rA)
    __device__ static void mid_vjp(P l, T, T, P r, T ya, T yb, T& oa, T& ob) {
        oa = r.A * fma(l.A, ya, l.B * yb);
        ob = r.A * yb;
    }
    // d(rA lA, rA lB + rB) = (trA lA + rA tlA, trA lB + rA tlB + trB)
    __device__ static P tcomb(P l, P tl, P r, P tr) {
        return {fma(tr.A, l.A, r.A * tl.A), fma(tr.A, l.B, fma(r.A, tl.B, tr.B))};
    }
    __device__ static T out_a(P p) { return p.A; }
    __device__ static T out_b(P p) { return p.B; }
};

// State of the lin_o scan of Sec. 5.2: the affine map x -> d + c x, where d
// has one component per element array and c is the scalar J_left factor.
// combine(e, l) composes "l after e" (e earlier in the scan order):
//   x -> l.d + l.c (e.d + e.c x) = (l.d + l.c e.d) + (l.c e.c) x,
// which is lin_o (d1,c1) (d2,c2) = (d2 + c2 d1, c2 c1); neutral (0, 1).
template <class T, int W, bool HasC>
struct Lin;

template <class T, int W>
struct Lin<T, W, true> {
    T d[W];
    T c;
    __device__ static Lin id() {
        Lin r;
#pragma unroll
        for (int i = 0; i < W; ++i) r.d[i] = T(0);
        r.c = T(1);
        return r;
    }
    __device__ static Lin comb(const Lin& e, const Lin& l) {
        Lin r;
#pragma unroll
        for (int i = 0; i < W; ++i) r.d[i] = fma(l.c, e.d[i], l.d[i]);
        r.c = l.c * e.c;
        return r;
    }
};

template <class T, int W>
struct Lin<T, W, false> {  // c == 1 always (ADD): plain sums
    T d[W];
    __device__ static Lin id() {
        Lin r;
#pragma unroll
        for (int i = 0; i < W; ++i) r.d[i] = T(0);
        return r;
    }
    __device__ static Lin comb(const Lin& e, const Lin& l) {
        Lin r;
#pragma unroll
        for (int i = 0; i < W; ++i) r.d[i] = e.d[i] + l.d[i];
        return r;
    }
};

}  // namespace adpar
