// Float-float arithmetic for the track fits on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2: about 48 significant bits. The building blocks are the
// error-free transformations TwoSum (Knuth), Fast2Sum (Dekker) and the
// FMA-based TwoProd, combined as in the double-word algorithms analysed by
// Joldes, Muller and Popescu (ACM Trans. Math. Softw. 44(2), 2017): each
// operation below has a relative error of a few units of 2^-46. The _rn
// intrinsics keep the compiler from contracting or reordering the error terms.
#pragma once

namespace lst {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_of(float a) { return ff{a, 0.f}; }
__device__ __forceinline__ double ff_d(ff a) { return double(a.hi) + double(a.lo); }

// a + b exactly (TwoSum)
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// a + b exactly when |a| >= |b| or a == 0 (Fast2Sum)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a b exactly (TwoProd with an FMA)
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff operator-(ff x) { return ff{-x.hi, -x.lo}; }

// x + y, accurate also under cancellation (AccurateDWPlusDW)
__device__ __forceinline__ ff operator+(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
    const ff v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }

// x + b (DWPlusFP)
__device__ __forceinline__ ff operator+(ff x, float b) {
    const ff s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}
__device__ __forceinline__ ff operator-(ff x, float b) { return x + (-b); }

// x b (DWTimesFP with an FMA)
__device__ __forceinline__ ff operator*(ff x, float b) {
    const ff c = two_prod(x.hi, b);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, b, c.lo));
}

// x y (DWTimesDW with FMAs)
__device__ __forceinline__ ff operator*(ff x, ff y) {
    const ff c = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}

// x / y: an approximate FP32 quotient (a few ulp), corrected once by the
// float-float remainder x - y q; the correction's own relative error (a few
// ulp of a term ~1e-7 of q) leaves the result within a few units of 2^-46.
__device__ __forceinline__ ff operator/(ff x, ff y) {
    const float ry = __fdividef(1.f, y.hi);
    const float q = __fmul_rn(x.hi, ry);
    const ff r = x - y * q;
    return fast_two_sum(q, __fmul_rn(r.hi, ry));
}
__device__ __forceinline__ ff operator/(ff x, float b) {
    const float rb = __fdividef(1.f, b);
    const float q = __fmul_rn(x.hi, rb);
    const ff r = x - two_prod(q, b);
    return fast_two_sum(q, __fmul_rn(r.hi, rb));
}

// sqrt(x) for x >= 0 (0 otherwise): an approximate FP32 root through the
// reciprocal square root, corrected once by the float-float residual x - s^2
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.f)) return ff{0.f, 0.f};
    const float rs = rsqrtf(x.hi);
    const float s = __fmul_rn(x.hi, rs);
    const ff p = two_prod(s, s);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    return fast_two_sum(s, __fmul_rn(d, __fmul_rn(0.5f, rs)));
}

__device__ __forceinline__ ff ff_abs(ff x) { return x.hi < 0.f ? -x : x; }

// Taylor coefficients of asin(u) / u = sum_n c_n u^(2n),
// c_n = (2n)! / (4^n (n!)^2 (2n + 1)).
__host__ __device__ constexpr double asin_coef(int n) {
    double p = 1.0;
    for (int k = 1; k <= n; ++k) p *= double(2 * k - 1) / double(2 * k);
    return p / double(2 * n + 1);
}

// sum_{n = m..12} c_n x^(n - m), by Horner
template <int m> __device__ __forceinline__ float asin_tail(float x) {
    constexpr float c = float(asin_coef(m));
    if constexpr (m == 12) return c;
    else return __fmaf_rn(asin_tail<m + 1>(x), x, c);
}

// asin(v) / v - 1 for 0 <= v <= 1/2: the v^2 / 6 and 3 v^4 / 40 terms in
// float-float and the rest (below 1e-3 for v <= 1/2) in FP32, with the series
// cut after v^24 (remainder below 1e-10).
__device__ __forceinline__ ff asin_ratio_m1(ff v) {
    const ff v2 = v * v, v4 = v2 * v2;
    const float x = v2.hi;
    return v2 / 6.f + v4 * 3.f / 40.f + __fmul_rn(asin_tail<3>(x), __fmul_rn(x, v4.hi));
}

// 2 asin(u) / ka for the arc of chord c on a circle of curvature ka >= 0,
// with u = c ka / 2 clipped to 1; c itself for ka = 0. Below u = 1/2 the arc
// is c (1 + (asin(u)/u - 1)); above, asin(u) = pi/2 - 2 asin(v) with
// v = sqrt((1 - u) / 2) <= 1/2 (the half-angle identity).
__device__ __forceinline__ ff ff_arc(ff c, ff ka) {
    ff u = c * ka * 0.5f;
    if (u.hi > 1.f) u = ff{1.f, 0.f};
    if (u.hi <= 0.5f) return c + c * asin_ratio_m1(u);
    const ff v = ff_sqrt((ff{1.f, 0.f} - u) * 0.5f);
    const ff asin_v = v + v * asin_ratio_m1(v);
    // pi/2 as a float-float constant
    const ff half_pi{1.57079637050628662f, -4.37113900018624283e-8f};
    return (half_pi - asin_v * 2.f) * 2.f / ka;
}

}  // namespace lst
