// plic_math.cuh -- scalar math for the PLIC kernels, per precision.
//
// Fm<float>  : the FP32 fast path: MUFU-based sin/cos (__sinf/__cosf), MUFU
//              reciprocal and reciprocal square root for division and sqrt, a
//              cube root from the MUFU exp2/log2 pair refined by one Newton
//              step, and arcsine/arccosine/polar angle from one arcsine series.
// Fm<double> : plain double-precision library functions.
//
// Constants are written as their closed forms (the decimals printed in the
// paper's listings are the FP32 roundings of these, Sec. 2.3 Eqs. 13-22).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace plic {

template <typename T> struct Fm;

// MUFU reciprocal (about 1 ulp; denormal inputs and results flush to zero).
// It gives the same values as __fdividef(1, x) in these kernels with fewer
// instructions (measured on the fused PLIC step: 1.386 -> 1.255 ms, output
// bit-identical).  a / b is a * rcp_approx(b): for 2^126 < |b| the reciprocal
// lies below the normal range and flushes to 0, as __fdividef's quotient
// does.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Arcsine for |x| <= 1 on the FP32 pipes, from the Maclaurin series of
// arcsin, asin(s) = sum_k C(2k,k) / (4^k (2k+1)) s^(2k+1), truncated after
// s^17 and used only for s <= 1/2 (truncation error < 2.4e-8), with the
// half-angle reduction asin(x) = pi/2 - 2 asin(sqrt((1 - x)/2)) for x > 1/2.
__device__ __forceinline__ float fast_asinf(float x) {
    const float a = fabsf(x);
    const bool big = a > 0.5f;
    const float z = big ? 0.5f * (1.0f - a) : a * a;
    const float s = big ? (z > 0.0f ? z * rsqrtf(z) : 0.0f) : a;
    float p = 0.011551800896139705f;                 // 6435/557056
    p = fmaf(p, z, 0.01396484375f);                  // 143/10240
    p = fmaf(p, z, 0.017352764423076924f);           // 231/13312
    p = fmaf(p, z, 0.022372159090909092f);           // 63/2816
    p = fmaf(p, z, 0.030381944444444444f);           // 35/1152
    p = fmaf(p, z, 0.044642857142857144f);           // 5/112
    p = fmaf(p, z, 0.075f);                          // 3/40
    p = fmaf(p, z, 0.16666666666666666f);            // 1/6
    p = fmaf(s * z, p, s);
    const float r = big ? fmaf(-2.0f, p, 1.5707963267948966f) : p;
    return copysignf(r, x);
}

template <> struct Fm<float> {
    typedef float T;
    // sqrt and division: MUFU-based (rsqrt, rcp) forms; 1-2 ulp, enough for a
    // solver whose result is either used as is (FP32) or Newton-polished
    static __device__ __forceinline__ T sqrt_(T x) {
        return x > 0.0f ? x * rsqrtf(x) : (x == 0.0f ? 0.0f : __int_as_float(0x7fffffff));
    }
    static __device__ __forceinline__ T rsqrt_(T x) { return rsqrtf(x); }
    // Cube root for x >= 0: 2^(log2(x)/3) from the MUFU pair (about 2^-22
    // relative), then one Newton step on r^3 = x, r <- r - (r^3 - x)/(3 r^2).
    static __device__ __forceinline__ T cbrt_(T x) {
        if (!(x > 0.0f)) return 0.0f;
        float s = 1.0f;
        if (x < 1e-30f) { x *= 4.7223665e21f; s = 5.9604645e-08f; }   // 2^72, 2^-24
        float r = exp2f_approx(__log2f_approx(x) * (1.0f / 3.0f));
        float r2 = r * r;
        return s * fmaf(-(r2 * r - x), rcp_approx(3.0f * r2), r);
    }
    static __device__ __forceinline__ T sin_(T x) { return __sinf(x); }
    // sine of an angle in [-pi/6, pi/6] (the roots' angles): the MUFU sine
    static __device__ __forceinline__ T sin_pi6_(T x) { return __sinf(x); }
    static __device__ __forceinline__ T cos_(T x) { return __cosf(x); }
    static __device__ __forceinline__ T asin_(T x) { return fast_asinf(x); }
    static __device__ __forceinline__ T acos_(T x) { return 1.5707963267948966f - fast_asinf(x); }
    // atan2(y, x) for x, y >= 0 from sine and cosine: the arcsine of the
    // smaller of y/r and x/r (at most 1/sqrt 2), reflected about pi/4 where
    // y > x; the arcsine of a sine near 1 would lose half the digits
    static __device__ __forceinline__ T polar_angle_(T x, T y) {
        const float r2 = fmaf(x, x, y * y);
        if (!(r2 > 0.0f)) return 0.0f;
        const float ir = rsqrtf(r2);
        const float a = fast_asinf(fminf(fminf(x, y) * ir, 1.0f));
        return y <= x ? a : 1.5707963267948966f - a;
    }
    static __device__ __forceinline__ T div_(T a, T b) { return a * rcp_approx(b); }
    static __device__ __forceinline__ T rcp_(T a) { return rcp_approx(a); }
    static __device__ __forceinline__ T fdim_(T a, T b) { return fmaxf(a - b, 0.0f); }
    static __device__ __forceinline__ T tiny() { return 1.17549435e-38f; }   // FLT_MIN
    static __device__ __forceinline__ T eps() { return 5.9604645e-08f; }    // 2^-24
    // binary exponent floor(log2 |w|) (the library's ilogb)
    static __device__ __forceinline__ int ilogb_(T w) { return ilogbf(w); }
    static __device__ __forceinline__ float exp2f_approx(float x) {
        float r;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float __log2f_approx(float x) {
        float r;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
};

template <> struct Fm<double> {
    typedef double T;
    static __device__ __forceinline__ T sqrt_(T x) { return sqrt(x); }
    static __device__ __forceinline__ T rsqrt_(T x) { return rsqrt(x); }
    static __device__ __forceinline__ T cbrt_(T x) { return cbrt(x); }
    static __device__ __forceinline__ T sin_(T x) { return sin(x); }
    // Sine of an angle |x| <= pi/6 (the trigonometric roots' angles) by its
    // Taylor series through x^15: the first omitted term, (pi/6)^17 / 17!, is
    // below 5e-20, so the result is the double rounding of the sum (Horner in
    // x^2, coefficients -1/(2k+1)!..., exact rationals rounded once); 10 FP64
    // operations against the library sine's argument reduction and wider range.
    static __device__ __forceinline__ T sin_pi6_(T x) {
        const T z = x * x;
        T p = -7.6471637318198164759e-13;                  // -1/15!
        p = fma(p, z, 1.6059043836821614599e-10);          //  1/13!
        p = fma(p, z, -2.5052108385441718775e-08);         // -1/11!
        p = fma(p, z, 2.7557319223985890653e-06);          //  1/9!
        p = fma(p, z, -1.9841269841269841270e-04);         // -1/7!
        p = fma(p, z, 8.3333333333333333333e-03);          //  1/5!
        p = fma(p, z, -1.6666666666666666667e-01);         // -1/3!
        return fma(x * z, p, x);
    }
    static __device__ __forceinline__ T cos_(T x) { return cos(x); }
    static __device__ __forceinline__ T asin_(T x) { return asin(x); }
    static __device__ __forceinline__ T acos_(T x) { return acos(x); }
    static __device__ __forceinline__ T polar_angle_(T x, T y) { return atan2(y, x); }
    static __device__ __forceinline__ T div_(T a, T b) { return a / b; }
    static __device__ __forceinline__ T rcp_(T a) { return 1.0 / a; }
    static __device__ __forceinline__ T fdim_(T a, T b) { return fmax(a - b, 0.0); }
    static __device__ __forceinline__ T tiny() { return 2.2250738585072014e-308; }  // DBL_MIN
    static __device__ __forceinline__ T eps() { return 1.1102230246251565e-16; }    // 2^-53
    static __device__ __forceinline__ int ilogb_(T w) { return ilogb(w); }
};

// Closed-form constants (Sec. 2.3, Eqs. 13-22; Sec. 2.4).  The two_* values are
// the factor 2 of Eq. 11 folded into a3, b3, a4, b4 (the FP32 paired solver).
template <typename T> struct Kc {
    static constexpr T cbrt54 = (T)3.7797631496846195;             // 54^(1/3)       (a3 / n1 n2)
    static constexpr T inv_cbrt432 = (T)0.13228342099734996;       // 1 / 432^(1/3)  (b3)
    static constexpr T inv_cbrt864 = (T)0.10499342082457276;       // 1 / 864^(1/3)  (a4 / t4)
    static constexpr T inv_cbrt3456 = (T)0.066141710498674978;     // 1 / 3456^(1/3) (b4)
    static constexpr T two_cbrt54 = (T)7.559526299369239;          // 2 * 54^(1/3)
    static constexpr T two_over_cbrt432 = (T)0.26456684199469993;  // 2 / 432^(1/3)
    static constexpr T two_over_cbrt864 = (T)0.20998684164914555;  // 2 / 864^(1/3)
    static constexpr T two_over_cbrt3456 = (T)0.13228342099734997; // 2 / 3456^(1/3)
    static constexpr T inv_sqrt12 = (T)0.28867513459481287;        // 1 / sqrt(12)
    static constexpr T pi_6 = (T)0.52359877559829887;              // pi / 6
    static constexpr T four_pi = (T)12.566370614359173;            // 4 pi
    static constexpr T third = (T)0.33333333333333333;
    static constexpr T twelfth = (T)0.083333333333333333;
};

template <typename T> __device__ __forceinline__ T sq(T x) { return x * x; }
template <typename T> __device__ __forceinline__ T cb(T x) { return x * x * x; }

}  // namespace plic
