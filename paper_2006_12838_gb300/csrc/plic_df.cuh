// plic_df.cuh -- double-float arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48
// significant bits.  Built from the error-free transformations two-sum
// (Knuth) and two-product via FMA (Dekker; Ogita, Rump and Oishi).
//
// Used where FP64 accuracy is wanted without the FP64 pipe (small on GB300):
// the FP64_REFINED offset (Newton steps on Eq. 10 in double-float) and the
// double-float fit of the curvature step.  Doubles enter and leave through
// integer bit manipulation (d2df, df2d), not through the FP64 units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace plic {

struct df { float hi, lo; };
__device__ __forceinline__ df df_make(float a) { return {a, 0.0f}; }
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}
// double-float times float
__device__ __forceinline__ df df_mul_f(df a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return quick_two_sum(p, e);
}
// times a power of two (exact)
__device__ __forceinline__ df df_scale(df a, float two_k) { return {a.hi * two_k, a.lo * two_k}; }
__device__ __forceinline__ df df_div(df a, df b) {
    const float q1 = a.hi / b.hi;
    const df r = df_add(a, df_neg(df_mul(b, df_make(q1))));
    const float q2 = r.hi / b.hi;
    return quick_two_sum(q1, q2);
}
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ df df_max0(df a) { return a.hi > 0.0f ? a : df_make(0.0f); }
__device__ __forceinline__ df df_clamp(df a, df lo, df hi) {
    return df_lt(a, lo) ? lo : (df_lt(hi, a) ? hi : a);
}

// A double as a double-float, by integer operations on its bits.  hi holds the
// leading 24 bits of the significand (truncated), lo the next 29 rounded to a
// float, so hi + lo equals x to 2^-48 relative.  Magnitudes below 2^-126 (the
// float normal range) become 0, above 2^127 infinity; NaN stays NaN.
__device__ __forceinline__ df d2df(double x) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const uint32_t sgn = (uint32_t)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7FF);
    const uint64_t m = u & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return {__uint_as_float(sgn | 0x7F800000u | (m ? 0x400000u : 0u)), 0.0f};
    const int E = e - 1023;
    if (E < -126) return {__uint_as_float(sgn), 0.0f};
    if (E > 127) return {__uint_as_float(sgn | 0x7F800000u), 0.0f};
    const float hi = __uint_as_float(sgn | ((uint32_t)(E + 127) << 23) | (uint32_t)(m >> 29));
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFull);     // the 29 bits below hi
    float lo = 0.0f;
    if (r != 0u && E <= 100) {
        // r * 2^(E - 52) = r * 2^(E + 12) * 2^-64, both factors in range
        lo = __uint2float_rn(r) * __uint_as_float((uint32_t)(E + 12 + 127) << 23) *
             __uint_as_float(0x1F800000u);           // 2^-64
        if (sgn) lo = -lo;
    }
    return quick_two_sum(hi, lo);
}

// K 2^-53 as a double-float (0 <= K < 2^53): K is normalised so that its
// leading bit is bit 52, then its top 24 bits (exact) and the next 29 bits
// (rounded) become the two floats, 2^-48 relative.  32-bit conversions only
// (the 64-bit integer conversions run on the FP64 pipe).
__device__ __forceinline__ df df_from_u64_2m53(uint64_t K) {
    if (K == 0ull) return df_make(0.0f);
    const int s = __clzll((long long)K) - 11;                  // K << s in [2^52, 2^53)
    const uint64_t Kn = K << s;
    const float hf = __uint2float_rn((uint32_t)(Kn >> 29));    // < 2^24: exact
    const float lf = __uint2float_rn((uint32_t)(Kn & 0x1FFFFFFFull));
    // hi * 2^(29 - 53 - s), lo * 2^(-53 - s): exponents in [-105, -24]
    const float shi = __uint_as_float((uint32_t)(127 - 24 - s) << 23);
    const float slo = __uint_as_float((uint32_t)(127 - 53 - s) << 23);
    return quick_two_sum(hf * shi, lf * slo);
}

// A float as a double, by integer operations (exact for normal floats; zero
// for float denormals, whose magnitude is below 2^-126).
__device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sgn = (uint64_t)(u >> 31) << 63;
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0u) return __longlong_as_double((long long)sgn);
    if (e == 0xFFu)
        return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull |
                                                ((u & 0x7FFFFFu) ? 0x8000000000000ull : 0ull)));
    return __longlong_as_double(
        (long long)(sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// A double-float as a double: both parts converted exactly, one FP64 add
// (exact: hi + lo has at most 48 significant bits).
__device__ __forceinline__ double df2d(df a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace plic
