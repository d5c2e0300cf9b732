// plic_pair.cuh -- the FP32 fast paths of the optimised and of Kawano's SZ
// solution (Sec. 2.4) and of the analytic solution (Sec. 2.3) for two cells
// at once, on the paired FP32 instructions of sm_100+ (one FFMA2/FADD2/FMUL2
// issues two FP32 operations).  Comparisons, selects and
// MUFU operations stay per component.
//
// The arithmetic is that of solve_sz_opt_default<float> + polish (see
// plic_solvers.cuh): the division-free case tests, the cancellation-free
// arcsine argument, all cases evaluated and selected, and, for the polished
// precision, one Newton step on the cubic of Eq. 10 for the cells whose root
// came from the trigonometric formula (cases 3/4; the closed forms of cases
// 1, 2, 5 are already accurate to a few ulp).
#pragma once
#include "plic_solvers.cuh"

namespace plic {
namespace p2 {

typedef float2 f2;

__device__ __forceinline__ f2 mk(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return __ffma2_rn(b, mk(-1.0f), a); }
__device__ __forceinline__ f2 fmax0(f2 a) { return make_float2(fmaxf(a.x, 0.0f), fmaxf(a.y, 0.0f)); }

struct b2 { bool x, y; };
__device__ __forceinline__ f2 sel(b2 c, f2 a, f2 b) { return make_float2(c.x ? a.x : b.x, c.y ? a.y : b.y); }
__device__ __forceinline__ b2 lt(f2 a, f2 b) { return {a.x < b.x, a.y < b.y}; }
__device__ __forceinline__ b2 le(f2 a, f2 b) { return {a.x <= b.x, a.y <= b.y}; }

__device__ __forceinline__ f2 rsqrt(f2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ f2 rcp(f2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ f2 sqrt_(f2 a) {
    return make_float2(Fm<float>::sqrt_(a.x), Fm<float>::sqrt_(a.y));
}

// cube root of x >= 0 as MUFU exp2(log2(x)/3): relative error below 6e-6
// even for x = 1e-30 (the MUFU log2's absolute error, times |log2 x|/3), and
// the cube root is only the case-(1) offset d1 <= n1, whose absolute error
// then stays below 2e-7 -- no Newton step.  1e-30 is added to x (its cube root,
// 1e-10, is far below the FP32 resolution of an offset), which removes the
// zero/denormal branches on the FMA pipe.
__device__ __forceinline__ f2 cbrt_(f2 x) {
    x = add(x, mk(1e-30f));
    return make_float2(Fm<float>::exp2f_approx(Fm<float>::__log2f_approx(x.x) * (1.0f / 3.0f)),
                       Fm<float>::exp2f_approx(Fm<float>::__log2f_approx(x.y) * (1.0f / 3.0f)));
}

// The same cube root with one Newton step (relative error at FP32 rounding):
// for the analytic solution, whose trigonometric root scales with u^(1/2).
__device__ __forceinline__ f2 cbrt_nr(f2 x) {
    const f2 r = cbrt_(x);
    const f2 r2 = mul(r, r);
    const f2 res = fma(r2, r, make_float2(-x.x - 1e-30f, -x.y - 1e-30f));     // r^3 - x
    return fma(make_float2(-res.x, -res.y), rcp(mul(mk(3.0f), r2)), r);
}

// sqrt of x >= 0 as x rsqrt(x) with 1e-30 added (no zero branch).  Both
// callers pass arguments that are >= 0 wherever the result is used: the
// arcsine's 1/2 (1 - a) with a <= 1, and the case-(2) radicand
// 8 n2 n3 V - n1^2/3, which is >= n1^2 in case (2) and exactly 8 n2 n3 V >= 0
// for n1 = 0.
__device__ __forceinline__ f2 sqrtp(f2 x) {
    x = add(x, mk(1e-30f));
    return mul(x, rsqrt(x));
}

// arcsine on [0, 1], two lanes at once: asin(s) = s + s^3 P(s^2) on
// s <= 1/2 with P a degree-4 least-squares fit to (asin(s) - s)/s^3 on
// [0, 1/4] (relative error below 2e-8, under the FP32 rounding), and the
// half-angle reduction asin(a) = pi/2 - 2 asin(sqrt((1 - a)/2)) above 1/2.
// The optimised-SZ argument is never negative: it is 1.5 n1 n2 (n1+n2-2 n3 V)/t^3
// with n1+n2 > 2 n3 V outside case (5), or 0.75 n1 n2 n3 (1-2V)/t^3 with V <= 1/2.
__device__ __forceinline__ f2 asin01(f2 a) {
    const b2 big = lt(mk(0.5f), a);
    const f2 zb = mul(mk(0.5f), sub(mk(1.0f), a));
    const f2 z = sel(big, zb, mul(a, a));
    const f2 s = sel(big, sqrtp(z), a);
    f2 p = mk(0.038206491619348526f);
    p = fma(p, z, mk(0.026494324207305908f));
    p = fma(p, z, mk(0.045010678470134735f));
    p = fma(p, z, mk(0.07498809695243835f));
    p = fma(p, z, mk(0.16666673123836517f));
    p = fma(mul(s, z), p, s);
    return sel(big, fma(mk(-2.0f), p, mk(1.5707963267948966f)), p);
}

// One Newton step on the cubic of Eq. 10 for cases (3)/(4) (d >= n2, n1 > 0),
// with g and g' multiplied through by n1 so that one reciprocal serves:
// n1 g = n1 (3 d (d - n1) + n1^2) - (d - n2)^3 - (d - n3)_+^3 - 6 n1 n2 n3 V,
// n1 g' = n1 (6 d - 3 n1) - 3 ((d - n2)^2 + (d - n3)_+^2) = 12 n1 n2 n3 x area > 0.
// V6 = 6 n1 n2 n3 V.
__device__ __forceinline__ f2 polish34(f2 d, f2 V6, f2 n1, f2 n2, f2 n3) {
    const f2 e2 = sub(d, n2), e3 = fmax0(sub(d, n3));
    const f2 e22 = mul(e2, e2), e33 = mul(e3, e3);
    const f2 cub = fma(e22, e2, mul(e33, e3));
    const f2 dd = sub(d, n1);
    f2 g = mul(n1, fma(mk(3.0f), mul(d, dd), mul(n1, n1)));
    g = sub(g, add(cub, V6));
    f2 gp = mul(n1, fma(mk(6.0f), d, mul(mk(-3.0f), n1)));
    gp = fma(mk(-3.0f), add(e22, e33), gp);
    return sub(d, mul(g, rcp(gp)));
}

// Reduced optimised-SZ solution for two cells (L1-normalised m1 <= m2 <= m3,
// reduced volume V).  The trigonometric root of cases (3)/(4) is formed (and,
// with POLISH, given its Newton step) first; the closed forms of cases (2),
// (1) and (5) then replace it, each select right after its test, so that no
// case flag stays live across the long trigonometric chain.
template <bool POLISH>
__device__ __forceinline__ f2 sz_opt(f2 V, f2 n1, f2 n2, f2 n3) {
    const f2 n12 = add(n1, n2), n3V = mul(n3, V);
    const f2 n3V2 = add(n3V, n3V);
    const f2 V6n2n3 = mul(mul(mk(6.0f), n2), n3V), sqn1 = mul(n1, n1);
    const f2 n1n2 = mul(n1, n2);
    // case (3) vs (4): 6 n1 n2 n3 V < n3^2 (3 n12 - n3) + n1^2 (n1 - 3 n3) + n2^2 (n2 - 3 n3)
    f2 num3 = mul(mul(n3, n3), fma(mk(3.0f), n12, make_float2(-n3.x, -n3.y)));
    num3 = fma(sqn1, fma(mk(-3.0f), n3, n1), num3);
    num3 = fma(mul(n2, n2), fma(mk(-3.0f), n3, n2), num3);
    const b2 n3small = lt(n3, n12);
    const f2 V6n1n2n3 = mul(V6n2n3, n1);
    const b2 v3lt = lt(V6n1n2n3, num3);
    const b2 c3 = {!n3small.x || v3lt.x, !n3small.y || v3lt.y};
    // arcsine argument without cancellation
    const f2 q3 = mul(mul(mk(1.5f), n1n2), sub(n12, n3V2));
    const f2 q4 = mul(mul(mul(mk(0.75f), n1n2), n3), fma(mk(-2.0f), V, mk(1.0f)));
    const f2 d32 = sub(n3, n2);
    const f2 t24 = mul(mk(0.25f), fma(n1, fma(mk(2.0f), add(n2, n3), make_float2(-n1.x, -n1.y)),
                                     make_float2(-d32.x * d32.x, -d32.y * d32.y)));
    const f2 q = sel(c3, q3, q4);
    const f2 t2 = sel(c3, add(n1n2, n1n2), t24);
    const f2 c = sel(c3, n12, mk(0.5f));
    const f2 rt = rsqrt(t2);
    const f2 t = mul(t2, rt);
    f2 arg = mul(q, mul(rt, mul(rt, rt)));
    arg = make_float2(fminf(arg.x, 1.0f), fminf(arg.y, 1.0f));
    const f2 th = mul(mk(0.33333333333333333f), asin01(arg));
    const f2 sn = make_float2(__sinf(th.x), __sinf(th.y));
    f2 d = fma(mul(mk(-2.0f), t), sn, c);
    if (POLISH) d = polish34(d, V6n1n2n3, n1, n2, n3);
    // case (2) where 3 n2 (2 n3 V + n1 - n2) < n1^2, unless case (1) holds
    const f2 t2a = mul(mul(mk(3.0f), n2), add(n3V2, sub(n1, n2)));
    const f2 d2 = mul(mk(0.5f), add(n1, sqrtp(fma(mk(8.0f), mul(n2, n3V), mul(mk(-0.33333333333333333f), sqn1)))));
    d = sel(lt(t2a, sqn1), d2, d);
    // case (1) where 6 n2 n3 V < n1^2
    const f2 d1 = cbrt_(V6n1n2n3);
    d = sel(lt(V6n2n3, sqn1), d1, d);
    // case (5) where n1 + n2 <= 2 n3 V
    const f2 d5 = fma(mk(0.5f), n12, n3V);
    return sel(le(n12, n3V2), d5, d);
}

// Kawano's Scardovelli-Zaleski solution (Sec. 2.4) for two cells, in the
// L1-normalised reduced space (m1 <= m2 <= m3, w the reduced volume), with
// the arithmetic of sz_orig_easy/sz_orig_hard<float> (plic_solvers.cuh): its
// volume thresholds Vb1 = m1^2/(6 m2 m3 + 1e-25) and Vb2 = Vb1 + (m2 -
// m1)/(2 m3), the case-(3) end Vb3 (the case-(5) threshold m12/(2 m3) when m3
// >= m1 + m2, else the volume of the plane through the vertex m3), and
// Viete's root of the monic cubic with s^2 and -q/2 multiplied out.  Every
// case is evaluated and the selects follow that implementation's order: (1),
// (2), then (5) unless its offset is 0 (that implementation then solves the
// case-(4) cubic, which gives NaN for m = (0, 0, 1), w = 0 through s^2 = -1/4),
// else (3)/(4).  With POLISH the root of cases (3)/(4) gets one Newton step;
// the closed forms are accurate as they are.
template <bool POLISH>
__device__ __forceinline__ f2 sz_orig(f2 w, f2 m1, f2 m2, f2 m3) {
    typedef Fm<float> F;
    const f2 m12 = add(m1, m2), m1m2 = mul(m1, m2);
    const f2 e3 = mul(m1m2, m3), sqm1 = mul(m1, m1);
    const f2 ir3 = rcp(m3);
    const f2 vb1 = mul(sqm1, rcp(fma(mk(6.0f), mul(m2, m3), mk(1e-25f))));
    const f2 vb2 = fma(mul(mk(0.5f), sub(m2, m1)), ir3, vb1);
    const b2 tall = {!(m3.x < m12.x), !(m3.y < m12.y)};
    const f2 vb5 = mul(mul(mk(0.5f), m12), ir3);
    const f2 d31 = sub(m3, m1), d32 = sub(m3, m2);
    const f2 cub3 = sub(mul(mul(m3, m3), m3),
                        fma(mul(d31, d31), d31, mul(mul(d32, d32), d32)));
    const f2 vb3 = sel(tall, vb5, mul(cub3, rcp(mul(mk(6.0f), e3))));
    const b2 c3 = lt(w, vb3);
    // Viete: s^2, -q/2 and the shift -a2/3 of the case
    const f2 s24 = mul(mk(0.25f), fma(m1, fma(mk(2.0f), add(m2, m3), make_float2(-m1.x, -m1.y)),
                                      make_float2(-d32.x * d32.x, -d32.y * d32.y)));
    const f2 s2 = sel(c3, add(m1m2, m1m2), s24);
    const f2 mq2 = sel(c3, mul(mul(mk(1.5f), m1m2), fma(mk(-2.0f), mul(m3, w), m12)),
                       mul(mul(mk(0.75f), e3), fma(mk(-2.0f), w, mk(1.0f))));
    const f2 shift = sel(c3, m12, mk(0.5f));
    const f2 s = make_float2(F::sqrt_(s2.x), F::sqrt_(s2.y));
    f2 r = mul(mq2, rcp(mul(s2, s)));
    r = make_float2(fminf(fmaxf(r.x, -1.0f), 1.0f), fminf(fmaxf(r.y, -1.0f), 1.0f));
    const f2 ang = mul(mk(0.33333333333333333f),
                       make_float2(F::acos_(r.x) + 12.566370614359172f, F::acos_(r.y) + 12.566370614359172f));
    f2 d = fma(add(s, s), make_float2(__cosf(ang.x), __cosf(ang.y)), shift);
    if (POLISH) d = polish34(d, mul(mul(mk(6.0f), e3), w), m1, m2, m3);
    // case (5): tall and w >= m12 / (2 m3), unless its offset is 0
    const f2 d5 = fma(m3, w, mul(mk(0.5f), m12));
    const b2 c5 = {tall.x && !(w.x < vb5.x) && d5.x != 0.0f, tall.y && !(w.y < vb5.y) && d5.y != 0.0f};
    d = sel(c5, d5, d);
    // case (2) below Vb2, case (1) below Vb1
    const f2 d2 = fma(mk(0.5f), m1, sqrtp(fma(mul(mk(2.0f), mul(m2, m3)), w,
                                              mul(mk(-0.083333333333333333f), sqm1))));
    d = sel(lt(w, vb2), d2, d);
    const f2 d1 = cbrt_(mul(mul(mk(6.0f), e3), w));
    return sel(lt(w, vb1), d1, d);
}

// The paper's analytic solution (Sec. 2.3, Eq. 25 with the tests of Eq. 24)
// for two cells, in the reduced space of the unit normal (n1 <= n2 <= n3,
// |n| = 1, V the reduced volume).  As in sz_opt: case (3) or (4) is decided
// first from the volume at d = n3 (the test d3 <= n3 of the paper, made before
// forming d3), so that one trigonometric root f(x, y, a, b, c) is evaluated
// with the coefficients of that case; with u^3 = x^2 + y^2 the arctangent
// atan(y/x) (x >= 0 here) is asin(y/u^(3/2)).  With POLISH the root gets
// one Newton step; then the closed forms of cases (2), (1), (5) replace it
// where their tests hold.
template <bool POLISH>
__device__ __forceinline__ f2 analytic(f2 V, f2 n1, f2 n2, f2 n3) {
    typedef Kc<float> K;
    const f2 n12 = add(n1, n2), n3V = mul(n3, V);
    const f2 n3V2 = add(n3V, n3V);
    const f2 V6n2n3 = mul(mul(mk(6.0f), n2), n3V), sqn1 = mul(n1, n1);
    const f2 n1n2 = mul(n1, n2);
    // case (3) vs (4): 6 n1 n2 n3 V < n3^2 (3 n12 - n3) + n1^2 (n1 - 3 n3) + n2^2 (n2 - 3 n3)
    f2 num3 = mul(mul(n3, n3), fma(mk(3.0f), n12, make_float2(-n3.x, -n3.y)));
    num3 = fma(sqn1, fma(mk(-3.0f), n3, n1), num3);
    num3 = fma(mul(n2, n2), fma(mk(-3.0f), n3, n2), num3);
    const b2 n3small = lt(n3, n12);
    const f2 V6n1n2n3 = mul(V6n2n3, n1);
    const b2 v3lt = lt(V6n1n2n3, num3);
    const b2 c3 = {!n3small.x || v3lt.x, !n3small.y || v3lt.y};
    // coefficients: case (3) x3 = 81 n1 n2 (n12 - 2 n3 V), y3^2 = 23328 (n1 n2)^3 - x3^2;
    // case (4) t4 = 9 (n12 + n3)^2 - 18, x4 = n1 n2 n3 (324 - 648 V), y4^2 = 4 t4^3 - x4^2
    const f2 x3 = mul(mul(mk(81.0f), n1n2), sub(n12, n3V2));
    const f2 p3 = mul(mul(n1n2, n1n2), n1n2);
    const f2 y3 = fma(mk(23328.0f), p3, make_float2(-x3.x * x3.x, -x3.y * x3.y));
    const f2 s4 = add(n12, n3);
    const f2 t4 = fma(mk(9.0f), mul(s4, s4), mk(-18.0f));
    f2 x4 = mul(mul(n1n2, n3), fma(mk(-648.0f), V, mk(324.0f)));
    x4 = make_float2(fmaxf(x4.x, 1.17549435e-38f), fmaxf(x4.y, 1.17549435e-38f));
    const f2 y4 = fma(mul(mk(4.0f), t4), mul(t4, t4), make_float2(-x4.x * x4.x, -x4.y * x4.y));
    const f2 x = sel(c3, x3, x4);
    const f2 ysq = fmax0(sel(c3, y3, y4));
    const f2 a = sel(c3, mul(mk(K::two_cbrt54), n1n2), mul(mk(K::two_over_cbrt864), t4));
    const f2 b = sel(c3, mk(K::two_over_cbrt432), mk(K::two_over_cbrt3456));
    const f2 c = sel(c3, n12, mul(mk(0.5f), s4));
    const f2 q = fma(x, x, ysq);                                     // u^3
    const f2 u = cbrt_nr(q);
    // atan(y/x) from sine and cosine: the arcsine of the smaller of the two
    // (<= 1/sqrt 2), reflected about pi/4 where y > x -- the arcsine of a
    // sine near 1 would lose half the digits (x -> 0 near V = 1/2 in case (4)
    // and near the case-(5) boundary in case (3))
    const f2 rq = rsqrt(add(q, mk(1e-30f)));
    const f2 sv = mul(sqrtp(ysq), rq), cv = mul(x, rq);
    const b2 refl = lt(cv, sv);
    const f2 am = sel(refl, cv, sv);
    const f2 as = asin01(make_float2(fminf(am.x, 1.0f), fminf(am.y, 1.0f)));
    const f2 th = mul(mk(0.33333333333333333f), sel(refl, sub(mk(1.5707963267948966f), as), as));
    const f2 ang = sub(mk(K::pi_6), th);
    const f2 sn = make_float2(__sinf(ang.x), __sinf(ang.y));
    f2 d = fma(mul(fma(b, u, a), rsqrt(u)), make_float2(-sn.x, -sn.y), c);
    if (POLISH) d = polish34(d, V6n1n2n3, n1, n2, n3);
    // case (2) where 3 n2 (2 n3 V + n1 - n2) < n1^2, unless case (1) holds
    const f2 t2a = mul(mul(mk(3.0f), n2), add(n3V2, sub(n1, n2)));
    const f2 d2 = fma(mk(0.5f), n1, mul(mk(K::inv_sqrt12),
                                        sqrtp(fma(mk(24.0f), mul(n2, n3V), make_float2(-sqn1.x, -sqn1.y)))));
    d = sel(lt(t2a, sqn1), d2, d);
    // case (1) where 6 n2 n3 V < n1^2 (the plain cube root: d1 <= n1, so its
    // relative error leaves an absolute one below 2e-7, as in sz_opt)
    const f2 d1 = cbrt_(V6n1n2n3);
    d = sel(lt(V6n2n3, sqn1), d1, d);
    // case (5) where n1 + n2 <= 2 n3 V
    const f2 d5 = fma(mk(0.5f), n12, n3V);
    return sel(le(n12, n3V2), d5, d);
}

// Forward volume (Eq. 10) of two cells at their offsets d0, in the cell's
// L1-normalised reduced space (m1 <= m2 <= m3, m1 + m2 + m3 = 1; Eq. 10 is
// homogeneous of degree 0 in (d, n)), il = 1/L:
//   d = 1/2 - |d0|/L (clamped at 0), then case (5) (d - m12/2)/m3 for
//   d >= m1 + m2, case (1) d^3/(6 m1 m2 m3) for d < m1, else
//   (3 d (d - m1) + m1^2 - ((d - m2)_+^3 + (d - m3)_+^3)/m1) / (6 m2 m3),
// and V0 = 1 - V for d0 > 0.
__device__ __forceinline__ f2 volume_reduced(f2 d0, f2 il, f2 m1, f2 m2, f2 m3) {
    const f2 ad = make_float2(fabsf(d0.x), fabsf(d0.y));
    const f2 d = fmax0(fma(make_float2(-ad.x, -ad.y), il, mk(0.5f)));
    // reciprocals: 1/m3 (m3 >= 1/3), 1/m1 and 1/(6 m2 m3), infinite for
    // m1 = 0 / m2 = 0; 1/m1 is capped at FLT_MAX so that the case-(2) term
    // (e2 = e3 = 0 there) stays 0, and the products with an infinite factor
    // belong to cases that the selects below do not take
    const f2 m12 = add(m1, m2);
    const f2 v5 = mul(fma(mk(-0.5f), m12, d), rcp(m3));
    const f2 r1 = rcp(m1), r23 = rcp(mul(mk(6.0f), mul(m2, m3)));
    const f2 v1 = mul(mul(mul(d, d), d), mul(r1, r23));
    const f2 inv1 = make_float2(fminf(r1.x, 3.40282347e38f), fminf(r1.y, 3.40282347e38f));
    const f2 e2 = fmax0(sub(d, m2)), e3 = fmax0(sub(d, m3));
    const f2 cub = fma(mul(e2, e2), e2, mul(mul(e3, e3), e3));
    f2 num = fma(mul(mk(3.0f), d), sub(d, m1), mul(m1, m1));
    num = fma(make_float2(-cub.x, -cub.y), inv1, num);
    const f2 v24 = mul(num, r23);
    f2 v = sel(lt(d, m1), v1, v24);
    v = sel(le(m12, d), v5, v);
    return make_float2(d0.x > 0.0f ? 1.0f - v.x : v.x, d0.y > 0.0f ? 1.0f - v.y : v.y);
}

// Whole cells: two (n, V0) -> d0 in FP32 by the optimised SZ solution
// (METHOD = M_SZ_OPT, in L1 units), Kawano's SZ solution (M_SZ_ORIG, in L1
// units) or the analytic solution (M_ANALYTIC, in the unit normal's units);
// with ROUNDTRIP, also the forward volume of the returned d0 into *vrt; with
// COUNT, invalid cells are added to `bad`.
template <int METHOD, bool POLISH, bool ROUNDTRIP = false, bool COUNT = true>
__device__ __forceinline__ f2 offset_pair(f2 nx, f2 ny, f2 nz, f2 V0, int& bad,
                                          f2* vrt = nullptr) {
    const f2 ax = make_float2(fabsf(nx.x), fabsf(nx.y));
    const f2 ay = make_float2(fabsf(ny.x), fabsf(ny.y));
    const f2 az = make_float2(fabsf(nz.x), fabsf(nz.y));
    const f2 n1 = make_float2(fminf(fminf(ax.x, ay.x), az.x), fminf(fminf(ax.y, ay.y), az.y));
    const f2 n3 = make_float2(fmaxf(fmaxf(ax.x, ay.x), az.x), fmaxf(fmaxf(ax.y, ay.y), az.y));
    const f2 L = add(add(ax, ay), az);
    // V = min(V0, 1 - V0) equals the exact reduction of Eq. 5 on [0, 1], and is
    // negative or NaN exactly when V0 is outside [0, 1] or NaN
    const f2 W = sub(mk(1.0f), V0);
    const f2 V = make_float2(fminf(V0.x, W.x), fminf(V0.y, W.y));
    const bool okx = V.x >= 0.0f && L.x > 0.0f && L.x <= 3.0f;
    const bool oky = V.y >= 0.0f && L.y > 0.0f && L.y <= 3.0f;
    if (COUNT) bad += (int)!okx + (int)!oky;
    const f2 il = rcp(L);
    const f2 m1 = mul(n1, il), m3 = mul(n3, il);
    const f2 m2 = fmax0(sub(mk(1.0f), add(m1, m3)));
    f2 h;
    if (METHOD == M_SZ_OPT) {
        h = mul(L, sub(mk(0.5f), sz_opt<POLISH>(V, m1, m2, m3)));
    } else if (METHOD == M_SZ_ORIG) {
        h = mul(L, sub(mk(0.5f), sz_orig<POLISH>(V, m1, m2, m3)));
    } else {
        const f2 n2 = fmax0(sub(sub(L, n1), n3));
        const f2 d = analytic<POLISH>(V, n1, n2, n3);
        h = fma(mk(0.5f), L, make_float2(-d.x, -d.y));
    }
    f2 r = make_float2(copysignf(h.x, V0.x - 0.5f), copysignf(h.y, V0.y - 0.5f));
    if (!okx) r.x = __int_as_float(0x7fffffff);
    if (!oky) r.y = __int_as_float(0x7fffffff);
    if (ROUNDTRIP) {
        // NaN where d0 is NaN: invalid inputs, and Kawano's NaN cells (the
        // volume's clamp of d would otherwise turn a NaN offset into a number)
        f2 v = volume_reduced(r, il, m1, m2, m3);
        if (r.x != r.x) v.x = __int_as_float(0x7fffffff);
        if (r.y != r.y) v.y = __int_as_float(0x7fffffff);
        *vrt = v;
    }
    return r;
}

}  // namespace p2
}  // namespace plic
