// plic_solvers.cuh -- per-cell device functions of the PLIC hot path.
//
// Reduced space (Sec. 2.1, Eqs. 2-8): n1 <= n2 <= n3 are the sorted |n_k|,
// V = min(V0, 1 - V0) in [0, 1/2], d in [0, (n1+n2+n3)/2] is the offset from
// the cube corner, and d0 = sign(V0 - 1/2) ((n1+n2+n3)/2 - d).
//
// Solvers (reduced space, one function each, templated on float/double):
//   solve_analytic  -- the paper's inversion (Sec. 2.3, Eqs. 11-25): the
//                      closed forms of cases (5), (1), (2) by the tests of
//                      Eq. 24, then the real root f(x, y, a, b, c) of Eq. 11
//                      for case (3) or (4).
//   solve_sz_orig   -- Scardovelli-Zaleski as Kawano implements it (Sec. 2.4):
//                      L1-normalised n, its volume thresholds, the case-(3)/(4)
//                      cubic in Viete's trigonometric form.
//   solve_sz_opt    -- the paper's optimised SZ (Sec. 2.4): order 5 -> 2 -> 1,
//                      cases (3)/(4) merged into one arcsine/sine root.
//   solve_newton    -- Newton-Raphson for cases (1), (3), (4) (Sec. 2.5).
//   solve_nested    -- nested intervals for cases (3), (4) (Sec. 2.5).
// FAITHFUL selects the paper-literal behaviour of each (the printed front end
// of Eqs. 4-5, the printed iteration counts on Eq. 10 as printed, no clamp of
// the trigonometric arguments, the analytic solution's a-posteriori case
// order); the default adds clamps, convergence tests and cancellation-free
// forms where the printed ones lose digits.
//
// polish()          -- one Newton step on the reduced volume (Eq. 10) written
//                      without cancellation; used by PLIC_FP32_POLISHED.
// reduced_volume()  -- the forward problem (Eq. 10).
// (The cut polygon of the adjoints is in plic_polygon.cuh.)
#pragma once
#include "plic_df.cuh"
#include "plic_math.cuh"

namespace plic {

enum { M_ANALYTIC = 0, M_SZ_ORIG = 1, M_SZ_OPT = 2, M_NEWTON = 3, M_NESTED = 4 };

// ----------------------------------------------------------------------------
// Sec. 2.1: sort |n| (Eqs. 2-4) and reduce V (Eq. 5).
// Default: exact median and exact V = V0 or 1 - V0.  Faithful: the listing's
// n2 = |nx| + |ny| + |nz| - n1 - n3 and V = 1/2 - |V0 - 1/2|.
// ----------------------------------------------------------------------------
template <typename T, bool FAITHFUL>
__device__ __forceinline__ void reduce_normal(T nx, T ny, T nz, T& n1, T& n2, T& n3) {
    const T ax = fabs(nx), ay = fabs(ny), az = fabs(nz);
    n1 = fmin(fmin(ax, ay), az);
    n3 = fmax(fmax(ax, ay), az);
    if (FAITHFUL) n2 = (ax + ay + az) - n1 - n3;               // Eq. 4 as printed
    else n2 = fmax(fmin(ax, ay), fmin(fmax(ax, ay), az));
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T reduce_volume(T V0) {
    if (FAITHFUL) return T(0.5) - fabs(V0 - T(0.5));          // Eq. 5 as printed
    return V0 <= T(0.5) ? V0 : T(1) - V0;
}

// ----------------------------------------------------------------------------
// Eq. 10 without cancellation: g(d) = 6 n2 n3 (V(d) - V) and g'(d) for
// 0 < d < n1 + n2 (cases 1-4), with 1/n1 passed in (0 when n1 = 0, where only
// case (2) reaches this function and the 1/n1 terms vanish).
//   d <  n1 : g = d^3/n1 - 6 n2 n3 V
//   d >= n1 : g = 3 d (d - n1) + n1^2 - ((d-n2)_+^3 + (d-n3)_+^3)/n1 - 6 n2 n3 V
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void reduced_residual(T d, T rhs, T n1, T n2, T n3, T inv_n1,
                                                 T& g, T& gp) {
    if (d < n1) {
        g = d * d * d * inv_n1 - rhs;
        gp = T(3) * d * d * inv_n1;
    } else {
        const T e2 = fmax(d - n2, T(0)), e3 = fmax(d - n3, T(0));
        g = T(3) * d * (d - n1) + n1 * n1 - (e2 * e2 * e2 + e3 * e3 * e3) * inv_n1 - rhs;
        gp = T(6) * d - T(3) * n1 - T(3) * (e2 * e2 + e3 * e3) * inv_n1;
    }
}

// One Newton step d <- d - g/g' on Eq. 10, valid in every case: for
// d >= n1 + n2 (the case-(5) range) the volume is linear in d and the step
// lands on the exact case-(5) solution; otherwise g is the cancellation-free
// cubic of reduced_residual().  A trigonometric root that left its case
// (possible where a case is a sliver, e.g. case (3) for n1 << n2) is moved back
// by this step onto the neighbouring case's solution, which agrees with the
// true root up to O(n1^2).
template <typename T>
__device__ __forceinline__ T polish(T d, T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    const T n12 = n1 + n2;
    if (d >= n12) return n3 * V + T(0.5) * n12;
    if (!(d > T(0))) return d;
    const T inv_n1 = n1 > T(0) ? F::rcp_(n1) : T(0);
    T g, gp;
    reduced_residual<T>(d, T(6) * n2 * n3 * V, n1, n2, n3, inv_n1, g, gp);
    return gp > T(0) ? d - F::div_(g, gp) : d;
}

// ----------------------------------------------------------------------------
// Eqs. 24-25: the closed-form cases.  classify() applies the a-priori tests on
// V of Eq. 24 (case (2) with the factor 2 that its condition d2 <= n2 gives)
// and keeps the products that the closed forms reuse.  The tests of cases (1)
// and (2) exclude each other (n1^2 > 6 V n2 n3 against n1^2 <= 6 V n2 n3), so
// (1) is tested before (2).  After case (5) n2 > 0; a normal with n1 = 0
// always ends in case (2) or (5), so cases (1), (3), (4) have n1 > 0.
// ----------------------------------------------------------------------------
template <typename T> struct Cases {
    T n12;   // n1 + n2
    T h;     // V n3            (the case-(5) offset is h + n12/2)
    T w;     // 6 V n2 n3       (compared with n1^2 in Eq. 24)
    T q;     // n1^2
    int c;   // 5, 1 or 2; 0 when the offset lies in case (3) or (4)
};

template <typename T>
__device__ __forceinline__ Cases<T> classify(T V, T n1, T n2, T n3) {
    Cases<T> k;
    k.n12 = n1 + n2;
    k.h = n3 * V;
    k.w = T(6) * n2 * k.h;
    k.q = n1 * n1;
    if (k.n12 <= k.h + k.h) k.c = 5;
    else if (k.w < k.q) k.c = 1;
    else if (T(3) * n2 * (k.h + k.h + n1 - n2) <= k.q) k.c = 2;
    else k.c = 0;
    return k;
}

// The offset of case (5), (2) or (1) of Eq. 25:
//   d5 = V n3 + (n1 + n2)/2,  d2 = n1/2 + sqrt(2 V n2 n3 - n1^2/12),
//   d1 = (6 V n1 n2 n3)^(1/3).
template <typename T>
__device__ __forceinline__ T closed_form(const Cases<T>& k, T n1) {
    typedef Fm<T> F;
    if (k.c == 5) return k.h + T(0.5) * k.n12;
    if (k.c == 2) return T(0.5) * n1 + F::sqrt_(k.w * T(1.0 / 3.0) - k.q * T(1.0 / 12.0));
    return F::cbrt_(k.w * n1);
}

// Cases (3) or (4): the volume grows with d, so the offset lies in case (3)
// (d <= n3) exactly when the volume at d = n3 is at least V; for
// n3 >= n1 + n2 the offsets beyond n1 + n2 belong to case (5), so case (3) is
// the only one left.  The volume at n3 comes from the cancellation-free
// residual of Eq. 10 (n1 > 0 here).
template <typename T>
__device__ __forceinline__ bool offset_in_case3(const Cases<T>& k, T n1, T n2, T n3) {
    if (!(n3 < k.n12)) return true;
    T g, gp;
    reduced_residual<T>(n3, k.w, n1, n2, n3, Fm<T>::rcp_(n1), g, gp);
    return g >= T(0);
}

// ----------------------------------------------------------------------------
// Sec. 2.3: the analytic solution.  The real form of Eq. 11,
//   f(x, y, a, b, c) = c - 2 (a + b u) u^(-1/2) sin(pi/6 - theta/3),
// with u = (x^2 + y^2)^(1/3) and theta = atan2(y, x), is the root of the cubic
// of case (3) with the coefficients of Eqs. 12-16 and of case (4) with those
// of Eqs. 17-22 (both need |n| = 1).  y enters only through y^2 >= 0 (its
// rounding may make it slightly negative: clamped at 0).
// Default: the case is decided first (offset_in_case3), and only that case's
// root is formed.  FAITHFUL: the paper's a-posteriori order -- d3 first, kept
// if d3 <= n3, else d4.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T eq11_root(T x, T y2, T a, T b, T c) {
    typedef Fm<T> F;
    y2 = fmax(y2, T(0));
    const T u3 = x * x + y2;
    const T u = F::cbrt_(u3);
    const T ru = F::rsqrt_(u);
    const T theta = F::polar_angle_(x, F::sqrt_(y2));
    return c - T(2) * (a * ru + b * (u * ru)) * F::sin_pi6_(Kc<T>::pi_6 - Kc<T>::third * theta);
}

template <typename T>
__device__ __forceinline__ T analytic_case3(T V, T n1, T n2, T n3, T n12) {
    const T p = n1 * n2;
    const T x = T(81) * p * (n12 - T(2) * V * n3);
    return eq11_root<T>(x, T(23328) * p * p * p - x * x, Kc<T>::cbrt54 * p, Kc<T>::inv_cbrt432, n12);
}

template <typename T>
__device__ __forceinline__ T analytic_case4(T V, T n1, T n2, T n3) {
    const T L = n1 + n2 + n3;
    const T t = T(9) * L * L - T(18);
    const T x = T(324) * n1 * n2 * n3 * (T(1) - T(2) * V);
    return eq11_root<T>(x, T(4) * t * t * t - x * x, Kc<T>::inv_cbrt864 * t, Kc<T>::inv_cbrt3456,
                        T(0.5) * L);
}

// Every solver comes in two parts (struct Solver below): easy() settles the
// closed-form cases and returns false for the cells that need the heavy part,
// hard() (the trigonometric root or the iterations); solve_<method> is one
// after the other.  The work-compacted kernel runs easy() on every cell and
// hard() only on the cells that need it, packed densely over the lanes.
template <typename T, bool FAITHFUL>
__device__ __forceinline__ bool analytic_easy(T V, T n1, T n2, T n3, T& d) {
    const Cases<T> k = classify<T>(V, n1, n2, n3);
    if (k.c == 0) return false;
    d = closed_form<T>(k, n1);
    return true;
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T analytic_hard(T V, T n1, T n2, T n3) {
    const Cases<T> k = classify<T>(V, n1, n2, n3);
    if (FAITHFUL) {
        const T d3 = analytic_case3<T>(V, n1, n2, n3, k.n12);
        return d3 <= n3 ? d3 : analytic_case4<T>(V, n1, n2, n3);
    }
    return offset_in_case3<T>(k, n1, n2, n3) ? analytic_case3<T>(V, n1, n2, n3, k.n12)
                                             : analytic_case4<T>(V, n1, n2, n3);
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_analytic(T V, T n1, T n2, T n3) {
    T d;
    return analytic_easy<T, FAITHFUL>(V, n1, n2, n3, d) ? d : analytic_hard<T, FAITHFUL>(V, n1, n2, n3);
}

// ----------------------------------------------------------------------------
// Sec. 2.4: the Scardovelli-Zaleski solution in the form of Kawano's
// implementation, which the paper compares.  Inputs: the L1-normalised
// m1 <= m2 <= m3 (m1 + m2 + m3 = 1) and the reduced volume w; the result is
// the offset in L1 units.  Its cases are told apart by volumes: case (1) ends
// at Vb1 = m1^2 / (6 m2 m3) (that implementation adds 1e-25 to the
// denominator), case (2) at Vb2 = Vb1 + (m2 - m1)/(2 m3); case (3) ends at the
// volume of the plane through the vertex m3 when m3 < m1 + m2 (case (4)
// follows), else at that of the plane d = m1 + m2 (case (5) follows).  Cases
// (3)/(4) are the monic cubic alpha^3 + a2 alpha^2 + a1 alpha + a0 = 0 of
// Eq. 10, solved in Viete's trigonometric form: with alpha = t - a2/3 it
// becomes t^3 + p t + q = 0, and the root is
//   alpha = -a2/3 + 2 s cos((acos(r) + 4 pi)/3),  s^2 = -p/3,  r = -q/(2 s^3).
// Default: s^2 and -q/2 multiplied out with m1 + m2 + m3 = 1 (case (3):
// 2 m1 m2 and 1.5 m1 m2 (m1 + m2 - 2 m3 w); case (4):
// (m1 (2 (m2 + m3) - m1) - (m3 - m2)^2)/4 and 0.75 m1 m2 m3 (1 - 2 w)), since
// the general forms subtract O(1) terms to reach O(s^3) and lose every digit
// when m1 << m2; r clamped to [-1, 1].  FAITHFUL: p and q from a2, a1, a0 and
// no clamp.
// That implementation treats a zero case-(5) offset as "no case found yet"
// and solves the case-(4) cubic instead.  For m = (0, 0, 1) and w = 0 (V0 in
// {0, 1}) that cubic has s^2 = -1/4 and the result is NaN, as the paper
// reports; this reproduces it.
// ----------------------------------------------------------------------------
template <typename T, bool FAITHFUL>
__device__ __forceinline__ bool sz_orig_easy(T w, T m1, T m2, T m3, T& a) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T m12 = m1 + m2;
    const T vb1 = F::div_(m1 * m1, T(6) * m2 * m3 + T(1e-25));
    if (w < vb1) {                                                                // (1)
        a = F::cbrt_(T(6) * m1 * m2 * m3 * w);
        return true;
    }
    if (w < vb1 + F::div_(T(0.5) * (m2 - m1), m3)) {                               // (2)
        a = T(0.5) * m1 + F::sqrt_(T(2) * m2 * m3 * w - K::twelfth * m1 * m1);
        return true;
    }
    if (!(m3 < m12) && !(w < F::div_(T(0.5) * m12, m3))) {
        a = m3 * w + T(0.5) * m12;                                                 // (5)
        return a != T(0);
    }
    return false;
}

// Cases (3)/(4) (and the zero case-(5) offset that implementation sends here).
template <typename T, bool FAITHFUL>
__device__ __forceinline__ T sz_orig_hard(T w, T m1, T m2, T m3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T m12 = m1 + m2, e3 = m1 * m2 * m3;
    const bool tall = !(m3 < m12);
    const T vb3 = tall ? F::div_(T(0.5) * m12, m3)
                       : F::div_(cb(m3) - cb(m3 - m1) - cb(m3 - m2), T(6) * e3);
    const bool case3 = w < vb3;
    T s2, mq2, shift;                     // s^2, -q/2, -a2/3
    if (FAITHFUL) {
        const T w6 = T(6) * e3 * w;
        const T a2 = case3 ? T(-3) * m12 : T(-1.5);
        const T a1 = case3 ? T(3) * (m1 * m1 + m2 * m2) : T(1.5) * (m1 * m1 + m2 * m2 + m3 * m3);
        const T a0 = case3 ? w6 - cb(m1) - cb(m2) : T(0.5) * (w6 - cb(m1) - cb(m2) - cb(m3));
        const T p = a1 - K::third * a2 * a2;
        const T q = T(2.0 / 27.0) * cb(a2) - K::third * a1 * a2 + a0;
        s2 = -K::third * p;
        mq2 = T(-0.5) * q;
        shift = -K::third * a2;
    } else {
        s2 = case3 ? T(2) * m1 * m2 : T(0.25) * (m1 * (T(2) * (m2 + m3) - m1) - sq(m3 - m2));
        mq2 = case3 ? T(1.5) * m1 * m2 * (m12 - T(2) * m3 * w) : T(0.75) * e3 * (T(1) - T(2) * w);
        shift = case3 ? m12 : T(0.5);
    }
    const T s = F::sqrt_(s2);
    T r = F::div_(mq2, s2 * s);
    if (!FAITHFUL) r = fmin(fmax(r, T(-1)), T(1));
    // cos((acos r + 4 pi)/3) = sin(acos(r)/3 - pi/6), an angle in [-pi/6, pi/6]
    // (FP64; FP32 keeps the cosine of the angle as written)
    if constexpr (sizeof(T) == 8) return shift + T(2) * s * F::sin_pi6_(K::third * F::acos_(r) - K::pi_6);
    return shift + T(2) * s * F::cos_(K::third * (F::acos_(r) + K::four_pi));
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_sz_orig(T w, T m1, T m2, T m3) {
    T a;
    return sz_orig_easy<T, FAITHFUL>(w, m1, m2, m3, a) ? a : sz_orig_hard<T, FAITHFUL>(w, m1, m2, m3);
}

// ----------------------------------------------------------------------------
// Sec. 2.4: the paper's optimised SZ solution: cases tested in the order
// (5), (2), (1), cases (3) and (4) merged into one arcsine/sine root through
// their coefficients (L1-normalised inputs, the reduced volume V; the result
// in L1 units).  Here
//  - the case tests are multiplied out so that no division is needed
//    (Vb1 <= n3 V  <=>  n1^2 <= 6 n2 n3 V;  the case-(3)/(4) boundary
//    6 n1 n2 n3 V < n3^3 - (n3 - n1)^3 - (n3 - n2)^3, written expanded),
//  - the arcsine argument is written without cancellation:
//    case (3): 1.5 n1 n2 (n1 + n2 - 2 n3 V) / (2 n1 n2)^(3/2),
//    case (4): 0.75 n1 n2 n3 (1 - 2V) / t^3, t^2 = (n1 (2(n2+n3) - n1) - (n3-n2)^2)/4
//    (exact for n1 + n2 + n3 = 1), clamped to [-1, 1] unless FAITHFUL.
// In FP32 every case is evaluated and the result selected (no divergent
// branches; the warp pays for cases (1), (2) and (5) a few instructions each).
// In FP64 the cases branch (the FP64 pipe is the bottleneck there).
// ----------------------------------------------------------------------------
template <typename T, bool CLAMP = true>
__device__ __forceinline__ T solve_sz_opt_default(T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n12 = n1 + n2, n3V = n3 * V;
    const T V6n2n3 = T(6) * n2 * n3V, sqn1 = n1 * n1;
    const bool c5 = n12 <= T(2) * n3V;
    const bool c1 = V6n2n3 < sqn1;
    const bool c2 = !c1 && T(3) * n2 * (T(2) * n3V + n1 - n2) < sqn1;
    const T n1n2 = n1 * n2;
    const T num3 = sq(n3) * (T(3) * n12 - n3) + sqn1 * (n1 - T(3) * n3) + sq(n2) * (n2 - T(3) * n3);
    const bool c3 = !(n3 < n12) || V6n2n3 * n1 < num3;
    if (sizeof(T) == 8) {
        if (c5) return n3V + T(0.5) * n12;
        if (c2) return T(0.5) * (n1 + F::sqrt_(T(8) * n2 * n3V - K::third * sqn1));
        if (c1) return F::cbrt_(V6n2n3 * n1);
    }
    const T q = c3 ? T(1.5) * n1n2 * (n12 - T(2) * n3V) : T(0.75) * n1n2 * n3 * (T(1) - T(2) * V);
    const T t2 = c3 ? T(2) * n1n2 : T(0.25) * (n1 * (T(2) * (n2 + n3) - n1) - sq(n3 - n2));
    const T c = c3 ? n12 : T(0.5);
    const T rt = F::rsqrt_(t2);
    const T t = t2 * rt;
    T arg = q * (rt * rt * rt);
    if (CLAMP) arg = fmin(fmax(arg, T(-1)), T(1));
    const T d34 = c - T(2) * t * F::sin_pi6_(K::third * F::asin_(arg));
    if (sizeof(T) == 8) return d34;
    const T d5 = n3V + T(0.5) * n12;
    const T d2 = T(0.5) * (n1 + F::sqrt_(T(8) * n2 * n3V - K::third * sqn1));
    const T d1 = F::cbrt_(V6n2n3 * n1);
    return c5 ? d5 : (c2 ? d2 : (c1 ? d1 : d34));
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_sz_opt(T V, T n1, T n2, T n3) {
    return solve_sz_opt_default<T, !FAITHFUL>(V, n1, n2, n3);
}

// The two parts of the optimised SZ solution (the FP64 path branches on the
// cases; the FP32 path selects and has its own paired kernel).
template <typename T, bool FAITHFUL>
__device__ __forceinline__ bool sz_opt_easy(T V, T n1, T n2, T n3, T& d) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n12 = n1 + n2, n3V = n3 * V;
    const T V6n2n3 = T(6) * n2 * n3V, sqn1 = n1 * n1;
    if (n12 <= T(2) * n3V) { d = n3V + T(0.5) * n12; return true; }
    if (V6n2n3 < sqn1) { d = F::cbrt_(V6n2n3 * n1); return true; }
    if (T(3) * n2 * (T(2) * n3V + n1 - n2) < sqn1) {
        d = T(0.5) * (n1 + F::sqrt_(T(8) * n2 * n3V - K::third * sqn1));
        return true;
    }
    return false;
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T sz_opt_hard(T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n12 = n1 + n2, n3V = n3 * V, n1n2 = n1 * n2;
    const T num3 = sq(n3) * (T(3) * n12 - n3) + n1 * n1 * (n1 - T(3) * n3) + sq(n2) * (n2 - T(3) * n3);
    const bool c3 = !(n3 < n12) || T(6) * n2 * n3V * n1 < num3;
    const T q = c3 ? T(1.5) * n1n2 * (n12 - T(2) * n3V) : T(0.75) * n1n2 * n3 * (T(1) - T(2) * V);
    const T t2 = c3 ? T(2) * n1n2 : T(0.25) * (n1 * (T(2) * (n2 + n3) - n1) - sq(n3 - n2));
    const T c = c3 ? n12 : T(0.5);
    const T rt = F::rsqrt_(t2);
    T arg = q * (rt * rt * rt);
    if (!FAITHFUL) arg = fmin(fmax(arg, T(-1)), T(1));
    return c - T(2) * (t2 * rt) * F::sin_pi6_(K::third * F::asin_(arg));
}

// ----------------------------------------------------------------------------
// Sec. 2.5: the iterative solvers.  Both take the closed forms for cases (5)
// and (2), then iterate on the volume of Eq. 10 inside the bracket of a case:
// [0, n1] for case (1) (Newton only; nested intervals use the cube root),
// [n2, n1 + n2] for case (3) and, in the paper's order, [n3, L/2] for case
// (4) when the case-(3) result passes n3.  The default forms iterate on the
// residual of reduced_residual(), which is Eq. 10 for every d < n1 + n2 (its
// (d - n3)_+ term covers case (4)); since the case-(4) range [n3, L/2] lies
// inside [n2, n1 + n2] (L/2 < n1 + n2 when n3 < n1 + n2), one bracket
// [n2, n1 + n2] holds the offset of both cases and is iterated once.  The
// bracket is chosen by selects, so all lanes of a warp run one loop.
//
// The paper-literal forms (FAITHFUL) run on Eq. 10 as printed: with k
// corners cut off (none in case (1), two in case (3), three in case (4)),
//   P(d) = d^3 - sum_{j <= k} (d - n_j)^3 = 6 n1 n2 n3 V,
// plain Newton steps from the middle of the bracket (7 in case (1), 4 in
// cases (3)/(4)), and k + 1 halvings for nested intervals, k the binary
// exponent of the bracket width times 2^24 (2^53 in FP64; k at least 0): the
// counts the paper uses, with no convergence test.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void eq10_printed(T d, int corners, T n1, T n2, T n3, T& P, T& dP) {
    P = d * d * d;
    dP = T(3) * d * d;
    const T nk[3] = {n1, n2, n3};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < corners) {
            const T e = d - nk[j];
            P -= e * e * e;
            dP -= T(3) * e * e;
        }
    }
}

template <typename T>
__device__ __forceinline__ T newton_printed(T lo, T hi, int corners, int steps, T rhs6, T n1, T n2,
                                            T n3) {
    T d = T(0.5) * (lo + hi);
    for (int i = 0; i < steps; ++i) {
        T P, dP;
        eq10_printed<T>(d, corners, n1, n2, n3, P, dP);
        d -= (P - rhs6) / dP;
    }
    return d;
}

template <typename T>
__device__ __forceinline__ T halve_printed(T lo, T hi, int corners, T rhs6, T n1, T n2, T n3) {
    int k = Fm<T>::ilogb_(hi - lo) + (sizeof(T) == 4 ? 24 : 53);
    k = k < 0 ? 0 : (k > 1100 ? 1100 : k);
    T d = T(0.5) * (lo + hi);
    for (int i = 0; i <= k; ++i) {
        T P, dP;
        eq10_printed<T>(d, corners, n1, n2, n3, P, dP);
        if (P < rhs6) lo = d; else hi = d;
        d = T(0.5) * (lo + hi);
    }
    return d;
}

// Default Newton: the cancellation-free residual of reduced_residual(), steps
// until |dd| <= 4 ulp (at most 16).  A step that leaves the bracket is clamped
// to the end it crossed (the root can sit exactly at an end, e.g. d = L/2 for
// V0 = 1/2); crossing the same end again bisects.  From the bracket midpoint
// this converges in at most 7 steps on the paper-shaped inputs.
template <typename T>
__device__ __forceinline__ T newton_bracketed(T d, T lo, T hi, T rhs, T n1, T n2, T n3,
                                              T inv_n1) {
    for (int it = 0; it < 16; ++it) {
        T g, gp;
        reduced_residual<T>(d, rhs, n1, n2, n3, inv_n1, g, gp);
        if (g < T(0)) lo = d; else hi = d;
        T dn = gp > T(0) ? d - Fm<T>::div_(g, gp) : T(0.5) * (lo + hi);
        if (dn > hi) dn = d == hi ? T(0.5) * (lo + hi) : hi;
        if (dn < lo) dn = d == lo ? T(0.5) * (lo + hi) : lo;
        const T step = fabs(dn - d);
        d = dn;
        if (step <= T(4) * Fm<T>::eps() * d) break;
    }
    return d;
}

// Default nested intervals: halve on the sign of the cancellation-free
// residual until the two ends are adjacent floating-point numbers (at most
// 128 halvings).
template <typename T>
__device__ __forceinline__ T halve_to_adjacent(T lo, T hi, T rhs, T n1, T n2, T n3, T inv_n1) {
    T d = T(0.5) * (lo + hi);
    for (int i = 0; i < 128; ++i) {
        T g, gp;
        reduced_residual<T>(d, rhs, n1, n2, n3, inv_n1, g, gp);
        if (g < T(0)) lo = d; else hi = d;
        const T m = T(0.5) * (lo + hi);
        if (m <= lo || m >= hi) break;
        d = m;
    }
    return d;
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ bool newton_easy(T V, T n1, T n2, T n3, T& d) {
    const Cases<T> k = classify<T>(V, n1, n2, n3);
    if (k.c != 5 && k.c != 2) return false;
    d = closed_form<T>(k, n1);
    return true;
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T newton_hard(T V, T n1, T n2, T n3) {
    const Cases<T> k = classify<T>(V, n1, n2, n3);
    const T half = T(0.5) * (k.n12 + n3);                 // L/2
    if (FAITHFUL) {
        const T rhs6 = k.w * n1;                           // 6 V n1 n2 n3
        if (k.c == 1) return newton_printed<T>(T(0), n1, 0, 7, rhs6, n1, n2, n3);
        const T d = newton_printed<T>(n2, k.n12, 2, 4, rhs6, n1, n2, n3);
        return d <= n3 ? d : newton_printed<T>(n3, half, 3, 4, rhs6, n1, n2, n3);
    }
    const T inv_n1 = T(1) / n1;
    // case (1): [0, n1], starting within a factor 2^(2/3) of the root
    // (d1^3 = X) from the binary exponent of X = 6 V n1 n2 n3; cases (3)/(4):
    // [n2, n1 + n2] from its middle
    const bool c1 = k.c == 1;
    const T X = k.w * n1;
    if (c1 && !(X > T(0))) return T(0);
    const T d1 = fmin(ldexp(T(1), Fm<T>::ilogb_(c1 ? X : T(1)) / 3), n1);
    const T lo = c1 ? T(0) : n2, hi = c1 ? n1 : k.n12;
    const T d0 = c1 ? d1 : T(0.5) * (n2 + k.n12);
    return newton_bracketed<T>(d0, lo, hi, k.w, n1, n2, n3, inv_n1);
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_newton(T V, T n1, T n2, T n3) {
    T d;
    return newton_easy<T, FAITHFUL>(V, n1, n2, n3, d) ? d : newton_hard<T, FAITHFUL>(V, n1, n2, n3);
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ bool nested_easy(T V, T n1, T n2, T n3, T& d) {
    return analytic_easy<T, FAITHFUL>(V, n1, n2, n3, d);
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T nested_hard(T V, T n1, T n2, T n3) {
    const Cases<T> k = classify<T>(V, n1, n2, n3);
    const T half = T(0.5) * (k.n12 + n3);
    if (FAITHFUL) {
        const T rhs6 = k.w * n1;
        const T d = halve_printed<T>(n2, k.n12, 2, rhs6, n1, n2, n3);
        return d <= n3 ? d : halve_printed<T>(n3, half, 3, rhs6, n1, n2, n3);
    }
    const T inv_n1 = T(1) / n1;
    return halve_to_adjacent<T>(n2, k.n12, k.w, n1, n2, n3, inv_n1);
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_nested(T V, T n1, T n2, T n3) {
    T d;
    return nested_easy<T, FAITHFUL>(V, n1, n2, n3, d) ? d : nested_hard<T, FAITHFUL>(V, n1, n2, n3);
}

// The split parts by method, for the work-compacted kernel (reduced inputs:
// the L1-normalised m for the SZ solutions, the unit-normal n otherwise).
template <int METHOD, typename T, bool FAITHFUL> struct Solver;
template <typename T, bool F> struct Solver<M_ANALYTIC, T, F> {
    static __device__ __forceinline__ bool easy(T V, T a, T b, T c, T& d) { return analytic_easy<T, F>(V, a, b, c, d); }
    static __device__ __forceinline__ T hard(T V, T a, T b, T c) { return analytic_hard<T, F>(V, a, b, c); }
};
template <typename T, bool F> struct Solver<M_SZ_ORIG, T, F> {
    static __device__ __forceinline__ bool easy(T V, T a, T b, T c, T& d) { return sz_orig_easy<T, F>(V, a, b, c, d); }
    static __device__ __forceinline__ T hard(T V, T a, T b, T c) { return sz_orig_hard<T, F>(V, a, b, c); }
};
template <typename T, bool F> struct Solver<M_SZ_OPT, T, F> {
    static __device__ __forceinline__ bool easy(T V, T a, T b, T c, T& d) { return sz_opt_easy<T, F>(V, a, b, c, d); }
    static __device__ __forceinline__ T hard(T V, T a, T b, T c) { return sz_opt_hard<T, F>(V, a, b, c); }
};
template <typename T, bool F> struct Solver<M_NEWTON, T, F> {
    static __device__ __forceinline__ bool easy(T V, T a, T b, T c, T& d) { return newton_easy<T, F>(V, a, b, c, d); }
    static __device__ __forceinline__ T hard(T V, T a, T b, T c) { return newton_hard<T, F>(V, a, b, c); }
};
template <typename T, bool F> struct Solver<M_NESTED, T, F> {
    static __device__ __forceinline__ bool easy(T V, T a, T b, T c, T& d) { return nested_easy<T, F>(V, a, b, c, d); }
    static __device__ __forceinline__ T hard(T V, T a, T b, T c) { return nested_hard<T, F>(V, a, b, c); }
};

// ----------------------------------------------------------------------------
// Whole cell: d0(V0, n) (Sec. 2, Eq. 1) for one method and precision.
// Invalid input (NaN, V0 outside [0,1], n = 0 or non-finite) gives NaN and
// sets `bad`.
// ----------------------------------------------------------------------------
template <int METHOD, typename T, bool POLISH, bool FAITHFUL>
__device__ __forceinline__ T offset_cell(T nx, T ny, T nz, T V0, int& bad) {
    T n1, n2, n3;
    reduce_normal<T, FAITHFUL>(nx, ny, nz, n1, n2, n3);
    const T L = fabs(nx) + fabs(ny) + fabs(nz);
    const bool ok = (V0 >= T(0)) && (V0 <= T(1)) && (L > T(0)) && (L <= T(3));
    if (!ok) {
        bad += 1;
        return T(NAN);
    }
    const T V = reduce_volume<T, FAITHFUL>(V0);
    if (METHOD == M_SZ_ORIG || METHOD == M_SZ_OPT) {
        // L1 normalisation (Sec. 2.4); the solvers return the offset in L1 units
        const T l = L;
        const T il = FAITHFUL ? T(1) / l : Fm<T>::rcp_(l);
        const T m1 = n1 * il, m3 = n3 * il;
        const T m2 = Fm<T>::fdim_(T(1), m1 + m3);
        T a = METHOD == M_SZ_ORIG ? solve_sz_orig<T, FAITHFUL>(V, m1, m2, m3)
                                  : solve_sz_opt<T, FAITHFUL>(V, m1, m2, m3);
        if (POLISH) a = polish<T>(a, V, m1, m2, m3);
        return l * copysign(T(0.5) - a, V0 - T(0.5));
    } else {
        T d = METHOD == M_ANALYTIC ? solve_analytic<T, FAITHFUL>(V, n1, n2, n3)
            : METHOD == M_NEWTON   ? solve_newton<T, FAITHFUL>(V, n1, n2, n3)
                                   : solve_nested<T, FAITHFUL>(V, n1, n2, n3);
        if (POLISH) d = polish<T>(d, V, n1, n2, n3);
        return copysign(T(0.5) * (n1 + n2 + n3) - d, V0 - T(0.5));
    }
}

// ----------------------------------------------------------------------------
// FP64 result from an FP32 solve, without the FP64 pipe (PLIC_FP64_REFINED).
// The doubles are split into double-floats (hi + lo, 48 significant bits) by
// integer operations; the symmetry reduction (Eqs. 2-8) sorts |n| on the bit
// patterns and forms V = min(V0, 1 - V0) from the bits (1 - V0 as an exact
// integer difference), so V keeps its relative precision; the method's FP32 solver runs on the reduced problem's
// leading floats; two Newton steps on Eq. 10 in double-float (the residual in
// double-float, the derivative's reciprocal in FP32) finish it, and the result
// goes back to a double with one FP64 add.  The FP32 root is within ~1e-7 of
// the root, the first step lands at ~1e-14, the second at the double-float
// resolution (~1e-15).  The residual is multiplied through by n1, so the steps
// divide by nothing but the FP32 derivative; n1 < 2^-60 counts as 0 there
// (its effect on d0 is below 1e-18).  V0 below 2^-126 counts as 0: d0 then
// differs from the exact offset by less than 3e-13.
// ----------------------------------------------------------------------------
template <int METHOD>
__device__ __forceinline__ double offset_cell_refined(double nx, double ny, double nz, double V0,
                                                      int& bad) {
    const uint64_t SIGN = 0x8000000000000000ull;
    // |n| sorted on the bits (the order of non-negative doubles is that of their
    // bit patterns; a NaN sorts last and makes L NaN)
    const uint64_t ux = (uint64_t)__double_as_longlong(nx) & ~SIGN;
    const uint64_t uy = (uint64_t)__double_as_longlong(ny) & ~SIGN;
    const uint64_t uz = (uint64_t)__double_as_longlong(nz) & ~SIGN;
    const uint64_t b1 = ux < uy ? (ux < uz ? ux : uz) : (uy < uz ? uy : uz);
    const uint64_t b3 = ux > uy ? (ux > uz ? ux : uz) : (uy > uz ? uy : uz);
    const uint64_t b2 = ux ^ uy ^ uz ^ b1 ^ b3;
    const df n1 = d2df(__longlong_as_double((long long)b1));
    const df n2 = d2df(__longlong_as_double((long long)b2));
    const df n3 = d2df(__longlong_as_double((long long)b3));
    const df L = df_add(df_add(n1, n2), n3);
    // 0 <= V0 <= 1 on the bits (-0 accepted, NaN refused)
    const uint64_t v = (uint64_t)__double_as_longlong(V0), va = v & ~SIGN;
    const bool vneg = (v >> 63) != 0 && va != 0;
    const bool ok = !vneg && va <= 0x3FF0000000000000ull && L.hi > 0.0f && L.hi <= 3.0f;
    if (!ok) {
        bad += 1;
        return __longlong_as_double(0x7FF8000000000000ll);
    }
    const bool upper = va > 0x3FE0000000000000ull;             // V0 > 1/2
    const bool lower = va < 0x3FE0000000000000ull;             // V0 < 1/2
    // V = 1 - V0 exactly on the bits for V0 > 1/2 (V0 = M 2^-53 with
    // M = 2^52 + mantissa, or 2^53 for V0 = 1): converting V0 to a
    // double-float first would cost the low bits that 1 - V0 keeps
    df V;
    if (upper) {
        const uint64_t M = (va >> 52) >= 1023ull ? (1ull << 53)
                                                  : ((1ull << 52) | (va & 0xFFFFFFFFFFFFFull));
        V = df_from_u64_2m53((1ull << 53) - M);
    } else {
        V = d2df(__longlong_as_double((long long)va));
    }
    const float Vf = V.hi;
    // FP32 solve of the reduced problem, as an offset d from the corner
    df d;
    if (METHOD == M_SZ_ORIG || METHOD == M_SZ_OPT) {
        const float il = Fm<float>::rcp_(L.hi);
        const float m1 = n1.hi * il, m3 = n3.hi * il;
        const float m2 = Fm<float>::fdim_(1.0f, m1 + m3);
        float a = METHOD == M_SZ_ORIG ? solve_sz_orig<float, false>(Vf, m1, m2, m3)
                                      : solve_sz_opt<float, false>(Vf, m1, m2, m3);
        a = polish<float>(a, Vf, m1, m2, m3);
        if (a != a) return __longlong_as_double(0x7FF8000000000000ll);  // Kawano's NaN
        d = df_mul_f(L, a);
    } else {
        float e = METHOD == M_ANALYTIC ? solve_analytic<float, false>(Vf, n1.hi, n2.hi, n3.hi)
                : METHOD == M_NEWTON   ? solve_newton<float, false>(Vf, n1.hi, n2.hi, n3.hi)
                                       : solve_nested<float, false>(Vf, n1.hi, n2.hi, n3.hi);
        e = polish<float>(e, Vf, n1.hi, n2.hi, n3.hi);
        if (e != e) return __longlong_as_double(0x7FF8000000000000ll);
        d = df_make(e);
    }
    const df zero = df_make(0.0f);
    const df h = df_scale(L, 0.5f);
    d = df_clamp(d, zero, h);
    // Newton steps on Eq. 10 multiplied by n1 (n1 g and n1 g'), in double-float
    const bool n1z = n1.hi < 8.67361738e-19f;                  // 2^-60
    const df n12 = df_add(n1, n2);
    const df rhs = df_mul_f(df_mul(df_mul(n2, n3), V), 6.0f); // 6 n2 n3 V
    const df R1 = n1z ? zero : df_mul(n1, rhs);                // 6 n1 n2 n3 V
    const df d5 = df_add(df_mul(n3, V), df_scale(n12, 0.5f)); // case (5), linear, exact
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (!df_lt(d, n12)) {
            d = d5;
        } else if (d.hi > 0.0f) {
            df g;
            float gp;
            if (n1z) {                                          // n1 = 0: case (2) only
                g = df_sub(df_mul_f(df_mul(d, d), 3.0f), rhs);
                gp = 6.0f * d.hi;
            } else if (df_lt(d, n1)) {                          // case (1)
                g = df_sub(df_mul(df_mul(d, d), d), R1);
                gp = 3.0f * d.hi * d.hi;
            } else {                                            // cases (2)-(4)
                const df e2 = df_max0(df_sub(d, n2)), e3 = df_max0(df_sub(d, n3));
                const df cub = df_add(df_mul(df_mul(e2, e2), e2), df_mul(df_mul(e3, e3), e3));
                const df t = df_add(df_mul_f(df_mul(d, df_sub(d, n1)), 3.0f), df_mul(n1, n1));
                g = df_sub(df_sub(df_mul(n1, t), cub), R1);
                gp = n1.hi * fmaf(6.0f, d.hi, -3.0f * n1.hi) -
                     3.0f * (e2.hi * e2.hi + e3.hi * e3.hi);
            }
            if (gp > 0.0f) d = df_sub(d, df_mul_f(g, Fm<float>::rcp_(gp)));
        }
        d = df_clamp(d, zero, h);
    }
    const double r = df2d(df_sub(h, d));
    return lower ? -r : r;
}

// ----------------------------------------------------------------------------
// Forward problem, Eq. 10 (cases written without cancellation), for
// 0 <= d <= L/2 with n1 <= n2 <= n3, n3 > 0.  Case (5) requires
// n1 + n2 <= d <= n3 (the form min(n1+n2, n3) <= d of Eq. 10 would also admit
// d = n3 when n3 < n1 + n2, where the case-(5) formula does not hold).
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T reduced_volume(T d, T n1, T n2, T n3) {
    const T n12 = n1 + n2;
    if (!(d > T(0))) return T(0);
    if (d >= n12) return (d - T(0.5) * n12) / n3;                                // case (5)
    if (d < n1) return d * d * d / (T(6) * n1 * n2 * n3);                         // case (1)
    T num = T(3) * d * (d - n1) + n1 * n1;                                        // case (2)
    if (d > n2) {                                                                // cases (3), (4)
        const T e2 = d - n2, e3 = fmax(d - n3, T(0));
        num -= (e2 * e2 * e2 + e3 * e3 * e3) / n1;
    }
    return num / (T(6) * n2 * n3);
}

template <typename T>
__device__ __forceinline__ T volume_cell(T nx, T ny, T nz, T d0) {
    T n1, n2, n3;
    reduce_normal<T, false>(nx, ny, nz, n1, n2, n3);
    const T L = n1 + n2 + n3;
    if (!(L > T(0)) || !(L <= T(3)) || d0 != d0) return T(NAN);
    const T h = T(0.5) * L, ad = fabs(d0);
    if (ad >= h) return d0 > T(0) ? T(1) : T(0);
    const T V = reduced_volume<T>(h - ad, n1, n2, n3);
    return d0 > T(0) ? T(1) - V : V;
}

}  // namespace plic
