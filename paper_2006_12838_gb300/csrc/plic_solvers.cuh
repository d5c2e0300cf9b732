// plic_solvers.cuh -- per-cell device functions of the PLIC hot path.
//
// Reduced space (Sec. 2.1, Eqs. 2-8): n1 <= n2 <= n3 are the sorted |n_k|,
// V = min(V0, 1 - V0) in [0, 1/2], d in [0, (n1+n2+n3)/2] is the offset from
// the cube corner, and d0 = sign(V0 - 1/2) ((n1+n2+n3)/2 - d).
//
// Solvers (reduced space, one function each, templated on float/double):
//   solve_analytic  -- the paper's inversion (Sec. 2.3, Eqs. 11-25): a-priori
//                      tests for cases (5), (2), (1) (Eq. 24, with the factor 2
//                      of the case-(2) test that the derivation d2 <= n2 gives),
//                      then the trigonometric root f(x, y, a, b, c) of Eq. 11
//                      for case (3) and, if d3 > n3, for case (4).
//   solve_sz_orig   -- Scardovelli-Zaleski as Kawano implements it (Sec. 2.4):
//                      L1-normalised n, thresholds v1, v3, the cubic solved by
//                      the cosine form.
//   solve_sz_opt    -- the paper's optimised SZ (Sec. 2.4): order 5 -> 2 -> 1,
//                      cases (3)/(4) merged through the coefficients (a, b, c)
//                      and the sine/arcsine form.
//   solve_newton    -- Newton-Raphson for cases (1), (3), (4) (Sec. 2.5).
//   solve_nested    -- nested intervals for cases (3), (4) (Sec. 2.5).
// FAITHFUL selects the paper-literal variant of each (printed iteration counts,
// no argument clamps); the default adds clamps, convergence tests and a
// cancellation-free cubic where the printed form loses digits.
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
    if (FAITHFUL) n2 = ax - n1 + ay + az - n3;
    else n2 = fmax(fmin(ax, ay), fmin(fmax(ax, ay), az));
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T reduce_volume(T V0) {
    if (FAITHFUL) return T(0.5) - fabs(V0 - T(0.5));
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
// Sec. 2.3: the analytic solution (Eq. 25 with the a-priori tests of Eq. 24).
// ----------------------------------------------------------------------------
template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_analytic(T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n12 = n1 + n2, n3V = n3 * V;
    if (n12 <= T(2) * n3V) return n3V + T(0.5) * n12;                          // case (5)
    const T V6n2n3 = T(6) * n2 * n3V, sqn1 = n1 * n1;
    if (V6n2n3 >= sqn1 && T(3) * n2 * (T(2) * n3V + n1 - n2) <= sqn1)            // case (2)
        return T(0.5) * n1 + K::inv_sqrt12 * F::sqrt_(T(24) * n2 * n3V - sqn1);
    if (V6n2n3 < sqn1) return F::cbrt_(V6n2n3 * n1);                             // case (1)
    // case (3): f(x3, y3, a3, b3, c3); x3 > 0 since n1, n2 > 0 here
    const T n1n2 = n1 * n2;
    const T x3 = T(81) * n1n2 * (n12 - T(2) * n3V);
    const T y32 = F::fdim_(T(23328) * cb(n1n2), x3 * x3);
    const T u3 = F::cbrt_(x3 * x3 + y32);
    const T d3 = n12 - (K::two_cbrt54 * n1n2 + K::two_over_cbrt432 * u3) * F::rsqrt_(u3) *
                           F::sin_(K::pi_6 - K::third * F::atan_(F::div_(F::sqrt_(y32), x3)));
    if (d3 <= n3) return d3;
    // case (4): f(x4, y4, a4, b4, c4); x4 kept > 0 so that atan(y/x) replaces atan2
    const T t4 = T(9) * sq(n12 + n3) - T(18);
    const T x4 = fmax(n1n2 * n3 * (T(324) - T(648) * V), F::tiny());
    T y42 = T(4) * cb(t4) - x4 * x4;
    if (!FAITHFUL) y42 = fmax(y42, T(0));
    const T u4 = F::cbrt_(x4 * x4 + y42);
    return T(0.5) * (n12 + n3) -
           (K::two_over_cbrt864 * t4 + K::two_over_cbrt3456 * u4) * F::rsqrt_(u4) *
               F::sin_(K::pi_6 - K::third * F::atan_(F::div_(F::sqrt_(y42), x4)));
}

// ----------------------------------------------------------------------------
// Sec. 2.4: Scardovelli-Zaleski as in Kawano's implementation.  Inputs are
// the L1-normalised reduced quantities (m1 <= m2 <= m3, m1 + m2 + m3 = 1) and
// the reduced volume w; returns the reduced offset alpha in L1 units.
// For m = (0, 0, 1) and w = 0 the cubic branch is re-entered with alpha == 0
// and its square-root argument is -1/4: the result is NaN, as the paper
// reports for this implementation.
// ----------------------------------------------------------------------------
template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_sz_orig(T w, T m1, T m2, T m3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T m12 = m1 + m2;
    T alpha = T(0);
    const T v1 = F::div_(sq(m1), T(6) * m2 * m3 + T(1e-25));
    const T w6 = T(6) * m1 * m2 * m3 * w;
    if (w < v1) {
        alpha = F::cbrt_(w6);                                                     // case (1)
    } else if (w < v1 + F::div_(T(0.5) * (m2 - m1), m3)) {
        alpha = T(0.5) * (m1 + F::sqrt_(sq(m1) + T(8) * m2 * m3 * (w - v1)));     // case (2)
    } else {
        T v3;
        if (m3 < m12) {
            v3 = (sq(m3) * (T(3) * m12 - m3) + sq(m1) * (m1 - T(3) * m3) +
                  sq(m2) * (m2 - T(3) * m3)) * F::rcp_(T(6) * m1 * m2 * m3);
        } else {
            v3 = F::div_(T(0.5) * m12, m3);
            if (v3 <= w) alpha = m3 * w + T(0.5) * m12;                           // case (5)
        }
        if (alpha == T(0)) {
            const bool case3 = w < v3;
            T q0, sp, a2;
            if (FAITHFUL) {
                T a0, a1;
                if (case3) {                                                      // case (3)
                    a2 = T(-3) * m12;
                    a1 = T(3) * (sq(m1) + sq(m2));
                    a0 = w6 - cb(m1) - cb(m2);
                } else {                                                          // case (4)
                    a2 = T(-1.5);
                    a1 = T(1.5) * (sq(m1) + sq(m2) + sq(m3));
                    a0 = T(0.5) * (w6 - cb(m1) - cb(m2) - cb(m3));
                }
                q0 = K::sixth * (a1 * a2 - T(3) * a0) - K::inv27 * cb(a2);
                sp = F::sqrt_(K::ninth * sq(a2) - K::third * a1);
            } else {
                // the same q0 and sp multiplied out: q0 = 1.5 m1 m2 (m12 - 2 m3 w),
                // sp^2 = 2 m1 m2 in case (3); q0 = 0.75 m1 m2 m3 (1 - 2w),
                // sp^2 = (m1 (2 (m2 + m3) - m1) - (m3 - m2)^2)/4 in case (4), using
                // m1 + m2 + m3 = 1.  The printed forms subtract O(1) terms to get
                // O(sp^3) and lose all digits when m1 << m2.
                a2 = case3 ? T(-3) * m12 : T(-1.5);
                q0 = case3 ? T(1.5) * m1 * m2 * (m12 - T(2) * m3 * w)
                           : T(0.75) * m1 * m2 * m3 * (T(1) - T(2) * w);
                sp = F::sqrt_(case3 ? T(2) * m1 * m2
                                    : T(0.25) * (m1 * (T(2) * (m2 + m3) - m1) - sq(m3 - m2)));
            }
            T arg = F::div_(q0, cb(sp));
            if (!FAITHFUL) arg = fmin(fmax(arg, T(-1)), T(1));
            alpha = T(2) * sp * F::cos_(K::four_pi_3 + K::third * F::acos_(arg)) - K::third * a2;
        }
    }
    return alpha;
}

// ----------------------------------------------------------------------------
// Sec. 2.4: the paper's optimised SZ solution (L1-normalised inputs, the
// reduced volume V; returns the reduced offset in L1 units).
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T solve_sz_opt_listing(T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n12 = n1 + n2, n3V = n3 * V;
    if (n12 <= T(2) * n3V) return n3V + T(0.5) * n12;                          // case (5)
    const T sqn1 = n1 * n1, n26 = T(6) * n2, v1 = sqn1 / n26;                   // n2 > 0 here
    if (v1 <= n3V && n3V < v1 + T(0.5) * (n2 - n1))                              // case (2)
        return T(0.5) * (n1 + F::sqrt_(sqn1 + T(8) * n2 * (n3V - v1)));
    const T V6 = n1 * n26 * n3V;
    if (n3V < v1) return F::cbrt_(V6);                                           // case (1)
    // n1 > 0 here
    const T v3 = n3 < n12 ? (sq(n3) * (T(3) * n12 - n3) + sqn1 * (n1 - T(3) * n3) +
                             sq(n2) * (n2 - T(3) * n3)) / (n1 * n26)
                          : T(0.5) * n12;
    const T sqn12 = sqn1 + sq(n2), V6cbn12 = V6 - cb(n1) - cb(n2);
    const bool case3 = n3V < v3;                                                 // else case (4)
    const T a = case3 ? V6cbn12 : T(0.5) * (V6cbn12 - cb(n3));
    const T b = case3 ? sqn12 : T(0.5) * (sqn12 + sq(n3));
    const T c = case3 ? n12 : T(0.5);
    const T t = F::sqrt_(sq(c) - b);
    const T arg = (cb(c) - T(0.5) * a - T(1.5) * b * c) / cb(t);
    return c - T(2) * t * F::sin_(K::third * F::asin_(arg));
}

// Default form of the optimised SZ solution.  Same cases, thresholds and
// trigonometric root as the listing, with
//  - the case tests multiplied out so that no division is needed
//    (v1 <= n3 V  <=>  n1^2 <= 6 n2 n3 V;  n3 V < v3  <=>  6 n1 n2 n3 V < num3),
//  - the arcsine argument (c^3 - a/2 - 3bc/2)/t^3 written without cancellation:
//    case (3): 1.5 n1 n2 (n1 + n2 - 2 n3 V) / (2 n1 n2)^(3/2),
//    case (4): 0.75 n1 n2 n3 (1 - 2V) / t^3, t^2 = (n1 (2(n2+n3) - n1) - (n3-n2)^2)/4,
//    (algebraically identical for n1 + n2 + n3 = 1), clamped to [-1, 1].
// In FP32 every case is evaluated and the result selected (no divergent
// branches; the warp pays for cases (1), (2) and (5) a few instructions each).
// In FP64 the cases branch (the FP64 pipe is the bottleneck there).
template <typename T>
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
    const T arg = fmin(fmax(q * (rt * rt * rt), T(-1)), T(1));
    const T d34 = c - T(2) * t * F::sin_(K::third * F::asin_(arg));
    if (sizeof(T) == 8) return d34;
    const T d5 = n3V + T(0.5) * n12;
    const T d2 = T(0.5) * (n1 + F::sqrt_(T(8) * n2 * n3V - K::third * sqn1));
    const T d1 = F::cbrt_(V6n2n3 * n1);
    return c5 ? d5 : (c2 ? d2 : (c1 ? d1 : d34));
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_sz_opt(T V, T n1, T n2, T n3) {
    if (FAITHFUL) return solve_sz_opt_listing<T>(V, n1, n2, n3);
    return solve_sz_opt_default<T>(V, n1, n2, n3);
}

// ----------------------------------------------------------------------------
// Sec. 2.5: Newton-Raphson.  Cases (5) and (2) in closed form; case (1) by
// Newton on d^3 = 6 V n1 n2 n3; cases (3) and (4) by Newton on the cubic of
// Eq. 10 from the midpoints of [n2, n1+n2] and [n3, L/2].
// Faithful: 7 steps from n1/2 (case 1), 4 steps (cases 3, 4), the cubic as
// printed.  Default: the cancellation-free cubic g of reduced_residual(), a
// start for case (1) from the exponent of 6 V n1 n2 n3, steps until
// |dd| <= 4 ulp (at most 16) and a bracket safeguard (see newton_bracketed).
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T newton_bracketed(T d, T lo, T hi, T rhs, T n1, T n2, T n3,
                                              T inv_n1) {
    // A step that leaves the bracket is clamped to the bracket end it crossed
    // (the root can sit exactly at an end, e.g. d = L/2 for V0 = 1/2); a second
    // crossing of the same end bisects.  From the bracket midpoint this
    // converges in at most 7 steps on the paper-shaped inputs; 16 bounds it.
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

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_newton(T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n1pn2 = n1 + n2, n3xV = n3 * V;
    if (n1pn2 <= T(2) * n3xV) return n3xV + T(0.5) * n1pn2;                     // case (5)
    const T V6n2n3 = T(6) * n2 * n3xV, sqn1 = n1 * n1;
    if (V6n2n3 >= sqn1 && T(3) * n2 * (T(2) * n3xV + n1 - n2) <= sqn1)          // case (2)
        return T(0.5) * n1 + K::inv_sqrt12 * F::sqrt_(T(24) * n2 * n3xV - sqn1);
    const T V6n1n2n3 = V6n2n3 * n1;
    if (FAITHFUL) {
        T d;
        if (V6n2n3 < sqn1) {                                                     // case (1)
            d = T(0.5) * n1;
            for (int i = 0; i < 7; ++i) d -= (cb(d) - V6n1n2n3) / (T(3) * sq(d));
            return d;
        }
        d = T(0.5) * (n2 + n1pn2);                                               // case (3)
        for (int i = 0; i < 4; ++i) {
            const T f = cb(d) - cb(d - n1) - cb(d - n2) - V6n1n2n3;
            const T fs = T(3) * (sq(d) - sq(d - n1) - sq(d - n2));
            d -= f / fs;
        }
        if (d <= n3) return d;
        d = T(0.5) * (n3 + T(0.5) * (n1pn2 + n3));                               // case (4)
        for (int i = 0; i < 4; ++i) {
            const T f = cb(d) - cb(d - n1) - cb(d - n2) - cb(d - n3) - V6n1n2n3;
            const T fs = T(3) * (sq(d) - sq(d - n1) - sq(d - n2) - sq(d - n3));
            d -= f / fs;
        }
        return d;
    }
    const T inv_n1 = T(1) / n1;                                                  // n1 > 0 here
    const T rhs = V6n2n3;
    if (V6n2n3 < sqn1) {                                                         // case (1)
        // start within a factor 2^(2/3) of the root from the binary exponent of
        // X = 6 V n1 n2 n3 (the "log2 hack" of the nested-interval listing)
        const T X = V6n1n2n3;
        if (!(X > T(0))) return T(0);
        const int e = F::log2_halvings(X) - (sizeof(T) == 4 ? 24 : 53);
        const T d0 = fmin(ldexp(T(1), e / 3), n1);
        return newton_bracketed<T>(d0, T(0), n1, rhs, n1, n2, n3, inv_n1);
    }
    T d = newton_bracketed<T>(T(0.5) * (n2 + n1pn2), n2, n1pn2, rhs, n1, n2, n3, inv_n1);
    if (d <= n3) return d;                                                       // case (3)
    const T hl = T(0.5) * (n1pn2 + n3);
    return newton_bracketed<T>(T(0.5) * (n3 + hl), n3, hl, rhs, n1, n2, n3, inv_n1);  // (4)
}

// ----------------------------------------------------------------------------
// Sec. 2.5: nested intervals.  Cases (5), (2), (1) in closed form; case (3) by
// halving [n2, n1+n2] and, if the result exceeds n3, case (4) by halving
// [n3, L/2].  Faithful: the printed predicate (cubes of Eq. 10) and
// floor(log2(width * 2^24)) + 1 halvings (2^53 in double), with the count
// clamped at 0 (the listing's unsigned count would wrap for widths below the
// unit roundoff).  Default: the cancellation-free predicate and halving until
// the ends are adjacent floating-point numbers (at most 128 halvings).
// ----------------------------------------------------------------------------
template <typename T, bool FAITHFUL>
__device__ __forceinline__ T bisect(T dmin, T dmax, T n1, T n2, T n3, bool with_n3, T V6n1n2n3,
                                    T rhs, T inv_n1) {
    T d = T(0.5) * (dmin + dmax);
    if (FAITHFUL) {
        int k = Fm<T>::log2_halvings(dmax - dmin);
        k = k < 0 ? 0 : (k > 1100 ? 1100 : k);
        for (int i = 0; i <= k; ++i) {
            T f = cb(d) - cb(d - n1) - cb(d - n2);
            if (with_n3) f -= cb(d - n3);
            if (f < V6n1n2n3) dmin = d; else dmax = d;
            d = T(0.5) * (dmin + dmax);
        }
        return d;
    }
    for (int i = 0; i < 128; ++i) {
        T g, gp;
        reduced_residual<T>(d, rhs, n1, n2, n3, inv_n1, g, gp);
        if (g < T(0)) dmin = d; else dmax = d;
        const T m = T(0.5) * (dmin + dmax);
        if (m <= dmin || m >= dmax) break;
        d = m;
    }
    return d;
}

template <typename T, bool FAITHFUL>
__device__ __forceinline__ T solve_nested(T V, T n1, T n2, T n3) {
    typedef Fm<T> F;
    typedef Kc<T> K;
    const T n1pn2 = n1 + n2, n3xV = n3 * V;
    if (n1pn2 <= T(2) * n3xV) return n3xV + T(0.5) * n1pn2;                     // case (5)
    const T V6n2n3 = T(6) * n2 * n3xV, sqn1 = n1 * n1;
    if (V6n2n3 >= sqn1 && T(3) * n2 * (T(2) * n3xV + n1 - n2) <= sqn1)          // case (2)
        return T(0.5) * n1 + K::inv_sqrt12 * F::sqrt_(T(24) * n2 * n3xV - sqn1);
    if (V6n2n3 < sqn1) return F::cbrt_(V6n2n3 * n1);                             // case (1)
    const T V6n1n2n3 = V6n2n3 * n1;
    const T inv_n1 = T(1) / n1;
    T d = bisect<T, FAITHFUL>(n2, n1pn2, n1, n2, n3, false, V6n1n2n3, V6n2n3, inv_n1);
    if (d <= n3) return d;                                                       // case (3)
    return bisect<T, FAITHFUL>(n3, T(0.5) * (n1pn2 + n3), n1, n2, n3, true, V6n1n2n3,
                               V6n2n3, inv_n1);                                  // case (4)
}

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
