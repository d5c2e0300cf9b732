// vof_curvature.cuh -- the per-cell curvature step (Sec. 4.2, Appendix B),
// shared by the single-field and the batched kernels.
//
// For one interface cell c of a field phi (x-fastest):
//   1. gather the 3^3 stencil (D3Q27 order of Appendix B);
//   2. Parker-Youngs normal n = -sum w_i e_i phi_i / |.| (Eq. 38; the weights
//      4/2/1 make it a separable [1 2 1] x [1 2 1] smoothed central difference);
//   3. frame b_z = n, b_y = (n x r)/|.|, b_x = b_y x b_z (Sec. 4.2), r rotated
//      cyclically in the event that it is parallel to n;
//   4. PLIC offsets d0(phi_0, n) and d0(phi_i, n) of the interface neighbours,
//      all with the centre normal (FP32 solver + one Newton polish), giving the
//      points p_i = (e_i . b_x, e_i . b_y, e_i . b_z + d0_i - d0_0) (Eq. 36), or
//      the cut-polygon centroids with PLIC_FLAG_POINT_CENTROID;
//   5. normal equations M = sum Q Q^T, b = sum z Q, Q = (x^2, y^2, xy, x, y),
//      accumulated in FP32 (Appendix B);
//   6. LDL^T solve of the leading block (dimension min(m, 5), reduced while a
//      pivot is <= 1e-6 trace(M)) in FP64, FP32 or double-float;
//   7. mean curvature of the paraboloid at the origin (Eq. 42), negated by
//      default so that a convex fluid region has kappa > 0.
#pragma once
#include <type_traits>
#include "plic_polygon.cuh"

namespace plic {

enum { FIT_FP64 = 0, FIT_FP32 = 1, FIT_DF32 = 2, FIT_AUTO = 3 };

// D3Q27 directions e_0..e_26, packed as (ex+1) + 3 (ey+1) + 9 (ez+1).
#define PLIC_E27_PACKED          \
    13,                          \
    14, 12, 16, 10, 22, 4,       \
    17, 9, 23, 3, 25, 1,         \
    11, 15, 5, 21, 19, 7,        \
    26, 0, 8, 18, 20, 6,         \
    24, 2
__constant__ unsigned char c_e27[27] = {PLIC_E27_PACKED};
struct E27Table {
    static constexpr unsigned char v[27] = {PLIC_E27_PACKED};
};

// e_i from the constant table: the cheapest in registers; the lanes of a warp
// that ask for different i are served one address at a time.
__device__ __forceinline__ void e_of(int i, int& ex, int& ey, int& ez) {
    const int p = c_e27[i];
    ex = p % 3 - 1;
    ey = (p / 3) % 3 - 1;
    ez = p / 9 - 1;
}

// e_i decoded from immediates, for indices that differ across the lanes of a
// warp: the components (+1) are 2-bit fields of two 32-bit words per axis
// (entries 0-15 and 16-26), entry i at bits 2 (i mod 16).
constexpr uint32_t e27_word(int axis, int half) {
    uint32_t w = 0;
    for (int i = 16 * half; i < 27 && i < 16 * half + 16; ++i) {
        const int p = E27Table::v[i];
        const int e = axis == 0 ? p % 3 : axis == 1 ? (p / 3) % 3 : p / 9;
        w |= (uint32_t)e << (2 * (i - 16 * half));
    }
    return w;
}
template <int AXIS>
struct E27Words {
    static constexpr uint32_t lo = e27_word(AXIS, 0), hi = e27_word(AXIS, 1);
};
template <int AXIS>
__device__ __forceinline__ int e27_comp(int i) {
    const uint32_t w = i < 16 ? E27Words<AXIS>::lo : E27Words<AXIS>::hi;
    return (int)((w >> (2 * (i & 15))) & 3u) - 1;
}

__device__ __forceinline__ void e_of_lanes(int i, int& ex, int& ey, int& ez) {
    ex = e27_comp<0>(i);
    ey = e27_comp<1>(i);
    ez = e27_comp<2>(i);
}

// The D3Q27 directions as a block-shared table (integer and float
// components), filled by the first 27 threads of the block (every thread of
// the block must call fill()): loops over per-lane entries look their
// directions up (one shared load each) instead of decoding them.
struct E27Shared {
    int4 ei[27];
    float4 ef[27];
    __device__ __forceinline__ void fill() {
        if (threadIdx.x < 27) {
            int ex, ey, ez;
            e_of_lanes((int)threadIdx.x, ex, ey, ez);
            ei[threadIdx.x] = make_int4(ex, ey, ez, 0);
            ef[threadIdx.x] = make_float4((float)ex, (float)ey, (float)ez, 0.0f);
        }
        __syncthreads();
    }
};

// The same table for a compile-time index (fully unrolled loops): folds to
// constants.
template <int I>
__device__ __forceinline__ void e_of_c(int& ex, int& ey, int& ez) {
    constexpr int p = E27Table::v[I];
    ex = p % 3 - 1;
    ey = (p / 3) % 3 - 1;
    ez = p / 9 - 1;
}
// f(std::integral_constant<int, Q>) for Q = FROM..26, in order.
template <int FROM, typename F>
__device__ __forceinline__ void for_e27(F&& f) {
    if constexpr (FROM < 27) {
        f(std::integral_constant<int, FROM>{});
        for_e27<FROM + 1>(f);
    }
}

template <int FIT> struct FitReal;
template <> struct FitReal<FIT_FP64> {
    typedef double R;
    static __device__ __forceinline__ R mk(float a) { return (double)a; }
    static __device__ __forceinline__ R add(R a, R b) { return a + b; }
    static __device__ __forceinline__ R sub(R a, R b) { return a - b; }
    static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
    static __device__ __forceinline__ R div(R a, R b) { return a / b; }
    static __device__ __forceinline__ float tof(R a) { return (float)a; }
    static __device__ __forceinline__ bool gt(R a, R b) { return a > b; }
};
template <> struct FitReal<FIT_FP32> {
    typedef float R;
    static __device__ __forceinline__ R mk(float a) { return a; }
    static __device__ __forceinline__ R add(R a, R b) { return a + b; }
    static __device__ __forceinline__ R sub(R a, R b) { return a - b; }
    static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
    // MUFU reciprocal and a multiply (2 ulp): the divisors are the LDL^T pivots,
    // positive and far inside the normal range
    static __device__ __forceinline__ R div(R a, R b) { return a * rcp_approx(b); }
    static __device__ __forceinline__ float tof(R a) { return a; }
    static __device__ __forceinline__ bool gt(R a, R b) { return a > b; }
};
template <> struct FitReal<FIT_DF32> {
    typedef df R;
    static __device__ __forceinline__ R mk(float a) { return df_make(a); }
    static __device__ __forceinline__ R add(R a, R b) { return df_add(a, b); }
    static __device__ __forceinline__ R sub(R a, R b) { return df_add(a, df_neg(b)); }
    static __device__ __forceinline__ R mul(R a, R b) { return df_mul(a, b); }
    static __device__ __forceinline__ R div(R a, R b) { return df_div(a, b); }
    static __device__ __forceinline__ float tof(R a) { return a.hi + a.lo; }
    static __device__ __forceinline__ bool gt(R a, R b) {
        return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
    }
};

// Packed upper triangle of the symmetric 5x5 normal matrix.
__host__ __device__ constexpr int uidx(int i, int j) {
    return i <= j ? i * 5 - i * (i - 1) / 2 + (j - i) : j * 5 - j * (j - 1) / 2 + (i - j);
}

// LDL^T factorisation of the leading block of the symmetric normal matrix
// (Appendix B reduces the fit dimension when fewer than 5 points exist).  The
// dimension is min(m, 5), reduced to j at the first pivot D_j <= 1e-6 trace(M)
// (D_j is the ratio of consecutive leading principal minors).  solve() uses
// the factors for any right-hand side (the fit, and the adjoint system of the
// backward pass); unused parameters are 0.
template <int FIT>
struct Ldlt {
    typedef FitReal<FIT> F;
    typedef typename F::R R;
    R Lm[5][5], D[5];
    int dim;
    __device__ __forceinline__ void factor(const float* Mf, int m) {
        const float trace = Mf[uidx(0, 0)] + Mf[uidx(1, 1)] + Mf[uidx(2, 2)] + Mf[uidx(3, 3)] + Mf[uidx(4, 4)];
        const R tol = F::mk(1e-6f * trace);
        dim = m < 5 ? m : 5;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            R dj = F::mk(Mf[uidx(j, j)]);
#pragma unroll
            for (int k = 0; k < j; ++k) dj = F::sub(dj, F::mul(F::mul(Lm[j][k], Lm[j][k]), D[k]));
            const bool act = j < dim;
            if (act && !F::gt(dj, tol)) dim = j;
            D[j] = dj;
            const bool use = j < dim;
            const R inv = use ? F::div(F::mk(1.0f), dj) : F::mk(0.0f);
#pragma unroll
            for (int i = j + 1; i < 5; ++i) {
                R s = F::mk(Mf[uidx(i, j)]);
#pragma unroll
                for (int k = 0; k < j; ++k) s = F::sub(s, F::mul(F::mul(Lm[i][k], Lm[j][k]), D[k]));
                Lm[i][j] = F::mul(s, inv);
            }
        }
    }
    __device__ __forceinline__ void solve(const float* bf, float x[5]) const {
        R y[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            R s = F::mk(bf[i]);
#pragma unroll
            for (int k = 0; k < i; ++k) s = F::sub(s, F::mul(Lm[i][k], y[k]));
            y[i] = i < dim ? s : F::mk(0.0f);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) y[i] = i < dim ? F::div(y[i], D[i]) : F::mk(0.0f);
        R xs[5];
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            R s = y[i];
#pragma unroll
            for (int k = i + 1; k < 5; ++k) s = F::sub(s, F::mul(Lm[k][i], xs[k]));
            xs[i] = i < dim ? s : F::mk(0.0f);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) x[i] = F::tof(xs[i]);
    }
};

// Adaptive factorisation (the FIT_AUTO policy): LDL^T in FP32, replaced by an
// FP64 factorisation when the FP32 pivots show an ill-conditioned matrix
// (smallest pivot below 1e-2 of the largest, or a dimension reduced by the
// FP32 pivots).  Same interface as Ldlt (factor(), solve(), dim).  The FP64
// factors are not kept: the rare wide solve refactorises from Mf, which must
// stay valid between factor() and the solves; this keeps the FP64 factors out
// of the registers of the common path.
struct LdltAuto {
    Ldlt<FIT_FP32> f;
    const float* Mf;
    int m, dim;
    bool wide;
    __device__ __forceinline__ void factor(const float* M, int mm) {
        Mf = M;
        m = mm;
        f.factor(M, mm);
        const int want = mm < 5 ? mm : 5;
        float dmin = 3.4e38f, dmax = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if (j < f.dim) { dmin = fminf(dmin, f.D[j]); dmax = fmaxf(dmax, f.D[j]); }
        wide = !(f.dim == want && dmin > 1e-2f * dmax);
        dim = f.dim;
        if (wide) {
            Ldlt<FIT_FP64> w;
            w.factor(M, mm);
            dim = w.dim;
        }
    }
    __device__ __forceinline__ void solve(const float* bf, float x[5]) const {
        if (wide) {
            Ldlt<FIT_FP64> w;
            w.factor(Mf, m);
            w.solve(bf, x);
        } else {
            f.solve(bf, x);
        }
    }
};

template <int FIT>
__device__ __forceinline__ int fit_solve(const float* Mf, const float* bf, int m, float x[5]) {
    Ldlt<FIT> f;
    f.factor(Mf, m);
    f.solve(bf, x);
    return f.dim;
}

// Eq. 42 at the origin: (A (I^2+1) + B (H^2+1) - C H I) / (H^2 + I^2 + 1)^(3/2).
__device__ __forceinline__ float paraboloid_kappa(const float x[5]) {
    const float A = x[0], B = x[1], C = x[2], H = x[3], I = x[4];
    const float s = fmaf(H, H, fmaf(I, I, 1.0f));
    const float r = rsqrtf(s);
    return (A * fmaf(I, I, 1.0f) + B * fmaf(H, H, 1.0f) - C * H * I) * (r * r * r);
}

// The reduced normal of the centre cell, shared by all PLIC solves of the cell.
template <int METHOD>
struct CellPlic {
    float n1, n2, n3, L, m1, m2, m3;
    __device__ __forceinline__ void prepare(float nx, float ny, float nz) {
        reduce_normal<float, false>(nx, ny, nz, n1, n2, n3);
        L = fabsf(nx) + fabsf(ny) + fabsf(nz);
        if (METHOD == M_SZ_ORIG) {
            m1 = n1 / L;
            m3 = n3 / L;
            m2 = fmaxf(1.0f - (m1 + m3), 0.0f);
        }
    }
    // d0(V0, n) in FP32 with one Newton polish (PLIC_FP32_POLISHED); V0 in (0, 1).
    __device__ __forceinline__ float offset(float V0) const {
        const float V = V0 <= 0.5f ? V0 : 1.0f - V0;
        if (METHOD == M_SZ_ORIG) {
            float a = solve_sz_orig<float, false>(V, m1, m2, m3);
            a = polish<float>(a, V, m1, m2, m3);
            return L * copysignf(0.5f - a, V0 - 0.5f);
        }
        float d = METHOD == M_ANALYTIC ? solve_analytic<float, false>(V, n1, n2, n3)
                : METHOD == M_NEWTON   ? solve_newton<float, false>(V, n1, n2, n3)
                                       : solve_nested<float, false>(V, n1, n2, n3);
        d = polish<float>(d, V, n1, n2, n3);
        return copysignf(0.5f * (n1 + n2 + n3) - d, V0 - 0.5f);
    }
};

// The optimised SZ solution (Sec. 2.4) with everything that depends on the
// normal alone computed once per curvature cell (all neighbour solves of a
// cell use the centre normal, Eq. 36).  Per solve there remain: the reduced
// volume, four threshold tests on V, the closed forms of cases (5), (2), (1)
// (the last as cbrt(6 m1 m2 m3) * cbrt(V)), the trigonometric root of cases
// (3)/(4) with the cancellation-free arcsine argument written as
// (n1+n2 - 2 m3 V) s3 or (1 - 2V) s4, and the FP32 Newton polish of the
// trigonometric root.  Same cases and formulas as solve_sz_opt_default; the
// thresholds are the product-form tests divided through once.
template <>
struct CellPlic<M_SZ_OPT> {
    float L, m1, m2, m3, n12;
    float V5, V1, V2, V3;
    float s3, t3, s4, t4, k2a, k2b, cb1, inv1, k6;
    __device__ __forceinline__ void prepare(float nx, float ny, float nz) {
        const float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
        L = ax + ay + az;
        // MUFU reciprocals (no IEEE division): the thresholds only choose
        // between case formulas that agree at the case boundaries
        const float il = rcp_approx(L);
        m1 = fminf(fminf(ax, ay), az) * il;
        m3 = fmaxf(fmaxf(ax, ay), az) * il;
        m2 = fmaxf(1.0f - (m1 + m3), 0.0f);
        n12 = m1 + m2;
        const float m1m2 = m1 * m2, sq1 = m1 * m1;
        const float k23 = 6.0f * m2 * m3;
        const float rk = k23 > 0.0f ? rcp_approx(k23) : 0.0f;
        inv1 = m1 > 0.0f ? rcp_approx(m1) : 0.0f;
        V5 = 0.5f * n12 * rcp_approx(m3);                  // case (5): V >= V5
        V1 = sq1 * rk;                                           // case (1): V < V1
        V2 = (sq1 - 3.0f * m2 * (m1 - m2)) * rk;                 // case (2): V < V2
        const float num3 = m3 * m3 * (3.0f * n12 - m3) + sq1 * (m1 - 3.0f * m3) + m2 * m2 * (m2 - 3.0f * m3);
        V3 = (m3 < n12 && m1m2 > 0.0f) ? num3 * rk * inv1 : 3.4e38f;  // case (3): V < V3
        const float t32 = 2.0f * m1m2;
        const float r3 = t32 > 0.0f ? rsqrtf(t32) : 0.0f;
        t3 = t32 * r3;
        s3 = 1.5f * m1m2 * r3 * r3 * r3;
        const float d32 = m3 - m2;
        const float t42 = 0.25f * (m1 * (2.0f * (m2 + m3) - m1) - d32 * d32);
        const float r4 = t42 > 0.0f ? rsqrtf(t42) : 0.0f;
        t4 = t42 * r4;
        s4 = 0.75f * m1m2 * m3 * r4 * r4 * r4;
        k2a = 8.0f * m2 * m3;
        k2b = sq1 * (1.0f / 3.0f);
        cb1 = Fm<float>::cbrt_(k23 * m1);
        k6 = k23;
    }
    __device__ __forceinline__ float offset(float V0) const {
        const float V = fminf(V0, 1.0f - V0);
        const bool c5 = V >= V5, c1 = V < V1, c2 = !c1 && V < V2, c3 = V < V3;
        const float d5 = fmaf(m3, V, 0.5f * n12);
        const float d2 = 0.5f * (m1 + Fm<float>::sqrt_(fmaxf(fmaf(k2a, V, -k2b), 1e-30f)));
        const float d1 = cb1 * Fm<float>::cbrt_(V);
        const float x = c3 ? fmaf(-2.0f * m3, V, n12) : fmaf(-2.0f, V, 1.0f);
        const float arg = fminf(x * (c3 ? s3 : s4), 1.0f);
        const float t = c3 ? t3 : t4, c = c3 ? n12 : 0.5f;
        float d = fmaf(-2.0f * t, __sinf((1.0f / 3.0f) * fast_asinf(arg)), c);
        // polish of the trigonometric root (cases 3/4: d >= m2, m1 > 0)
        const float e2 = d - m2, e3 = fmaxf(d - m3, 0.0f);
        const float e22 = e2 * e2, e33 = e3 * e3;
        const float g = fmaf(3.0f * d, d - m1, m1 * m1) - fmaf(e22, e2, e33 * e3) * inv1 - k6 * V;
        const float gp = fmaf(6.0f, d, -3.0f * m1) - 3.0f * (e22 + e33) * inv1;
        d = d - g * rcp_approx(gp);
        d = c1 ? d1 : d;
        d = c2 ? d2 : d;
        d = c5 ? d5 : d;
        return L * copysignf(0.5f - d, V0 - 0.5f);
    }
};

// Normal of the 3^3 stencil around cell c (Appendix B): Parker-Youngs
// weights 4/2/1 (Eq. 38), or all 1 for the centre-of-mass normal.  Row by
// row: the weights of the x-difference of row (dy, dz) are w(dy) w(dz) with
// w(0) = 2, w(+-1) = 1; the row sums for the y and z components weigh the
// middle entry 2 (all 1 for CM).  Returns false for a zero weighted sum.
__device__ __forceinline__ bool stencil_normal(const float* __restrict__ phi, int64_t c, int nx,
                                               int64_t nxy, bool cm, float& nx_, float& ny_,
                                               float& nz_) {
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    const float w0 = cm ? 1.0f : 2.0f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const float* row = phi + c + dz * nxy + (int64_t)dy * nx;
            const float a = __ldg(row - 1), b = __ldg(row), e = __ldg(row + 1);
            const float wy = dy == 0 ? w0 : 1.0f, wz = dz == 0 ? w0 : 1.0f;
            const float sum = fmaf(w0, b, a + e);
            gx = fmaf(wy * wz, e - a, gx);
            gy = fmaf((float)dy * wz, sum, gy);
            gz = fmaf((float)dz * wy, sum, gz);
        }
    const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
    if (!(gl > 0.0f)) { nx_ = ny_ = nz_ = 0.0f; return false; }
    const float inv = -1.0f / gl;
    nx_ = gx * inv; ny_ = gy * inv; nz_ = gz * inv;
    return true;
}

// The neighbour-normal variant (PLIC_FLAG_NEIGHBOR_NORMAL), one thread per
// list entry; defined in vof_curvature_nn.cu.  out[k] = scale * kappa[k].
plic_status launch_curvature_nn(const float* phi, int nx, int ny, int nz, const int32_t* idx,
                                int64_t n_iface, const int64_t* d_n_iface, float* out,
                                plic_method m, uint32_t flags, int fit, float scale,
                                void* stream, const char* who);

}  // namespace plic
