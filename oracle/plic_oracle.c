/*
 * plic_oracle.c -- plain, slow FP64 reference for the PLIC hot path of
 * Lehmann & Gekle, "Analytic Solution to the Piecewise Linear Interface
 * Construction Problem and its Application in Curvature Calculation for
 * Volume-of-Fluid Simulation Codes" (arXiv 2006.12838).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the timed
 * CPU baseline of the benchmark may load this library.  The GPU library never
 * links it, and it shares no code, header or table with the GPU library.
 *
 * What it computes (all FP64, general normals, no normalisation assumed):
 *   - oracle_volume      V0(n, d0) = vol{x in [-1/2,1/2]^3 : n.x <= d0}
 *                        (the problem statement of Sec. 2, Eq. 1, evaluated in
 *                        the reduced space of Eqs. 2-8 with the per-case
 *                        volume of Eq. 10, written without cancellation).
 *   - oracle_offset      the inverse: the unique d0 in [-L/2, L/2] with
 *                        V0(n, d0) = V0, found by bisection down to adjacent
 *                        doubles (V0 is monotone in d0, Sec. 2.1).
 *   - oracle_area_centroid  area and centroid of the cut polygon, by clipping
 *                        the plane against the 12 cube edges; these give the
 *                        adjoints dd0/dV0 = |n|/A and grad_n d0 = centroid.
 *   - oracle_curvature   the curvature step of Sec. 4.2 and Appendix B:
 *                        Parker-Youngs normal (Eq. 38), local frame (Sec. 4.2),
 *                        PLIC-corrected neighbour points (Eq. 36), paraboloid
 *                        least squares solved by Gaussian elimination with
 *                        partial pivoting, mean curvature (Eq. 42).
 *   - oracle_curvature_grad_fd  central finite differences of sum_i w_i kappa_i
 *                        with respect to the fill field.
 *   - oracle_cm_normal   the centre-of-mass normal of Appendix B (unit weights).
 *   - oracle_sphere_volume / oracle_sphere_offset  the plane-sphere problem of
 *                        Sec. 3: spherical-cap volume of the unit-volume ball
 *                        and its inverse by bisection.
 *
 * Readings of the paper that this file fixes (where it is silent or garbled):
 *   - case (5) holds for n1+n2 <= d <= n3; written as min(n1+n2,n3) <= d the
 *     condition of Eq. 10 would also admit d == n3 when n3 < n1+n2, where the
 *     case-(5) formula is wrong.
 *   - the D3Q27 direction order is recovered from the gradient sums of
 *     Appendix B (the printed table of Eq. 37 is garbled).
 *   - curvature sign: by default kappa = -(Eq. 42), positive for a convex fluid
 *     region, because the Parker-Youngs normal points into the gas.
 *   - with m < 5 interface neighbours, or a near-singular normal matrix, only the
 *     leading parameters in the order (A, B, C, H, I) are fitted; the others stay 0.
 *   - only cells whose 26 neighbours are all inside the field are curvature
 *     cells; the interface set is 0 < phi < 1 on the stored values.
 *   - neighbour-normal variant (Sec. 4.2 mentions it; the paper gives no
 *     formula): neighbour i contributes the point e_i + d0(phi_i, n_i) n_i
 *     relative to the centre's d0(phi_0, n) n, with n_i its own normal; this is
 *     Eq. 36 when n_i = n.  A neighbour whose own 3^3 stencil leaves the field,
 *     or whose normal is undefined, uses the centre normal.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------------------
 * Sec. 2.1, Eqs. 2-4: mirror the normal to |n| and sort the components.
 * ------------------------------------------------------------------------- */
static void sort3(double a, double b, double c, double *n1, double *n2, double *n3)
{
    double t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    *n1 = a; *n2 = b; *n3 = c;
}

/* ---------------------------------------------------------------------------
 * Eq. 10 (Sec. 2.2): volume below the plane n1*y1 + n2*y2 + n3*y3 = d inside
 * the unit cube [0,1]^3, for 0 <= n1 <= n2 <= n3, n3 > 0, 0 <= d <= L/2.
 *   case (1)  d < n1             : d^3 / (6 n1 n2 n3)
 *   case (2)  n1 <= d <= n2      : (d^3 - (d-n1)^3) / (6 n1 n2 n3)
 *                                 = (3 d (d-n1) + n1^2) / (6 n2 n3)
 *   case (3)/(4) n2 < d < n1+n2  : (d^3 - (d-n1)^3 - (d-n2)^3 - (d-n3)_+^3) / (6 n1 n2 n3)
 *                                 = (3 d (d-n1) + n1^2 - ((d-n2)^3 + (d-n3)_+^3)/n1) / (6 n2 n3)
 *   case (5)  n1+n2 <= d <= n3   : (d - (n1+n2)/2) / n3
 * The expanded forms divide out the factor n1 that d^3 - (d-n1)^3 carries, so
 * no term cancels when n1 is small (2D-like normals).  In cases (3)/(4)
 * 0 < d-n2 < n1, so (d-n2)^3/n1 < n1^2 is bounded.
 * ------------------------------------------------------------------------- */
static double vol_reduced(double d, double n1, double n2, double n3)
{
    if (!(d > 0.0)) return 0.0;
    if (d >= n1 + n2)                       /* case (5); implies n1+n2 <= n3 here */
        return (d - 0.5 * (n1 + n2)) / n3;
    if (d < n1)                             /* case (1) */
        return d * d * d / (6.0 * n1 * n2 * n3);
    if (d <= n2)                            /* case (2) */
        return (3.0 * d * (d - n1) + n1 * n1) / (6.0 * n2 * n3);
    {                                       /* cases (3) and (4): n1 > 0 here */
        double e2 = d - n2;
        double e3 = d > n3 ? d - n3 : 0.0;
        return (3.0 * d * (d - n1) + n1 * n1 - (e2 * e2 * e2 + e3 * e3 * e3) / n1)
               / (6.0 * n2 * n3);
    }
}

/* Sec. 2 (Eq. 1 with Eqs. 5-8): V0(n, d0) for a general, non-zero normal.
 * The shift to the corner origin gives d = L/2 - |d0| (Eq. 7), and the half
 * with d0 > 0 follows from V0(n, d0) = 1 - V0(n, -d0) (Eq. 6). */
ORC_EXPORT double oracle_volume(double nx, double ny, double nz, double d0)
{
    double n1, n2, n3, h;
    if (isnan(nx) || isnan(ny) || isnan(nz) || isnan(d0)) return NAN;
    sort3(fabs(nx), fabs(ny), fabs(nz), &n1, &n2, &n3);
    if (!(n3 > 0.0) || isinf(n3)) return NAN;
    h = 0.5 * (n1 + n2 + n3);
    if (d0 <= -h) return 0.0;
    if (d0 >= h) return 1.0;
    if (d0 <= 0.0) return vol_reduced(h + d0, n1, n2, n3);
    return 1.0 - vol_reduced(h - d0, n1, n2, n3);
}

/* Sec. 2, Eq. 1: d0 in [-L/2, L/2] with V0(n, d0) = V0, by bisection.
 * Following Eqs. 5-8 the search runs in the reduced space: V = V0 for
 * V0 <= 1/2 and V = 1 - V0 otherwise (both exact in binary floating point),
 * then d in [0, L/2] with vol_reduced(d) = V is bracketed until the ends are
 * adjacent doubles, and d0 = sign(V0 - 1/2) (L/2 - d).  Comparing against the
 * exact V instead of against V0 keeps the volume residual relative to V,
 * which matters for V0 close to 1.  The end with the smaller residual is
 * returned.  V0 = 0 and V0 = 1 give -L/2 and +L/2 (d = 0 in Eq. 8). */
ORC_EXPORT double oracle_offset(double nx, double ny, double nz, double V0)
{
    double n1, n2, n3, h, lo, hi, V, d;
    int it;
    if (isnan(nx) || isnan(ny) || isnan(nz) || isnan(V0)) return NAN;
    if (V0 < 0.0 || V0 > 1.0) return NAN;
    sort3(fabs(nx), fabs(ny), fabs(nz), &n1, &n2, &n3);
    if (!(n3 > 0.0) || isinf(n3)) return NAN;
    h = 0.5 * (n1 + n2 + n3);
    V = V0 <= 0.5 ? V0 : 1.0 - V0;
    lo = 0.0;
    hi = h;
    if (V == 0.0) {
        d = 0.0;
    } else {
        for (it = 0; it < 2200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (vol_reduced(mid, n1, n2, n3) < V) lo = mid;
            else hi = mid;
        }
        d = (V - vol_reduced(lo, n1, n2, n3) <= vol_reduced(hi, n1, n2, n3) - V) ? lo : hi;
    }
    return V0 < 0.5 ? -(h - d) : (h - d);
}

/* ---------------------------------------------------------------------------
 * Cut polygon of the plane n.x = d0 with the cube [-1/2,1/2]^3: its area A and
 * centroid c.  By the implicit function theorem applied to Eq. 1,
 *   dV0/dd0 = A/|n|,  dV0/dn_k = -A c_k/|n|,
 *   dd0/dV0 = |n|/A,  dd0/dn_k = c_k.
 * The polygon is found by intersecting the plane with the 12 cube edges,
 * ordering the intersection points by angle around their mean in the plane,
 * and summing a triangle fan.  Returns the number of intersection points.
 * ------------------------------------------------------------------------- */
static const int CUBE_EDGES[12][2] = {
    {0, 1}, {2, 3}, {4, 5}, {6, 7},       /* along x */
    {0, 2}, {1, 3}, {4, 6}, {5, 7},       /* along y */
    {0, 4}, {1, 5}, {2, 6}, {3, 7}        /* along z */
};

/* Vertex v of the cell [-1/2,1/2]^3 of Sec. 2.1; bit k of v picks the sign of
 * coordinate k. */
static void cube_vertex(int v, double p[3])
{
    p[0] = (v & 1) ? 0.5 : -0.5;
    p[1] = (v & 2) ? 0.5 : -0.5;
    p[2] = (v & 4) ? 0.5 : -0.5;
}

/* Area and centroid of the cut polygon of the plane n.x = d0 (Eq. 1), as the
 * block comment above describes. */
ORC_EXPORT int oracle_area_centroid(double nx, double ny, double nz, double d0,
                                    double *area, double centroid[3])
{
    double n[3] = {nx, ny, nz};
    double pts[12][3], ang[12], m[3] = {0, 0, 0}, u[3], w[3], len;
    int np = 0, e, i, j, k;
    double f[8];

    for (i = 0; i < 8; ++i) {
        double p[3];
        cube_vertex(i, p);
        f[i] = n[0] * p[0] + n[1] * p[1] + n[2] * p[2] - d0;
    }
    for (e = 0; e < 12; ++e) {
        int a = CUBE_EDGES[e][0], b = CUBE_EDGES[e][1];
        if ((f[a] < 0.0) != (f[b] < 0.0)) {
            double pa[3], pb[3], t = f[a] / (f[a] - f[b]);
            cube_vertex(a, pa);
            cube_vertex(b, pb);
            for (k = 0; k < 3; ++k) pts[np][k] = pa[k] + t * (pb[k] - pa[k]);
            ++np;
        }
    }
    *area = 0.0;
    centroid[0] = centroid[1] = centroid[2] = 0.0;
    if (np < 3) return np;

    for (i = 0; i < np; ++i)
        for (k = 0; k < 3; ++k) m[k] += pts[i][k] / np;
    /* in-plane basis u, w with u perpendicular to n */
    if (fabs(n[0]) <= fabs(n[1]) && fabs(n[0]) <= fabs(n[2])) { u[0] = 0; u[1] = n[2]; u[2] = -n[1]; }
    else if (fabs(n[1]) <= fabs(n[2])) { u[0] = n[2]; u[1] = 0; u[2] = -n[0]; }
    else { u[0] = n[1]; u[1] = -n[0]; u[2] = 0; }
    len = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (k = 0; k < 3; ++k) u[k] /= len;
    w[0] = n[1] * u[2] - n[2] * u[1];
    w[1] = n[2] * u[0] - n[0] * u[2];
    w[2] = n[0] * u[1] - n[1] * u[0];
    for (i = 0; i < np; ++i) {
        double q[3] = {pts[i][0] - m[0], pts[i][1] - m[1], pts[i][2] - m[2]};
        ang[i] = atan2(q[0] * w[0] + q[1] * w[1] + q[2] * w[2],
                       q[0] * u[0] + q[1] * u[1] + q[2] * u[2]);
    }
    /* insertion sort by angle */
    for (i = 1; i < np; ++i) {
        double a = ang[i], p[3] = {pts[i][0], pts[i][1], pts[i][2]};
        for (j = i - 1; j >= 0 && ang[j] > a; --j) {
            ang[j + 1] = ang[j];
            for (k = 0; k < 3; ++k) pts[j + 1][k] = pts[j][k];
        }
        ang[j + 1] = a;
        for (k = 0; k < 3; ++k) pts[j + 1][k] = p[k];
    }
    for (i = 1; i + 1 < np; ++i) {
        double a[3], b[3], c[3], ta;
        for (k = 0; k < 3; ++k) { a[k] = pts[i][k] - pts[0][k]; b[k] = pts[i + 1][k] - pts[0][k]; }
        c[0] = a[1] * b[2] - a[2] * b[1];
        c[1] = a[2] * b[0] - a[0] * b[2];
        c[2] = a[0] * b[1] - a[1] * b[0];
        ta = 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        *area += ta;
        for (k = 0; k < 3; ++k) centroid[k] += ta * (pts[0][k] + pts[i][k] + pts[i + 1][k]) / 3.0;
    }
    if (*area > 0.0)
        for (k = 0; k < 3; ++k) centroid[k] /= *area;
    return np;
}

/* ---------------------------------------------------------------------------
 * Batched wrappers (OpenMP over cells): Eq. 10 (oracle_volume), Eq. 1
 * (oracle_offset) and the cut polygon of Eq. 1 (oracle_area_centroid), cell by
 * cell.
 * ------------------------------------------------------------------------- */
ORC_EXPORT void oracle_volume_batch(const double *nx, const double *ny, const double *nz,
                                    const double *d0, double *V0, int64_t n)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) V0[i] = oracle_volume(nx[i], ny[i], nz[i], d0[i]);
}

ORC_EXPORT void oracle_offset_batch(const double *nx, const double *ny, const double *nz,
                                    const double *V0, double *d0, int64_t n)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 256)
    for (i = 0; i < n; ++i) d0[i] = oracle_offset(nx[i], ny[i], nz[i], V0[i]);
}

ORC_EXPORT void oracle_area_centroid_batch(const double *nx, const double *ny, const double *nz,
                                           const double *d0, double *area, double *cx,
                                           double *cy, double *cz, int64_t n)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double c[3];
        oracle_area_centroid(nx[i], ny[i], nz[i], d0[i], &area[i], c);
        cx[i] = c[0]; cy[i] = c[1]; cz[i] = c[2];
    }
}

/* OpenMP threads the batched functions use (plumbing; no passage). */
ORC_EXPORT int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the batched functions that follow (timing on one core). */
ORC_EXPORT void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * Curvature (Sec. 4.2 and Appendix B).
 *
 * D3Q27 directions e_0..e_26 in the order that the gradient sums of
 * Appendix B imply (Eq. 37 itself is garbled in the source):
 * 1..6 faces, 7..18 edges, 19..26 corners, opposite pairs adjacent.
 * ------------------------------------------------------------------------- */
static const int E27[27][3] = {
    { 0, 0, 0},
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
    { 1, 1, 0}, {-1,-1, 0}, { 1, 0, 1}, {-1, 0,-1}, { 0, 1, 1}, { 0,-1,-1},
    { 1,-1, 0}, {-1, 1, 0}, { 1, 0,-1}, {-1, 0, 1}, { 0, 1,-1}, { 0,-1, 1},
    { 1, 1, 1}, {-1,-1,-1}, { 1, 1,-1}, {-1,-1, 1}, { 1,-1, 1}, {-1, 1,-1},
    {-1, 1, 1}, { 1,-1,-1}
};

/* The D3Q27 directions above (Appendix B), as 27 x 3 ints. */
ORC_EXPORT void oracle_d3q27(int *e81)
{
    int i, k;
    for (i = 0; i < 27; ++i)
        for (k = 0; k < 3; ++k) e81[3 * i + k] = E27[i][k];
}

/* Eq. 38: Parker-Youngs normal n = -sum w_i e_i phi_i / |.|, with w_i = 4, 2, 1
 * for |e_i| = 1, sqrt 2, sqrt 3.  Returns 0 when the weighted sum vanishes. */
ORC_EXPORT int oracle_py_normal(const double *phi27, double n[3])
{
    double g[3] = {0, 0, 0}, len;
    int i, k;
    for (i = 1; i < 27; ++i) {
        int e2 = E27[i][0] * E27[i][0] + E27[i][1] * E27[i][1] + E27[i][2] * E27[i][2];
        double w = e2 == 1 ? 4.0 : (e2 == 2 ? 2.0 : 1.0);
        for (k = 0; k < 3; ++k) g[k] += w * E27[i][k] * phi27[i];
    }
    len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(len > 0.0)) { n[0] = n[1] = n[2] = 0.0; return 0; }
    for (k = 0; k < 3; ++k) n[k] = -g[k] / len;
    return 1;
}

/* Appendix B, centre-of-mass normal: n = -sum e_i phi_i / |.| (all weights 1).
 * Returns 0 when the sum vanishes. */
ORC_EXPORT int oracle_cm_normal(const double *phi27, double n[3])
{
    double g[3] = {0, 0, 0}, len;
    int i, k;
    for (i = 1; i < 27; ++i)
        for (k = 0; k < 3; ++k) g[k] += E27[i][k] * phi27[i];
    len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(len > 0.0)) { n[0] = n[1] = n[2] = 0.0; return 0; }
    for (k = 0; k < 3; ++k) n[k] = -g[k] / len;
    return 1;
}

/* Gaussian elimination with partial pivoting on a k x k system (row-major
 * a[5][5], right-hand side b[5]); solution in x.  Returns the determinant.
 * The solve of the paraboloid fit's normal equations (Appendix B, Eqs. 43-48). */
static double gauss_solve(int k, const double ain[5][5], const double *bin, double *x)
{
    double a[5][6], det = 1.0;
    int i, j, r;
    for (i = 0; i < k; ++i) {
        for (j = 0; j < k; ++j) a[i][j] = ain[i][j];
        a[i][k] = bin ? bin[i] : 0.0;
    }
    for (j = 0; j < k; ++j) {
        int p = j;
        for (r = j + 1; r < k; ++r)
            if (fabs(a[r][j]) > fabs(a[p][j])) p = r;
        if (p != j) {
            for (i = 0; i <= k; ++i) { double t = a[j][i]; a[j][i] = a[p][i]; a[p][i] = t; }
            det = -det;
        }
        det *= a[j][j];
        if (a[j][j] == 0.0) return 0.0;
        for (r = j + 1; r < k; ++r) {
            double f = a[r][j] / a[j][j];
            for (i = j; i <= k; ++i) a[r][i] -= f * a[j][i];
        }
    }
    if (x) {
        for (j = k - 1; j >= 0; --j) {
            double s = a[j][k];
            for (i = j + 1; i < k; ++i) s -= a[j][i] * x[i];
            x[j] = s / a[j][j];
        }
    }
    return det;
}

/* Relative size below which a pivot of the normal matrix counts as singular
 * (pivot = ratio of consecutive leading principal minors, compared with the
 * trace of M). */
#define ORC_FIT_TAU 1e-6

/* Appendix B (Eqs. 43-48): least-squares paraboloid z = A x^2 + B y^2 + C x y
 * + H x + I y through m points.  M = sum Q Q^T, b = sum z Q with
 * Q = (x^2, y^2, xy, x, y).  The fit dimension is min(m, 5), reduced further
 * while a leading pivot det(M_j)/det(M_{j-1}) is below ORC_FIT_TAU * trace(M);
 * the leading block is solved by Gaussian elimination with partial pivoting,
 * the remaining parameters stay 0.  Returns the dimension used. */
static int lsq_fit(int m, const double *px, const double *py, const double *pz, double *x5,
                   double *minpiv);

ORC_EXPORT int oracle_lsq_paraboloid(int m, const double *px, const double *py,
                                     const double *pz, double *x5)
{
    return lsq_fit(m, px, py, pz, x5, NULL);
}

/* The fit of oracle_lsq_paraboloid; *minpiv (nullable) receives the smallest
 * leading pivot of the dimension used, divided by trace(M) (1 when no
 * parameter is fitted): a measure of the fit's conditioning, reported beside
 * kappa. */
static int lsq_fit(int m, const double *px, const double *py, const double *pz, double *x5,
                   double *minpiv)
{
    double M[5][5], b[5], tr = 0.0, detprev = 1.0, pmin = 1.0;
    int i, j, p, dim;
    memset(M, 0, sizeof M);
    memset(b, 0, sizeof b);
    for (i = 0; i < 5; ++i) x5[i] = 0.0;
    for (p = 0; p < m; ++p) {
        double Q[5] = {px[p] * px[p], py[p] * py[p], px[p] * py[p], px[p], py[p]};
        for (i = 0; i < 5; ++i) {
            for (j = 0; j < 5; ++j) M[i][j] += Q[i] * Q[j];
            b[i] += pz[p] * Q[i];
        }
    }
    for (i = 0; i < 5; ++i) tr += M[i][i];
    dim = m < 5 ? m : 5;
    for (j = 1; j <= dim; ++j) {
        double det = gauss_solve(j, (const double (*)[5])M, NULL, NULL);
        if (!(det / detprev > ORC_FIT_TAU * tr)) { dim = j - 1; break; }
        if (det / detprev / tr < pmin) pmin = det / detprev / tr;
        detprev = det;
    }
    if (dim > 0) gauss_solve(dim, (const double (*)[5])M, b, x5);
    if (minpiv) *minpiv = pmin;
    return dim;
}

/* Eq. 42: mean curvature of the paraboloid at the origin. */
ORC_EXPORT double oracle_paraboloid_kappa(const double *x5)
{
    double A = x5[0], B = x5[1], C = x5[2], H = x5[3], I = x5[4];
    double s = H * H + I * I + 1.0;
    return (A * (I * I + 1.0) + B * (H * H + 1.0) - C * H * I) / (s * sqrt(s));
}

#define ORC_POINT_CENTROID 2u
#define ORC_KAPPA_PAPER_SIGN 4u
#define ORC_NORMAL_CM 64u
#define ORC_NEIGHBOR_NORMAL 128u

/* Sec. 4.2: curvature of one interface cell from its 3^3 fill stencil in D3Q27
 * order.  Steps: Parker-Youngs normal (Eq. 38; the centre-of-mass normal of
 * Appendix B with ORC_NORMAL_CM); frame b_z = n, b_y = (b_z x r)/|.|,
 * b_x = b_y x b_z with the fixed r of Sec. 4.2 (rotated cyclically in the
 * event that it is parallel to n); PLIC-corrected points of the interface
 * neighbours (Eq. 36); least-squares paraboloid; Eq. 42.
 * Point mode (default): foot of the PLIC plane along the normal, as in Eq. 36.
 * ORC_POINT_CENTROID: centroid of each neighbour's cut polygon instead.
 * Normals of the neighbour planes: the centre normal (Eq. 36), or, with
 * ORC_NEIGHBOR_NORMAL and nn81 != NULL, nn81[3i..3i+2] for neighbour i where
 * that entry is non-zero (the centre normal where it is zero).
 * iface27 (nullable) fixes which neighbours count as interface cells; when it
 * is NULL the test 0 < phi_i < 1 is applied to phi27 itself.
 * Writes the fit dimension and the number of neighbour points; returns kappa
 * (-(Eq. 42) unless ORC_KAPPA_PAPER_SIGN). */
static double curvature_cell(const double *phi27, const int *iface27, const double *nn81,
                             unsigned flags, int *dim_out, int *npts_out, double *minpiv);

ORC_EXPORT double oracle_curvature_cell(const double *phi27, const int *iface27,
                                        const double *nn81, unsigned flags,
                                        int *dim_out, int *npts_out)
{
    return curvature_cell(phi27, iface27, nn81, flags, dim_out, npts_out, NULL);
}

/* oracle_curvature_cell, with the fit's conditioning (lsq_fit) in *minpiv
 * (nullable; 1 when no fit is made). */
static double curvature_cell(const double *phi27, const int *iface27, const double *nn81,
                             unsigned flags, int *dim_out, int *npts_out, double *minpiv)
{
    static const double R[3] = {0.56270900, 0.32704452, 0.75921047};
    double n[3], by[3], bx[3], r[3], len, d00, c0[3] = {0, 0, 0}, x5[5];
    double px[26], py[26], pz[26];
    int i, k, m = 0, dim, ok;

    if (dim_out) *dim_out = 0;
    if (npts_out) *npts_out = 0;
    if (minpiv) *minpiv = 1.0;
    ok = (flags & ORC_NORMAL_CM) ? oracle_cm_normal(phi27, n) : oracle_py_normal(phi27, n);
    if (!ok) return 0.0;
    r[0] = R[0]; r[1] = R[1]; r[2] = R[2];
    for (k = 0; k < 2; ++k) {
        by[0] = n[1] * r[2] - n[2] * r[1];
        by[1] = n[2] * r[0] - n[0] * r[2];
        by[2] = n[0] * r[1] - n[1] * r[0];
        len = sqrt(by[0] * by[0] + by[1] * by[1] + by[2] * by[2]);
        if (len > 1e-6) break;
        r[0] = R[1]; r[1] = R[2]; r[2] = R[0];
    }
    for (k = 0; k < 3; ++k) by[k] /= len;
    bx[0] = by[1] * n[2] - by[2] * n[1];
    bx[1] = by[2] * n[0] - by[0] * n[2];
    bx[2] = by[0] * n[1] - by[1] * n[0];

    d00 = oracle_offset(n[0], n[1], n[2], phi27[0]);
    if (flags & ORC_POINT_CENTROID) {
        double a;
        oracle_area_centroid(n[0], n[1], n[2], d00, &a, c0);
    }
    for (i = 1; i < 27; ++i) {
        double v = phi27[i], d0i, q[3], ni[3];
        int is_iface = iface27 ? iface27[i] : (v > 0.0 && v < 1.0);
        if (!is_iface) continue;
        for (k = 0; k < 3; ++k) ni[k] = n[k];
        if ((flags & ORC_NEIGHBOR_NORMAL) && nn81 &&
            (nn81[3 * i] != 0.0 || nn81[3 * i + 1] != 0.0 || nn81[3 * i + 2] != 0.0))
            for (k = 0; k < 3; ++k) ni[k] = nn81[3 * i + k];
        d0i = oracle_offset(ni[0], ni[1], ni[2], v);
        if (flags & ORC_POINT_CENTROID) {
            double a, ci[3];
            oracle_area_centroid(ni[0], ni[1], ni[2], d0i, &a, ci);
            for (k = 0; k < 3; ++k) q[k] = E27[i][k] + ci[k] - c0[k];
        } else {
            /* foot points d0 n of the two planes (Eq. 36 for ni = n) */
            for (k = 0; k < 3; ++k) q[k] = E27[i][k] + d0i * ni[k] - d00 * n[k];
        }
        px[m] = q[0] * bx[0] + q[1] * bx[1] + q[2] * bx[2];
        py[m] = q[0] * by[0] + q[1] * by[1] + q[2] * by[2];
        pz[m] = q[0] * n[0] + q[1] * n[1] + q[2] * n[2];
        ++m;
    }
    dim = lsq_fit(m, px, py, pz, x5, minpiv);
    if (dim_out) *dim_out = dim;
    if (npts_out) *npts_out = m;
    if (dim == 0) return 0.0;
    return (flags & ORC_KAPPA_PAPER_SIGN) ? oracle_paraboloid_kappa(x5)
                                          : -oracle_paraboloid_kappa(x5);
}

/* Gather the 27 stencil values phi(x + e_i) of cell (x,y,z) of a field stored
 * x-fastest, in the D3Q27 order of Appendix B. */
static void gather27(const float *phi, int nx, int ny, int64_t c, double *out)
{
    int i;
    for (i = 0; i < 27; ++i) {
        int64_t o = E27[i][0] + (int64_t)nx * (E27[i][1] + (int64_t)ny * E27[i][2]);
        out[i] = (double)phi[c + o];
    }
}

/* Neighbour normals for ORC_NEIGHBOR_NORMAL (the variant of Sec. 4.2 in which
 * each neighbour's PLIC point uses its own normal): for each interface
 * neighbour i of cell c whose own 26 neighbours lie inside the field, its PY
 * (Eq. 38) or CM (Appendix B) normal; zero (centre normal) otherwise. */
static void neighbour_normals(const float *phi, int nx, int ny, int nz, int64_t c,
                              const double *s27, unsigned flags, double *nn81)
{
    int64_t x = c % nx, y = (c / nx) % ny, z = c / ((int64_t)nx * ny);
    int i, k;
    for (i = 0; i < 81; ++i) nn81[i] = 0.0;
    for (i = 1; i < 27; ++i) {
        int64_t xi = x + E27[i][0], yi = y + E27[i][1], zi = z + E27[i][2];
        double t[27], ni[3];
        int ok;
        if (!(s27[i] > 0.0 && s27[i] < 1.0)) continue;
        if (xi < 1 || yi < 1 || zi < 1 || xi > nx - 2 || yi > ny - 2 || zi > nz - 2) continue;
        gather27(phi, nx, ny, xi + (int64_t)nx * (yi + (int64_t)ny * zi), t);
        ok = (flags & ORC_NORMAL_CM) ? oracle_cm_normal(t, ni) : oracle_py_normal(t, ni);
        if (ok)
            for (k = 0; k < 3; ++k) nn81[3 * i + k] = ni[k];
    }
}

/* Curvature (Sec. 4.2, Appendix B: oracle_curvature_cell) for a list of
 * interface cells (linear indices x + nx*(y + ny*z)). */
ORC_EXPORT void oracle_curvature_batch(const float *phi, int nx, int ny, int nz,
                                       const int32_t *idx, int64_t n_iface, unsigned flags,
                                       double *kappa, int32_t *dim, int32_t *npts,
                                       double *minpiv)
{
    int64_t k;
#pragma omp parallel for schedule(dynamic, 64)
    for (k = 0; k < n_iface; ++k) {
        double s[27], nn[81];
        int dm, np;
        gather27(phi, nx, ny, idx[k], s);
        if (flags & ORC_NEIGHBOR_NORMAL) neighbour_normals(phi, nx, ny, nz, idx[k], s, flags, nn);
        kappa[k] = curvature_cell(s, NULL, (flags & ORC_NEIGHBOR_NORMAL) ? nn : NULL, flags,
                                  &dm, &np, minpiv ? minpiv + k : NULL);
        if (dim) dim[k] = dm;
        if (npts) npts[k] = np;
    }
}

/* Normals (PY of Eq. 38, or the CM normal of Appendix B with ORC_NORMAL_CM)
 * of a list of interface cells; zero where undefined. */
ORC_EXPORT void oracle_normal_batch(const float *phi, int nx, int ny, int nz,
                                    const int32_t *idx, int64_t n_iface, unsigned flags,
                                    double *nx_out, double *ny_out, double *nz_out)
{
    int64_t k;
    (void)nz;
#pragma omp parallel for schedule(static)
    for (k = 0; k < n_iface; ++k) {
        double s[27], n[3];
        gather27(phi, nx, ny, idx[k], s);
        if (flags & ORC_NORMAL_CM) oracle_cm_normal(s, n);
        else oracle_py_normal(s, n);
        nx_out[k] = n[0];
        ny_out[k] = n[1];
        nz_out[k] = n[2];
    }
}

/* The adjoint of the curvature step (Sec. 4.2, Appendix B) by brute force:
 * central finite differences of J = sum_k w_k kappa_k with respect to every
 * fill value in the field (FP64 perturbations of the FP32 field values).  The
 * interface set is the given list and is held fixed.  For each interface cell
 * k and each of its 27 stencil entries j, kappa_k is re-evaluated at
 * phi_j +- h; the difference quotient is accumulated into g[j].  g is dense,
 * nx*ny*nz, and is overwritten. */
ORC_EXPORT void oracle_curvature_grad_fd(const float *phi, int nx, int ny, int nz,
                                         const int32_t *idx, int64_t n_iface,
                                         const double *w, double h, unsigned flags,
                                         double *g)
{
    int64_t N = (int64_t)nx * ny * nz, k;
    double *contrib = (double *)malloc(sizeof(double) * 27 * (size_t)(n_iface > 0 ? n_iface : 1));
    memset(g, 0, sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(dynamic, 16)
    for (k = 0; k < n_iface; ++k) {
        double s[27];
        int j, mask[27];
        gather27(phi, nx, ny, idx[k], s);
        for (j = 0; j < 27; ++j) mask[j] = s[j] > 0.0 && s[j] < 1.0;
        for (j = 0; j < 27; ++j) {
            double keep = s[j], kp, km;
            s[j] = keep + h;
            kp = oracle_curvature_cell(s, mask, NULL, flags, NULL, NULL);
            s[j] = keep - h;
            km = oracle_curvature_cell(s, mask, NULL, flags, NULL, NULL);
            s[j] = keep;
            contrib[27 * k + j] = w[k] * (kp - km) / (2.0 * h);
        }
    }
    for (k = 0; k < n_iface; ++k) {
        int j;
        for (j = 0; j < 27; ++j) {
            int64_t o = E27[j][0] + (int64_t)nx * (E27[j][1] + (int64_t)ny * E27[j][2]);
            g[idx[k] + o] += contrib[27 * k + j];
        }
    }
    free(contrib);
    (void)nz;
}

/* ---------------------------------------------------------------------------
 * Sec. 3: plane-sphere intersection.  The ball has unit volume, so its radius
 * is r = (3/(4 pi))^(1/3).  V0(d0) is the volume of the part of the ball on
 * the side n.x <= d0 of a plane at signed distance d0 from the centre: a
 * spherical cap of height h = r + d0, V0 = pi h^2 (3r - h)/3
 * = pi/3 (r + d0)^2 (2r - d0); 0 for d0 <= -r and 1 for d0 >= r.  The
 * normal's direction does not matter.
 * ------------------------------------------------------------------------- */
static double sphere_radius(void) { return cbrt(3.0 / (4.0 * 3.14159265358979323846)); }

/* The cap volume of Sec. 3 described above. */
ORC_EXPORT double oracle_sphere_volume(double d0)
{
    double r = sphere_radius(), h;
    if (isnan(d0)) return NAN;
    if (d0 <= -r) return 0.0;
    if (d0 >= r) return 1.0;
    h = r + d0;
    return 3.14159265358979323846 / 3.0 * h * h * (3.0 * r - h);
}

/* The inverse problem of Sec. 3: d0 in [-r, r] with V0(d0) = V0, by
 * bisection down to adjacent doubles (V0 increases strictly on [-r, r]).  By
 * the symmetry V0(-d0) = 1 - V0(d0) the search runs for W = min(V0, 1 - V0)
 * on [-r, 0] and the sign is restored, so the residual stays relative to W. */
ORC_EXPORT double oracle_sphere_offset(double V0)
{
    double r = sphere_radius(), W, lo, hi, d;
    int it;
    if (isnan(V0) || V0 < 0.0 || V0 > 1.0) return NAN;
    W = V0 <= 0.5 ? V0 : 1.0 - V0;
    lo = -r;
    hi = 0.0;
    if (W == 0.0) {
        d = -r;
    } else {
        for (it = 0; it < 2200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (oracle_sphere_volume(mid) < W) lo = mid;
            else hi = mid;
        }
        d = (W - oracle_sphere_volume(lo) <= oracle_sphere_volume(hi) - W) ? lo : hi;
    }
    return V0 <= 0.5 ? d : -d;
}

/* Sec. 3, cell by cell (OpenMP). */
ORC_EXPORT void oracle_sphere_volume_batch(const double *d0, double *V0, int64_t n)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) V0[i] = oracle_sphere_volume(d0[i]);
}

/* Sec. 3, cell by cell (OpenMP). */
ORC_EXPORT void oracle_sphere_offset_batch(const double *V0, double *d0, int64_t n)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) d0[i] = oracle_sphere_offset(V0[i]);
}
