// plic_polygon.cuh -- area and centroid of the cut polygon of a PLIC plane.
//
// By the implicit function theorem applied to Eq. 1 (unit n), the adjoints of
// the forward and inverse problems need the area A and centroid c of the
// polygon in which the plane n . x = d0 cuts the cube:
//   dV0/dd0 = A,  dV0/dn = -A c,  dd0/dV0 = 1/A,  dd0/dn = c.
// The polygon of each intersection case of Eq. 10 is listed explicitly in the
// reduced corner frame, fanned into triangles, and mapped back.
#pragma once
#include "plic_solvers.cuh"

namespace plic {

// ----------------------------------------------------------------------------
// Cut polygon of the plane n . x = d0 with the cube [-1/2,1/2]^3 (unit n):
// area A and centroid c (cube-centred).  In reduced corner coordinates the
// polygon's vertices are known per case (Sec. 2.2, Fig. 1): a triangle (1), a
// quadrilateral (2), a pentagon (3), a hexagon (4), a parallelogram (5); they
// are listed in cyclic order and summed as a triangle fan.  Returns false
// where the polygon degenerates (d0 at +-L/2 or invalid input).
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ bool cut_polygon(T nx, T ny, T nz, T d0, T& A, T& cx, T& cy, T& cz) {
    const T ax = fabs(nx), ay = fabs(ny), az = fabs(nz);
    // sorting permutation: which original axis holds n1, n2, n3
    int i1, i2, i3;
    if (ax <= ay) {
        if (ay <= az) { i1 = 0; i2 = 1; i3 = 2; }
        else if (ax <= az) { i1 = 0; i2 = 2; i3 = 1; }
        else { i1 = 2; i2 = 0; i3 = 1; }
    } else {
        if (ax <= az) { i1 = 1; i2 = 0; i3 = 2; }
        else if (ay <= az) { i1 = 1; i2 = 2; i3 = 0; }
        else { i1 = 2; i2 = 1; i3 = 0; }
    }
    const T a3[3] = {ax, ay, az};
    const T n1 = a3[i1], n2 = a3[i2], n3 = a3[i3];
    const T L = n1 + n2 + n3, h = T(0.5) * L;
    const T d = h - fabs(d0);
    A = T(0); cx = cy = cz = T(0);
    if (!(L > T(0)) || !(d > T(0))) return false;
    // reciprocals: MUFU-based in FP32 (2 ulp; the adjoints need no more), IEEE in FP64
    const T r2 = n2 > T(0) ? Fm<T>::rcp_(n2) : T(0), r3 = Fm<T>::rcp_(n3);
    const T r1 = n1 > T(0) ? Fm<T>::rcp_(n1) : T(0);
    T p[6][3];
    int np;
    const T n12 = n1 + n2;
    if (d >= n12) {                                   // (5) parallelogram over the unit square
        p[0][0] = 0; p[0][1] = 0; p[0][2] = d * r3;
        p[1][0] = 1; p[1][1] = 0; p[1][2] = (d - n1) * r3;
        p[2][0] = 1; p[2][1] = 1; p[2][2] = (d - n12) * r3;
        p[3][0] = 0; p[3][1] = 1; p[3][2] = (d - n2) * r3;
        np = 4;
    } else if (d < n1) {                              // (1) triangle
        p[0][0] = d * r1; p[0][1] = 0; p[0][2] = 0;
        p[1][0] = 0; p[1][1] = d * r2; p[1][2] = 0;
        p[2][0] = 0; p[2][1] = 0; p[2][2] = d * r3;
        np = 3;
    } else if (d <= n2) {                             // (2) quadrilateral
        p[0][0] = 0; p[0][1] = 0; p[0][2] = d * r3;
        p[1][0] = 0; p[1][1] = d * r2; p[1][2] = 0;
        p[2][0] = 1; p[2][1] = (d - n1) * r2; p[2][2] = 0;
        p[3][0] = 1; p[3][1] = 0; p[3][2] = (d - n1) * r3;
        np = 4;
    } else if (d <= n3) {                             // (3) pentagon
        p[0][0] = 0; p[0][1] = 0; p[0][2] = d * r3;
        p[1][0] = 0; p[1][1] = 1; p[1][2] = (d - n2) * r3;
        p[2][0] = (d - n2) * r1; p[2][1] = 1; p[2][2] = 0;
        p[3][0] = 1; p[3][1] = (d - n1) * r2; p[3][2] = 0;
        p[4][0] = 1; p[4][1] = 0; p[4][2] = (d - n1) * r3;
        np = 5;
    } else {                                          // (4) hexagon
        p[0][0] = 1; p[0][1] = 0; p[0][2] = (d - n1) * r3;
        p[1][0] = (d - n3) * r1; p[1][1] = 0; p[1][2] = 1;
        p[2][0] = 0; p[2][1] = (d - n3) * r2; p[2][2] = 1;
        p[3][0] = 0; p[3][1] = 1; p[3][2] = (d - n2) * r3;
        p[4][0] = (d - n2) * r1; p[4][1] = 1; p[4][2] = 0;
        p[5][0] = 1; p[5][1] = (d - n1) * r2; p[5][2] = 0;
        np = 6;
    }
    // triangle fan from p[0]; signed areas along the unit normal (n1,n2,n3)/|n|
    const T inv_len = Fm<T>::rsqrt_(n1 * n1 + n2 * n2 + n3 * n3);
    const T u1 = n1 * inv_len, u2 = n2 * inv_len, u3 = n3 * inv_len;
    T s = T(0), m1 = T(0), m2 = T(0), m3 = T(0);
#pragma unroll
    for (int k = 1; k < 5; ++k) {
        if (k + 1 < np) {
            const T a1 = p[k][0] - p[0][0], a2 = p[k][1] - p[0][1], a3_ = p[k][2] - p[0][2];
            const T b1 = p[k + 1][0] - p[0][0], b2 = p[k + 1][1] - p[0][1], b3 = p[k + 1][2] - p[0][2];
            const T t = T(0.5) * (u1 * (a2 * b3 - a3_ * b2) + u2 * (a3_ * b1 - a1 * b3) +
                                  u3 * (a1 * b2 - a2 * b1));
            s += t;
            m1 += t * (p[0][0] + p[k][0] + p[k + 1][0]);
            m2 += t * (p[0][1] + p[k][1] + p[k + 1][1]);
            m3 += t * (p[0][2] + p[k][2] + p[k + 1][2]);
        }
    }
    A = fabs(s);
    if (!(A > T(0))) return false;
    const T inv3s = Fm<T>::rcp_(T(3) * s);
    // centroid in reduced corner coordinates, then back: mirror for V0 > 1/2
    // (d0 > 0), unsort, shift to the cube centre, restore the signs of n
    T c[3];
    const T red[3] = {m1 * inv3s, m2 * inv3s, m3 * inv3s};
    c[i1] = red[0]; c[i2] = red[1]; c[i3] = red[2];
    const bool mirror = d0 > T(0);
    const T sx = nx < T(0) ? T(-1) : T(1), sy = ny < T(0) ? T(-1) : T(1), sz = nz < T(0) ? T(-1) : T(1);
    cx = sx * ((mirror ? T(1) - c[0] : c[0]) - T(0.5));
    cy = sy * ((mirror ? T(1) - c[1] : c[1]) - T(0.5));
    cz = sz * ((mirror ? T(1) - c[2] : c[2]) - T(0.5));
    return true;
}

// The same area and centroid without building the polygon, for the adjoint
// kernels.  In the reduced corner frame (n1 <= n2 <= n3 the sorted |n_k|,
// d = (n1+n2+n3)/2 - |d0|, cube [0,1]^3, V(d; n) = vol{n . x <= d}), the
// transport theorem gives dV/dd = A/|n| and dV/dn_k = -A c_k/|n|, so
// c_k = -(dV/dn_k)/(dV/dd).  Differentiating the case formulas of Eq. 10:
//   case (1), d < n1:        dV/dd = d^2/(2 n1 n2 n3),   c_k = d/(3 n_k);
//   cases (2)-(4), else:     with e2 = (d-n2)_+, e3 = (d-n3)_+ and
//                            N = 3d(d-n1) + n1^2 - (e2^3 + e3^3)/n1 (= 6 n2 n3 V),
//                            G = 6d - 3n1 - 3(e2^2 + e3^2)/n1 (= 6 n2 n3 dV/dd):
//                            c1 = (3d - 2n1 - (e2^3 + e3^3)/n1^2)/G,
//                            c2 = (N/n2 - 3 e2^2/n1)/G, c3 = (N/n3 - 3 e3^2/n1)/G
//                            (the 1/n1 terms vanish with e2 = e3 = 0 in case (2),
//                            which also covers n1 = 0);
//   case (5), d >= n1 + n2:  dV/dd = 1/n3, c = (1/2, 1/2, (d - (n1+n2)/2)/n3).
// The reduced centroid is then mapped back like cut_polygon's: mirrored for
// d0 > 0, unsorted (ties broken by axis order), shifted to the cube centre and
// given the signs of n.  Returns false (A = 0) for d <= 0 or n = 0.
template <typename T>
__device__ __forceinline__ bool area_centroid(T nx, T ny, T nz, T d0, T& A, T& cx, T& cy, T& cz) {
    typedef Fm<T> F;
    const T ax = fabs(nx), ay = fabs(ny), az = fabs(nz);
    const T n1 = fmin(fmin(ax, ay), az), n3 = fmax(fmax(ax, ay), az);
    const T n2 = fmax(fmin(ax, ay), fmin(fmax(ax, ay), az));
    const T L = ax + ay + az;
    const T d = T(0.5) * L - fabs(d0);
    A = T(0); cx = cy = cz = T(0);
    if (!(L > T(0)) || !(d > T(0))) return false;
    const T n12 = n1 + n2;
    const T r3 = F::rcp_(n3);
    const T r2 = n2 > T(0) ? F::rcp_(n2) : T(0);
    const T r1 = n1 > T(0) ? F::rcp_(n1) : T(0);
    T vp, c0, c1, c2;
    if (d >= n12) {                                    // (5)
        vp = r3;
        c0 = T(0.5); c1 = T(0.5); c2 = (d - T(0.5) * n12) * r3;
    } else if (d < n1) {                               // (1)
        const T t = d * (T(1) / T(3));
        vp = T(0.5) * d * d * r1 * r2 * r3;
        c0 = t * r1; c1 = t * r2; c2 = t * r3;
    } else {                                           // (2)-(4)
        const T e2 = fmax(d - n2, T(0)), e3 = fmax(d - n3, T(0));
        const T e22 = e2 * e2, e33 = e3 * e3;
        const T cub = (e22 * e2 + e33 * e3) * r1;
        const T N = T(3) * d * (d - n1) + n1 * n1 - cub;
        const T G = T(6) * d - T(3) * n1 - T(3) * (e22 + e33) * r1;
        const T iG = F::rcp_(G);
        vp = G * (T(1) / T(6)) * r2 * r3;
        c0 = (T(3) * d - T(2) * n1 - cub * r1) * iG;
        c1 = (N * r2 - T(3) * e22 * r1) * iG;
        c2 = (N * r3 - T(3) * e33 * r1) * iG;
    }
    A = F::sqrt_(n1 * n1 + n2 * n2 + n3 * n3) * vp;
    if (!(A > T(0))) return false;
    // ranks of the three axes in the sort (ties by axis order)
    const int rx = (ax > ay) + (ax > az), ry = (ay >= ax) + (ay > az), rz = (az >= ax) + (az >= ay);
    auto pick = [&](int r) { return r == 0 ? c0 : (r == 1 ? c1 : c2); };
    const bool mirror = d0 > T(0);
    const T ux = pick(rx), uy = pick(ry), uz = pick(rz);
    cx = (mirror ? T(0.5) - ux : ux - T(0.5));
    cy = (mirror ? T(0.5) - uy : uy - T(0.5));
    cz = (mirror ? T(0.5) - uz : uz - T(0.5));
    if (nx < T(0)) cx = -cx;
    if (ny < T(0)) cy = -cy;
    if (nz < T(0)) cz = -cz;
    return true;
}

}  // namespace plic
