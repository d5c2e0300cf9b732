// plic_polygon.cuh -- area and centroid of the cut polygon of a PLIC plane.
//
// By the implicit function theorem applied to Eq. 1 (unit n), the adjoints of
// the forward and inverse problems need the area A and centroid c of the
// polygon in which the plane n . x = d0 cuts the cube:
//   dV0/dd0 = A,  dV0/dn = -A c,  dd0/dV0 = 1/A,  dd0/dn = c;
// the curvature step's centroid points use c as well.  Both are obtained from
// the derivatives of the case volumes of Eq. 10, without building the polygon.
#pragma once
#include "plic_solvers.cuh"

namespace plic {

// In the reduced corner frame (n1 <= n2 <= n3 the sorted |n_k|,
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
// The reduced centroid is then mapped back to the cube: mirrored for
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
