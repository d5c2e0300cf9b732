"""Pins for the oracle's adjoints: cut-polygon area A and centroid c, giving
dd0/dV0 = |n|/A and grad_n d0 = c (implicit function theorem on Eq. 1).

Checked against: the axis-aligned closed form, the triangle of case (1) and
the parallelogram of case (5) (textbook areas), a brute-force sampling of the
plane, central finite differences of the oracle's own inverse and forward,
and the Euler identity n . grad_n d0 = d0 of the 1-homogeneous d0(n).
"""
import math

import numpy as np


def _rand_normals(rng, m):
    g = rng.standard_normal((m, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_axis_aligned(orc):
    d0 = np.linspace(-0.45, 0.45, 19)
    for k in range(3):
        for s in (1.0, -1.0):
            n = np.zeros(3)
            n[k] = s
            A, cx, cy, cz = orc.area_centroid(n[0], n[1], n[2], d0)
            c = np.stack([cx, cy, cz], 1)
            np.testing.assert_allclose(A, 1.0, atol=1e-15)
            exp = np.zeros((d0.size, 3))
            exp[:, k] = s * d0
            np.testing.assert_allclose(c, exp, atol=1e-15)


def test_case1_triangle_and_case5_parallelogram(orc):
    rng = np.random.default_rng(31)
    n = np.abs(_rand_normals(rng, 200))
    n.sort(axis=1)                               # n1 <= n2 <= n3, unit
    n1, n2, n3 = n.T
    h = 0.5 * n.sum(1)
    # case (1): reduced d < n1, the cut is the triangle with axis intercepts
    # s_i = d/n_i; its area is sqrt(s1^2 s2^2 + s2^2 s3^2 + s1^2 s3^2)/2.
    d = rng.uniform(0.05, 0.95, 200) * n1
    A, *_ = orc.area_centroid(n1, n2, n3, d - h)
    s1, s2, s3 = d / n1, d / n2, d / n3
    exp = 0.5 * np.sqrt((s1 * s2) ** 2 + (s2 * s3) ** 2 + (s1 * s3) ** 2)
    np.testing.assert_allclose(A, exp, rtol=1e-12)
    # case (5): n1 + n2 <= d <= n3, a parallelogram over the unit square of the
    # (y1, y2) face: area = |n| / n3 and centroid (1/2, 1/2, (d-(n1+n2)/2)/n3) in
    # corner coordinates.
    m = n1 + n2 < n3
    d = n1[m] + n2[m] + rng.uniform(0.05, 0.95, m.sum()) * (n3[m] - n1[m] - n2[m])
    d = np.minimum(d, h[m])
    A, cx, cy, cz = orc.area_centroid(n1[m], n2[m], n3[m], d - h[m])
    np.testing.assert_allclose(A, 1 / n3[m], rtol=1e-12)
    np.testing.assert_allclose(cx, 0.0, atol=1e-12)
    np.testing.assert_allclose(cy, 0.0, atol=1e-12)
    np.testing.assert_allclose(cz, (d - 0.5 * (n1[m] + n2[m])) / n3[m] - 0.5, atol=1e-12)


def test_brute_force_plane_sampling(orc):
    # Sample the plane on a 1200^2 grid in an in-plane basis and keep the
    # samples inside the cube: their count gives the area, their mean the
    # centroid.  Resolution error ~ perimeter * spacing.
    rng = np.random.default_rng(32)
    g = (np.arange(1200) + 0.5) / 1200 * 2.0 - 1.0
    S, T = np.meshgrid(g, g, indexing="ij")
    dA = (2.0 / 1200) ** 2
    for n in _rand_normals(rng, 8):
        h = 0.5 * np.abs(n).sum()
        for d0 in (-0.6 * h, 0.0, 0.3 * h):
            u = np.cross(n, [0.3, 0.5, 0.8])
            u /= np.linalg.norm(u)
            w = np.cross(n, u)
            P = d0 * n + S[..., None] * u + T[..., None] * w
            inside = np.all(np.abs(P) <= 0.5, axis=-1)
            A_bf = inside.sum() * dA
            c_bf = P[inside].mean(0)
            A, cx, cy, cz = orc.area_centroid(n[0], n[1], n[2], d0)
            assert abs(A[0] - A_bf) <= 0.01 * max(A[0], 0.1)
            assert np.linalg.norm(np.array([cx[0], cy[0], cz[0]]) - c_bf) <= 5e-3


def test_finite_differences_and_euler(orc):
    rng = np.random.default_rng(33)
    n = _rand_normals(rng, 3000)
    V0 = rng.uniform(0.01, 0.99, 3000)
    d0 = orc.offset(n[:, 0], n[:, 1], n[:, 2], V0)
    g = rng.standard_normal(3000)
    gV, gx, gy, gz = orc.offset_grad(n[:, 0], n[:, 1], n[:, 2], d0, g)
    A, cx, cy, cz = orc.area_centroid(n[:, 0], n[:, 1], n[:, 2], d0)
    keep = A > 0.05
    h = 1e-6
    fd = (orc.offset(n[:, 0], n[:, 1], n[:, 2], V0 + h)
          - orc.offset(n[:, 0], n[:, 1], n[:, 2], V0 - h)) / (2 * h)
    np.testing.assert_allclose((g * fd)[keep], gV[keep], rtol=1e-6, atol=1e-8)
    for k, gk in enumerate((gx, gy, gz)):
        e = np.zeros(3)
        e[k] = h
        fd = (orc.offset(n[:, 0] + e[0], n[:, 1] + e[1], n[:, 2] + e[2], V0)
              - orc.offset(n[:, 0] - e[0], n[:, 1] - e[1], n[:, 2] - e[2], V0)) / (2 * h)
        np.testing.assert_allclose((g * fd)[keep], gk[keep], rtol=1e-5, atol=1e-8)
    # Euler identity for the 1-homogeneous d0(n): n . grad_n d0 = d0
    np.testing.assert_allclose(n[:, 0] * cx + n[:, 1] * cy + n[:, 2] * cz, d0, atol=1e-14)


def test_volume_grad_finite_differences(orc):
    rng = np.random.default_rng(34)
    n = _rand_normals(rng, 2000)
    hh = 0.5 * np.abs(n).sum(1)
    d0 = rng.uniform(-0.9, 0.9, 2000) * hh
    g = rng.standard_normal(2000)
    gd, gx, gy, gz = orc.volume_grad(n[:, 0], n[:, 1], n[:, 2], d0, g)
    h = 1e-6
    fd = (orc.volume(n[:, 0], n[:, 1], n[:, 2], d0 + h)
          - orc.volume(n[:, 0], n[:, 1], n[:, 2], d0 - h)) / (2 * h)
    np.testing.assert_allclose(g * fd, gd, rtol=1e-6, atol=1e-8)
    for k, gk in enumerate((gx, gy, gz)):
        e = np.zeros(3)
        e[k] = h
        fd = (orc.volume(n[:, 0] + e[0], n[:, 1] + e[1], n[:, 2] + e[2], d0)
              - orc.volume(n[:, 0] - e[0], n[:, 1] - e[1], n[:, 2] - e[2], d0)) / (2 * h)
        np.testing.assert_allclose(g * fd, gk, rtol=1e-5, atol=1e-8)
    assert math.isclose(orc.volume_grad(1, 0, 0, 0.1, 1.0)[0][0], 1.0)
