"""Pins for the oracle's forward volume V0(n, d0) (Sec. 2, Eqs. 1-10).

Each pin is independent of the oracle's own per-case formulas: closed forms the
paper derives, a textbook formula, the 8-vertex inclusion-exclusion sum in 50
digits, Monte-Carlo and midpoint-grid brute force, and the symmetries of the
problem statement.
"""
import itertools
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

EPS = np.finfo(np.float64).eps


def _rand_normals(rng, m):
    g = rng.standard_normal((m, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_axis_aligned_closed_form(orc):
    # Sec. 2.3, 1D case (Eq. 26): with n = +-e_k the volume is d0 + 1/2.
    d0 = np.linspace(-0.5, 0.5, 101)
    for k in range(3):
        for s in (1.0, -1.0):
            n = np.zeros(3)
            n[k] = s
            V = orc.volume(n[0], n[1], n[2], d0)
            np.testing.assert_allclose(V, d0 + 0.5, rtol=0, atol=2 * EPS)
    # outside the cube the volume saturates at 0 and 1
    assert orc.volume(1, 0, 0, -0.7)[0] == 0.0
    assert orc.volume(0, 0, -1, 0.9)[0] == 1.0


def test_2d_closed_form(orc):
    # Sec. 2.3, 2D case (Eq. 27): n1 = 0, reduced d <= n2 gives V = d^2/(2 n2 n3)
    # (a right triangle), otherwise V = (d - n2/2)/n3 (a trapezoid).
    rng = np.random.default_rng(11)
    for _ in range(50):
        a = rng.uniform(0.05, 1.0)
        b = rng.uniform(0.05, 1.0)
        nrm = math.hypot(a, b)
        n2, n3 = sorted((a / nrm, b / nrm))
        for d in rng.uniform(0, 0.5 * (n2 + n3), 8):
            d0 = -(0.5 * (n2 + n3) - d)          # V0 <= 1/2 side (Eq. 8)
            exp = d * d / (2 * n2 * n3) if d <= n2 else (d - n2 / 2) / n3
            got = orc.volume(0.0, a / nrm, -b / nrm, d0)[0]
            assert abs(got - exp) <= 8 * EPS, (a, b, d, got, exp)


def test_space_diagonal_textbook(orc):
    # n = (1,1,1)/sqrt(3): the region x+y+z <= t of the unit cube has the
    # textbook volume t^3/6 - (t-1)_+^3/2 for t in [0, 3/2].
    s = 1 / math.sqrt(3)
    for t in np.linspace(0, 1.5, 61):
        d0 = s * t - 1.5 * s                   # plane x+y+z = t in corner coordinates
        exp = t ** 3 / 6 - max(t - 1, 0) ** 3 / 2
        for signs in itertools.product((1, -1), repeat=3):
            got = orc.volume(signs[0] * s, signs[1] * s, signs[2] * s, d0)[0]
            assert abs(got - exp) <= 16 * EPS


def test_symmetry_and_48_maps(orc):
    # Eq. 6: V0(n, -d0) = 1 - V0(n, d0); Eqs. 2-4: invariance under the 48
    # sign/permutation maps of n.
    rng = np.random.default_rng(12)
    n = _rand_normals(rng, 400)
    h = 0.5 * np.abs(n).sum(1)
    d0 = rng.uniform(-1, 1, 400) * h
    V = orc.volume(n[:, 0], n[:, 1], n[:, 2], d0)
    Vm = orc.volume(n[:, 0], n[:, 1], n[:, 2], -d0)
    np.testing.assert_allclose(V + Vm, 1.0, rtol=0, atol=4 * EPS)
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = n[:, perm] * np.array(signs)
            Vp = orc.volume(m[:, 0], m[:, 1], m[:, 2], d0)
            np.testing.assert_array_equal(Vp, V)


def _volume_mp(n, d0):
    """8-vertex inclusion-exclusion in 50 digits (all |n_k| > 0):
    vol{y in [0,1]^3: a.y <= D} = sum_v (-1)^|v| (D - a.v)_+^3 / (6 a1 a2 a3)."""
    with mpmath.workdps(50):
        a = [abs(mpmath.mpf(float(x))) for x in n]
        D = mpmath.mpf(float(d0)) + (a[0] + a[1] + a[2]) / 2
        tot = mpmath.mpf(0)
        for v in itertools.product((0, 1), repeat=3):
            t = D - sum(a[k] * v[k] for k in range(3))
            if t > 0:
                tot += (-1) ** sum(v) * t ** 3
        return tot / (6 * a[0] * a[1] * a[2])


def test_high_precision_inclusion_exclusion(orc):
    rng = np.random.default_rng(13)
    n = _rand_normals(rng, 300)
    n[:40, 0] *= 1e-3                      # near-2D normals: small n1
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    h = 0.5 * np.abs(n).sum(1)
    d0 = rng.uniform(-1, 1, 300) * h
    V = orc.volume(n[:, 0], n[:, 1], n[:, 2], d0)
    for i in range(300):
        ref = float(_volume_mp(n[i], d0[i]))
        # rounding of d = L/2 - |d0| moves V by at most (dV/dd) * 4 eps L/2,
        # with dV/dd <= sqrt(3)/n3-ish <= 3; the per-case formula adds a few eps.
        tol = 32 * EPS * (abs(ref) + 3 * h[i])
        assert abs(V[i] - ref) <= tol, (i, n[i], d0[i], V[i], ref)


def test_monte_carlo(orc):
    # Brute force: fraction of 2e6 uniform points of [-1/2,1/2]^3 below the plane.
    rng = np.random.default_rng(14)
    pts = rng.random((2_000_000, 3)) - 0.5
    n = _rand_normals(rng, 12)
    n[0] = [0.0, 0.6, 0.8]
    n[1] = [1.0, 0.0, 0.0]
    for i in range(12):
        h = 0.5 * np.abs(n[i]).sum()
        for d0 in (-0.8 * h, -0.3 * h, 0.1 * h, 0.6 * h):
            mc = np.mean(pts @ n[i] <= d0)
            V = orc.volume(n[i, 0], n[i, 1], n[i, 2], d0)[0]
            sigma = math.sqrt(max(V * (1 - V), 1e-12) / pts.shape[0])
            assert abs(mc - V) <= 5 * sigma + 1e-6, (n[i], d0, mc, V)


def test_midpoint_grid_brute_force(orc):
    # Brute force on a 160^3 midpoint grid; the error of a midpoint count is
    # bounded by the number of grid cells the plane crosses (<= sqrt3*3/160
    # of the volume).
    g = (np.arange(160) + 0.5) / 160 - 0.5
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    rng = np.random.default_rng(15)
    n = _rand_normals(rng, 6)
    for i in range(6):
        h = 0.5 * np.abs(n[i]).sum()
        for d0 in (-0.7 * h, -0.2 * h, 0.4 * h):
            cnt = np.mean(n[i, 0] * X + n[i, 1] * Y + n[i, 2] * Z <= d0)
            V = orc.volume(n[i, 0], n[i, 1], n[i, 2], d0)[0]
            assert abs(cnt - V) <= 3 * math.sqrt(3) / 160


def test_scale_invariance_and_invalid(orc):
    # Eq. 1 is homogeneous: V0(lambda n, lambda d0) = V0(n, d0) (general n).
    rng = np.random.default_rng(16)
    n = _rand_normals(rng, 100)
    d0 = rng.uniform(-0.8, 0.8, 100)
    V = orc.volume(n[:, 0], n[:, 1], n[:, 2], d0)
    V4 = orc.volume(4 * n[:, 0], 4 * n[:, 1], 4 * n[:, 2], 4 * d0)
    np.testing.assert_allclose(V4, V, rtol=0, atol=4 * EPS)
    assert np.isnan(orc.volume(0, 0, 0, 0.1)[0])
    assert np.isnan(orc.volume(np.nan, 0, 1, 0.1)[0])
