"""Pins for the oracle's inverse d0(n, V0) (bisection on Eq. 1).

The bisection is checked against the paper's closed-form and analytic
solutions (Eq. 25 with Eqs. 11, 13-22, evaluated in 50-digit arithmetic), the
1D and 2D closed forms of Sec. 2.3, and the tie-breaks of Eq. 8.
"""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

EPS = np.finfo(np.float64).eps


def _rand_normals(rng, m):
    g = rng.standard_normal((m, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _paper_offset_mp(n, V0):
    """Eq. 25 (a-posteriori conditions, order 5 -> 2 -> 1 -> 3 -> 4) with the
    real trigonometric root f of Eq. 11 and the constants of Eqs. 13-22, in
    50-digit arithmetic, for a unit normal with all components non-zero.
    Returns (d0, case)."""
    with mpmath.workdps(50):
        a = sorted(abs(mpmath.mpf(float(x))) for x in n)
        nrm = mpmath.sqrt(a[0] ** 2 + a[1] ** 2 + a[2] ** 2)
        n1, n2, n3 = (x / nrm for x in a)          # exactly unit in 50 digits
        V0m = mpmath.mpf(float(V0))
        V = mpmath.mpf(0.5) - abs(V0m - mpmath.mpf(0.5))

        def f(x, y, A, B, C):
            r2 = x * x + y * y
            return C - 2 * (A + B * mpmath.cbrt(r2)) / r2 ** (mpmath.mpf(1) / 6) * \
                mpmath.sin(mpmath.pi / 6 - mpmath.atan2(y, x) / 3)

        d5 = V * n3 + (n1 + n2) / 2
        d2 = n1 / 2 + mpmath.sqrt(max(2 * V * n2 * n3 - n1 * n1 / 12, 0))
        d1 = mpmath.cbrt(6 * V * n1 * n2 * n3)
        x3 = 81 * n1 * n2 * (n1 + n2 - 2 * V * n3)
        y3 = mpmath.sqrt(max(23328 * (n1 * n2) ** 3 - x3 * x3, 0))
        d3 = f(x3, y3, mpmath.cbrt(54) * n1 * n2, 1 / mpmath.cbrt(432), n1 + n2)
        t4 = 9 * (n1 + n2 + n3) ** 2 - 18
        x4 = 324 * n1 * n2 * n3 * (1 - 2 * V)
        y4 = mpmath.sqrt(max(4 * t4 ** 3 - x4 * x4, 0))
        d4 = f(x4, y4, t4 / mpmath.cbrt(864), 1 / mpmath.cbrt(3456), (n1 + n2 + n3) / 2)
        if n1 + n2 <= d5 <= n3:
            d, case = d5, 5
        elif n1 <= d2 <= n2:
            d, case = d2, 2
        elif d1 < n1:
            d, case = d1, 1
        elif n2 <= d3 <= min(n1 + n2, n3):
            d, case = d3, 3
        else:
            d, case = d4, 4
        # Eq. 8; the oracle works with the given (double) n, so the unit-n
        # offset is scaled back by |n|
        d0 = mpmath.sign(V0m - mpmath.mpf(0.5)) * ((n1 + n2 + n3) / 2 - d) * nrm
        return float(d0), case


def test_paper_analytic_solution_all_cases(orc):
    rng = np.random.default_rng(21)
    n = _rand_normals(rng, 400)
    V0 = rng.random(400)
    # push some cells into the small-V corner cases (1) and (2)
    V0[:60] = rng.random(60) * 1e-2
    V0[60:90] = 1 - rng.random(30) * 1e-3
    d0 = orc.offset(n[:, 0], n[:, 1], n[:, 2], V0)
    seen = set()
    for i in range(400):
        ref, case = _paper_offset_mp(n[i], V0[i])
        seen.add(case)
        assert abs(d0[i] - ref) <= 1e-14, (i, case, n[i], V0[i], d0[i], ref)
    assert seen == {1, 2, 3, 4, 5}, seen


def test_1d_closed_form(orc):
    # Sec. 2.3 (Eq. 26): d = V, i.e. d0 = V0 - 1/2 for axis-aligned normals.
    V0 = np.concatenate([np.linspace(0, 1, 257), [1e-300, 1 - 2 ** -53]])
    for k in range(3):
        for s in (1.0, -1.0):
            n = np.zeros(3)
            n[k] = s
            d0 = orc.offset(n[0], n[1], n[2], V0)
            np.testing.assert_allclose(d0, V0 - 0.5, rtol=0, atol=2 * EPS)


def test_2d_closed_form(orc):
    # Sec. 2.3 (Eq. 27): d = sqrt(2 V n2 n3) if d <= n2, else V n3 + n2/2.
    rng = np.random.default_rng(22)
    for _ in range(200):
        a, b = rng.uniform(0.02, 1, 2)
        nrm = math.hypot(a, b)
        n2, n3 = sorted((a / nrm, b / nrm))
        V0 = rng.random()
        V = 0.5 - abs(V0 - 0.5)
        d = math.sqrt(2 * V * n2 * n3)
        if d > n2:
            d = V * n3 + n2 / 2
        exp = math.copysign(0.5 * (n2 + n3) - d, V0 - 0.5)
        got = orc.offset(-a / nrm, 0.0, b / nrm, V0)[0]
        assert abs(got - exp) <= 1e-15, (a, b, V0, got, exp)


def test_ties_and_invalid(orc):
    rng = np.random.default_rng(23)
    n = _rand_normals(rng, 50)
    h = 0.5 * np.abs(n).sum(1)
    # Eq. 8 with d = 0: V0 = 0 and V0 = 1 give -L/2 and +L/2 exactly.
    np.testing.assert_allclose(orc.offset(n[:, 0], n[:, 1], n[:, 2], 0.0), -h, rtol=0, atol=2 * EPS)
    np.testing.assert_allclose(orc.offset(n[:, 0], n[:, 1], n[:, 2], 1.0), h, rtol=0, atol=2 * EPS)
    # V0 = 1/2 gives d0 = 0 (up to the bisection's last step).
    assert np.abs(orc.offset(n[:, 0], n[:, 1], n[:, 2], 0.5)).max() <= 1e-15
    for bad in (-1e-9, 1 + 1e-9, np.nan):
        assert np.isnan(orc.offset(0.6, 0.8, 0.0, bad)[0])
    assert np.isnan(orc.offset(0.0, 0.0, 0.0, 0.3)[0])


def test_round_trip_and_monotone(orc):
    rng = np.random.default_rng(24)
    n = _rand_normals(rng, 5000)
    V0 = rng.random(5000)
    d0 = orc.offset(n[:, 0], n[:, 1], n[:, 2], V0)
    V = orc.volume(n[:, 0], n[:, 1], n[:, 2], d0)
    assert np.abs(V - V0).max() <= 4 * EPS
    # strictly increasing in V0 for a fixed normal
    Vs = np.sort(rng.random(2000))
    ds = orc.offset(0.3, -0.5, math.sqrt(1 - 0.34), Vs)
    assert np.all(np.diff(ds) >= 0)
