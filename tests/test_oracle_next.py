"""Pins for the oracle's plane-sphere problem (Sec. 3), the centre-of-mass
normal (Appendix B) and the neighbour-normal curvature variant (Sec. 4.2).

- Sphere: the radius gives unit volume; the cap volume equals the integral of
  the slice areas pi (r^2 - z^2) (scipy quad); V(-d) = 1 - V(d); dV/dd is the
  slice area; the bisection inverse meets the paper's trigonometric closed
  form of Sec. 3 evaluated in 50-digit mpmath.
- CM normal: against the nine-term sums printed in Appendix B (golden file)
  and exact on linear fields.
- Neighbour normals: with every neighbour given the centre normal the variant
  is Eq. 36; planar fields give 0; spheres give 1/R; the batched gather of the
  neighbours' own stencils matches a numpy re-gather; kappa is invariant under
  axis flips and permutations of the whole field.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2006_12838_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
R_UNIT = (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)


# ---------------------------------------------------------------------------
# Sec. 3: plane-sphere
# ---------------------------------------------------------------------------
def test_sphere_radius_and_ends(orc):
    assert abs(4.0 / 3.0 * math.pi * orc.sphere_radius() ** 3 - 1.0) < 1e-15
    v = orc.sphere_volume([-R_UNIT - 1e-3, -R_UNIT, 0.0, R_UNIT, R_UNIT + 1e-3])
    assert v[0] == 0.0 and v[1] <= 1e-30 and abs(v[3] - 1.0) <= 2e-16 and v[4] == 1.0
    assert abs(v[2] - 0.5) < 1e-15
    d = orc.sphere_offset([0.0, 0.5, 1.0])
    assert abs(d[0] + R_UNIT) <= 2e-16 and abs(d[1]) < 1e-15 and abs(d[2] - R_UNIT) <= 2e-16
    assert d[0] == -d[2]


@pytest.mark.filterwarnings("ignore::UserWarning")
def test_sphere_volume_is_integral_of_slices(orc):
    integrate = pytest.importorskip("scipy.integrate")
    r = R_UNIT
    ds = np.linspace(-r, r, 41)[1:-1]
    got = orc.sphere_volume(ds)
    for d, g in zip(ds, got):
        want, err = integrate.quad(lambda z: math.pi * (r * r - z * z), -r, d, epsabs=1e-15,
                                   epsrel=1e-14)
        assert abs(g - want) <= 1e-14, (d, g, want)


def test_sphere_symmetry_and_slope(orc):
    rng = np.random.default_rng(71)
    d = rng.uniform(-R_UNIT, R_UNIT, 2000)
    v1, v2 = orc.sphere_volume(d), orc.sphere_volume(-d)
    assert np.abs(v1 + v2 - 1.0).max() <= 1e-15
    h = 1e-6
    fd = (orc.sphere_volume(d + h) - orc.sphere_volume(d - h)) / (2 * h)
    inner = np.abs(d) < R_UNIT - 2 * h
    np.testing.assert_allclose(fd[inner], math.pi * (R_UNIT ** 2 - d[inner] ** 2), atol=1e-8)


def test_sphere_inverse_matches_paper_closed_form(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(72)
    V0 = np.concatenate([rng.uniform(0, 1, 300), [1e-12, 1e-6, 0.25, 0.5 - 1e-9, 0.75,
                                                  1 - 1e-6, 1 - 1e-12]])
    got = orc.sphere_offset(V0)
    for v, g in zip(V0, got):
        v = mpmath.mpf(float(v))
        # Sec. 3: d0 = (6/pi)^(1/3) sin(pi/6 - atan2(2 sqrt(V0 - V0^2), 2 V0 - 1) / 3)
        want = mpmath.cbrt(6 / mpmath.pi) * mpmath.sin(
            mpmath.pi / 6 - mpmath.atan2(2 * mpmath.sqrt(v - v * v), 2 * v - 1) / 3)
        assert abs(g - float(want)) <= 2e-16 * max(1.0, abs(float(want))) + 1e-16, (v, g, want)
    rt = orc.sphere_volume(got)
    assert np.abs(rt - V0).max() <= 8e-16        # 4 ulp at 1


# ---------------------------------------------------------------------------
# Appendix B: centre-of-mass normal
# ---------------------------------------------------------------------------
def _read_gold(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_cm_normal_matches_printed_sums(orc):
    rng = np.random.default_rng(73)
    axis = {"x": 0, "y": 1, "z": 2}
    rows = _read_gold("d3q27_gradient_sums.txt")
    for _ in range(50):
        s = rng.uniform(0, 1, 27)
        g = np.zeros(3)
        for comp, sign, *idx in rows:
            g[axis[comp]] += (1 if sign == "+" else -1) * sum(s[int(i)] for i in idx)
        np.testing.assert_allclose(orc.cm_normal(s), -g / np.linalg.norm(g), rtol=0, atol=1e-13)
    assert orc.cm_normal(np.full(27, 0.3)) is None


def test_cm_normal_linear_field_exact(orc):
    e = orc.d3q27().astype(float)
    rng = np.random.default_rng(74)
    for _ in range(20):
        a = rng.standard_normal(3)
        s = 0.5 + 0.05 * (e @ a)
        np.testing.assert_allclose(orc.cm_normal(s), -a / np.linalg.norm(a), atol=1e-14)


def test_normal_batch_matches_single(orc):
    phi = synth.fill_spheres((24, 24, 24), [(11.6, 12.3, 11.9, 7.4)]).numpy()
    idx = orc.interface_cells(phi)
    e = orc.d3q27()
    nz, ny, nx = phi.shape
    for flags, single in ((0, orc.py_normal), (orc.NORMAL_CM, orc.cm_normal)):
        n = orc.normals(phi, idx, flags)
        for k in range(0, idx.size, max(1, idx.size // 40)):
            c = idx[k]
            x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
            s = np.array([phi[z + v[2], y + v[1], x + v[0]] for v in e], float)
            np.testing.assert_allclose(n[:, k], single(s), atol=1e-15)


# ---------------------------------------------------------------------------
# Sec. 4.2: neighbour-normal variant
# ---------------------------------------------------------------------------
def _stencil(phi, e, x, y, z):
    return np.array([phi[z + v[2], y + v[1], x + v[0]] for v in e], float)


def test_neighbour_normal_with_centre_normals_is_eq36(orc):
    phi = synth.fill_spheres((24, 24, 24), [(11.6, 12.3, 11.9, 7.4)]).numpy()
    idx = orc.interface_cells(phi)
    e = orc.d3q27()
    nz, ny, nx = phi.shape
    for c in idx[:: max(1, idx.size // 30)]:
        x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
        s = _stencil(phi, e, x, y, z)
        n = orc.py_normal(s)
        nn = np.tile(n, (27, 1))
        for pf in (0, orc.POINT_CENTROID):
            k0, d0, p0 = orc.curvature_cell(s, pf)
            k1, d1, p1 = orc.curvature_cell(s, pf | orc.NEIGHBOR_NORMAL, nn=nn)
            assert abs(k1 - k0) <= 1e-12 * max(1.0, abs(k0)) and d1 == d0 and p1 == p0


def test_neighbour_normal_batch_matches_numpy_gather(orc):
    phi = synth.fill_spheres((20, 22, 24), [(9.6, 10.3, 11.9, 6.4)]).numpy()
    idx = orc.interface_cells(phi)
    e = orc.d3q27()
    nz, ny, nx = phi.shape
    for flags in (orc.NEIGHBOR_NORMAL, orc.NEIGHBOR_NORMAL | orc.NORMAL_CM):
        kb, _, _ = orc.curvature(phi, idx, flags)
        nfun = orc.cm_normal if flags & orc.NORMAL_CM else orc.py_normal
        for k in range(0, idx.size, max(1, idx.size // 25)):
            c = idx[k]
            x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
            s = _stencil(phi, e, x, y, z)
            nn = np.zeros((27, 3))
            for i in range(1, 27):
                xi, yi, zi = x + e[i][0], y + e[i][1], z + e[i][2]
                inside = 1 <= xi <= nx - 2 and 1 <= yi <= ny - 2 and 1 <= zi <= nz - 2
                if 0 < s[i] < 1 and inside:
                    ni = nfun(_stencil(phi, e, xi, yi, zi))
                    if ni is not None:
                        nn[i] = ni
            want, _, _ = orc.curvature_cell(s, flags, nn=nn)
            assert abs(kb[k] - want) <= 1e-12 * max(1.0, abs(want))


def test_neighbour_normal_planar_and_spheres(orc):
    # planar field with a normal for which the PY normal is exact by symmetry:
    # every neighbour normal equals the centre normal, kappa = 0
    n = np.array([0.0, -0.5 ** 0.5, 0.5 ** 0.5])
    e = 14
    c = np.array([e / 2, e / 2, e / 2])
    g = np.stack(np.meshgrid(np.arange(e), np.arange(e), np.arange(e), indexing="ij"), -1)[..., ::-1]
    dist = (g - c) @ n
    phi = orc.volume(np.full(dist.size, n[0]), np.full(dist.size, n[1]), np.full(dist.size, n[2]),
                     -dist.ravel()).reshape(dist.shape).astype(np.float32)
    idx = orc.interface_cells(phi)
    k, _, _ = orc.curvature(phi, idx, orc.NEIGHBOR_NORMAL)
    assert np.abs(k).max() < 1e-6
    for R in (8.0, 16.0):
        e = int(2 * R + 8)
        phi = synth.fill_spheres((e, e, e), [(e / 2 + 0.21, e / 2 - 0.37, e / 2 + 0.11, R)]).numpy()
        idx = orc.interface_cells(phi)
        k0, _, _ = orc.curvature(phi, idx)
        k1, dim, _ = orc.curvature(phi, idx, orc.NEIGHBOR_NORMAL)
        e0 = np.abs(k0 - 1 / R).sum() / (idx.size / R)
        e1 = np.abs(k1 - 1 / R).sum() / (idx.size / R)
        print("R=%g L1 error: centre normal %.4f, neighbour normals %.4f" % (R, e0, e1))
        assert e1 < 0.10 and abs(k1.mean() * R - 1) < 0.03
        assert (dim == 5).mean() > 0.99


def test_neighbour_normal_field_symmetry(orc):
    phi = synth.fill_spheres((18, 18, 18), [(8.7, 9.2, 8.9, 5.3)]).numpy()
    idx = orc.interface_cells(phi)
    k0, _, _ = orc.curvature(phi, idx, orc.NEIGHBOR_NORMAL)
    nz, ny, nx = phi.shape
    pos = np.stack([idx // (nx * ny), (idx // nx) % ny, idx % nx], 1)   # (z, y, x)
    for perm in ((0, 1, 2), (2, 0, 1), (1, 0, 2)):
        for flip in itertools.product((False, True), repeat=3):
            t = np.transpose(phi, perm)
            p = pos[:, perm].copy()
            for ax in range(3):
                if flip[ax]:
                    t = np.flip(t, ax)
                    p[:, ax] = t.shape[ax] - 1 - p[:, ax]
            t = np.ascontiguousarray(t)
            lin = (p[:, 0] * t.shape[1] + p[:, 1]) * t.shape[2] + p[:, 2]
            order = np.argsort(lin)
            k1, _, _ = orc.curvature(t, lin[order].astype(np.int32), orc.NEIGHBOR_NORMAL)
            np.testing.assert_allclose(k1, k0[order], rtol=1e-9, atol=1e-12)
