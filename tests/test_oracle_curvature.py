"""Pins for the oracle's curvature step (Sec. 4.2, Appendix B).

- D3Q27 order against the gradient sums printed in Appendix B (golden file).
- Parker-Youngs normal of a linear field is exact (the weighted direction
  tensor sum_i w_i e_i e_i^T is isotropic for the weights of Eq. 38).
- Least squares against exact paraboloid samples and numpy.linalg.lstsq.
- Eq. 42 against 2H = div(grad f / sqrt(1 + |grad f|^2)) by central
  differences (an independent form of the Monge-patch mean curvature).
- Whole step: planar fields give kappa = 0; spheres and cylinders give
  kappa -> 1/R and 1/(2R); kappa is invariant under the 48 cube symmetries.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2006_12838_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_gold(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_d3q27_matches_appendix_b_gradient_sums(orc):
    e = orc.d3q27()
    assert (e[0] == 0).all()
    assert len({tuple(v) for v in e}) == 27
    axis = {"x": 0, "y": 1, "z": 2}
    for comp, sign, *idx in _read_gold("d3q27_gradient_sums.txt"):
        want = sorted(int(i) for i in idx)
        s = 1 if sign == "+" else -1
        got = sorted(i for i in range(1, 27) if e[i, axis[comp]] == s)
        assert got == want, (comp, sign, got, want)


def test_py_weights_golden_and_linear_field_exact(orc):
    e = orc.d3q27()
    wt = {int(a): float(b) for a, b in _read_gold("py_weights.txt")}
    T = sum(wt[int((v * v).sum())] * np.outer(v, v) for v in e[1:])
    np.testing.assert_allclose(T, T[0, 0] * np.eye(3), atol=1e-12)
    rng = np.random.default_rng(41)
    for _ in range(50):
        a = rng.standard_normal(3)
        phi27 = 0.5 + 0.1 * (e @ a)
        n = orc.py_normal(phi27)
        np.testing.assert_allclose(n, -a / np.linalg.norm(a), atol=1e-14)
    assert orc.py_normal(np.full(27, 0.3)) is None


def test_lsq_exact_and_lstsq(orc):
    rng = np.random.default_rng(42)
    for _ in range(30):
        x5 = rng.standard_normal(5)
        m = rng.integers(5, 27)
        px, py = rng.uniform(-1.7, 1.7, (2, m))
        Q = np.stack([px * px, py * py, px * py, px, py], 1)
        pz = Q @ x5
        got, dim = orc.lsq_paraboloid(px, py, pz)
        assert dim == 5
        np.testing.assert_allclose(got, x5, atol=1e-10)
        pzn = pz + 0.01 * rng.standard_normal(m)
        got, dim = orc.lsq_paraboloid(px, py, pzn)
        ref = np.linalg.lstsq(Q, pzn, rcond=None)[0]
        np.testing.assert_allclose(got, ref, atol=1e-9)
    # reduced dimension (Appendix B): m < 5 points fit the leading m parameters
    for m in (1, 2, 3, 4):
        px, py = rng.uniform(-1.5, 1.5, (2, m))
        pz = rng.standard_normal(m)
        Q = np.stack([px * px, py * py, px * py, px, py], 1)[:, :m]
        got, dim = orc.lsq_paraboloid(px, py, pz)
        assert dim == m
        np.testing.assert_allclose(got[:m], np.linalg.solve(Q, pz), rtol=1e-8, atol=1e-9)
        assert (got[m:] == 0).all()
    assert orc.lsq_paraboloid([], [], [])[1] == 0


def test_eq42_against_divergence_form(orc):
    rng = np.random.default_rng(43)
    h = 1e-5
    for _ in range(40):
        A, B, C, H, I = rng.standard_normal(5)

        def field(x, y):
            fx = 2 * A * x + C * y + H
            fy = 2 * B * y + C * x + I
            s = np.sqrt(1 + fx * fx + fy * fy)
            return fx / s, fy / s

        div = ((field(h, 0)[0] - field(-h, 0)[0]) + (field(0, h)[1] - field(0, -h)[1])) / (2 * h)
        assert abs(orc.paraboloid_kappa([A, B, C, H, I]) - 0.5 * div) <= 1e-7 * (1 + abs(div))
    # sphere cap z = (x^2 + y^2) / (2R): mean curvature 1/R
    assert abs(orc.paraboloid_kappa([1 / 8, 1 / 8, 0, 0, 0]) - 0.25) < 1e-15


def _planar_field(orc, n, shape=(9, 9, 9), d0c=0.13):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(*(np.arange(k, dtype=float) for k in shape), indexing="ij")
    c = np.array([nx // 2, ny // 2, nz // 2], float)
    d = d0c - (n[0] * (x - c[0]) + n[1] * (y - c[1]) + n[2] * (z - c[2]))
    return orc.volume(n[0], n[1], n[2], d.ravel()).reshape(shape).astype(np.float32)


@pytest.mark.parametrize("n", [(1, 0, 0), (0, -1, 0), (0, 0, 1),
                               (0.5 ** 0.5, 0.5 ** 0.5, 0), (0, -0.5 ** 0.5, 0.5 ** 0.5),
                               (0.5 ** 0.5, 0, -0.5 ** 0.5)])
def test_planar_fields_give_zero_curvature(orc, n):
    n = np.array(n, float)
    phi = _planar_field(orc, n)
    idx = orc.interface_cells(phi)
    assert idx.size > 0
    for flags in (0, orc.POINT_CENTROID):
        kappa, dim, npt = orc.curvature(phi, idx, flags)
        assert np.all(np.abs(kappa) < 1e-6), kappa
    # the Parker-Youngs normal is exact on these symmetric planar stencils
    e = orc.d3q27()
    nz, ny, nx = phi.shape
    for c in idx[:5]:
        x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
        s = np.array([phi[z + v[2], y + v[1], x + v[0]] for v in e], float)
        # the field is a function of n.x with fill increasing against n
        np.testing.assert_allclose(orc.py_normal(s), n, atol=1e-6)


def test_spheres_and_cylinders(orc):
    # Mean curvature: 1/R for a sphere, 1/(2R) for a cylinder (kappa1 + kappa2
    # = 2/R and 1/R).  On exactly sub-sampled fills the per-cell scatter grows
    # with R (as Sec. 4.3 also observes), so the gate is on the mean (within
    # 3 %) and on the L1 error of Sec. 4.3 (Eq. 49) loosely: 10 % for the
    # paper's foot points, 6 % for polygon centroids, up to R = 20.
    for R in (8.0, 20.0):
        e = int(2 * R + 8)
        phi = synth.fill_spheres((e, e, e), [(e / 2 + 0.21, e / 2 - 0.37, e / 2 + 0.11, R)]).numpy()
        idx = orc.interface_cells(phi)
        for flags, gate in ((0, 0.10), (orc.POINT_CENTROID, 0.06)):
            kappa, dim, npt = orc.curvature(phi, idx, flags)
            err = np.abs(kappa - 1 / R).sum() / (idx.size / R)
            assert err < gate, (R, flags, err)
            assert abs(kappa.mean() * R - 1) < 0.03
            assert (dim == 5).mean() > 0.99
    R = 10.0
    phi = synth.fill_cylinder((12, 30, 30), 2, (14.6, 15.3), R).numpy()
    idx = orc.interface_cells(phi)
    kappa, dim, npt = orc.curvature(phi, idx)
    err = np.abs(kappa - 0.5 / R).sum() / (idx.size * 0.5 / R)
    assert err < 0.15, err          # half the sphere's curvature: twice the relative scatter
    assert abs(kappa.mean() * 2 * R - 1) < 0.03
    k2, *_ = orc.curvature(phi, idx, orc.KAPPA_PAPER_SIGN)
    np.testing.assert_array_equal(k2, -kappa)


def test_cube_symmetry_invariance(orc):
    e = orc.d3q27()
    lut = {tuple(v): i for i, v in enumerate(e)}
    phi = synth.fill_spheres((28, 28, 28), [(13.7, 14.2, 13.9, 9.3)]).numpy()
    idx = orc.interface_cells(phi)
    nz, ny, nx = phi.shape
    rng = np.random.default_rng(44)
    for c in rng.choice(idx, 12, replace=False):
        x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
        s = np.array([phi[z + v[2], y + v[1], x + v[0]] for v in e], float)
        k0, dim0, _ = orc.curvature_cell(s)
        if dim0 < 5:
            continue
        for perm in itertools.permutations(range(3)):
            for sg in itertools.product((1, -1), repeat=3):
                S = np.zeros((3, 3))
                for r in range(3):
                    S[r, perm[r]] = sg[r]
                t = np.empty(27)
                for i, v in enumerate(e):
                    t[lut[tuple((S @ v).astype(int))]] = s[i]
                k, dim, _ = orc.curvature_cell(t)
                assert abs(k - k0) <= 1e-9 * max(1.0, abs(k0)), (perm, sg, k, k0)


def test_fd_gradient_consistency(orc):
    phi = synth.fill_spheres((16, 16, 16), [(7.6, 8.1, 7.8, 5.2)]).numpy()
    rng = np.random.default_rng(45)
    p = phi.copy()
    iface = (p > 0) & (p < 1)
    # fills kept in [0.02, 0.98]: near 0 and 1 the offset d0 ~ V^(1/3) bends so
    # fast that an FD step of 1e-4 is no longer in its asymptotic range
    p[iface] = np.clip(p[iface] + 1e-3 * rng.standard_normal(iface.sum()), 0.02, 0.98)
    idx = orc.interface_cells(p)
    w = rng.standard_normal(idx.size)
    g1 = orc.curvature_grad_fd(p, idx, w, 1e-4)
    g2 = orc.curvature_grad_fd(p, idx, w, 5e-5)
    np.testing.assert_allclose(g1, g2, rtol=1e-3, atol=1e-3 * np.abs(g1).max())
    # zero outside the union of the stencils of the curvature cells
    near = np.zeros(p.shape, bool)
    nz, ny, nx = p.shape
    for c in idx:
        x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
        near[z - 1:z + 2, y - 1:y + 2, x - 1:x + 2] = True
    assert np.all(g1[~near] == 0)


def test_fd_gradient_matches_global_difference_quotient(orc):
    """The oracle's curvature gradient against the plain definition of a
    derivative: for a probe cell j, phi_j is moved by +-h in the whole field,
    kappa is recomputed by the curvature oracle on the fixed list, and
    sum_k w_k (kappa_k(+) - kappa_k(-)) is divided by the actual step.  A
    mirrored or shifted scatter offset, or a weight applied to the wrong cell,
    moves the gradient of j to another cell and fails here.  The field is the
    adjoint workload in miniature: an ellipsoid with 1e-3 noise on the
    interface cells, clamped to [2e-4, 1 - 2e-4], so that no probe (an
    interface cell) crosses 0 or 1 under the step."""
    phi, _ = synth.adjoint_field(seed=4, edge=48, semi=(8.0, 11.0, 14.0))
    p = phi.numpy().copy()
    idx = orc.interface_cells(p)
    rng = np.random.default_rng(46)
    w = rng.standard_normal(idx.size)
    h = 1e-6
    g = orc.curvature_grad_fd(p, idx, w, h).ravel()
    nz, ny, nx = p.shape
    offs = np.array([dx + nx * (dy + ny * dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                     for dx in (-1, 0, 1)])
    cover = np.zeros(p.size, np.int64)
    for o in offs:
        np.add.at(cover, idx.astype(np.int64) + o, 1)
    flat = p.ravel()
    iface = (flat > 0) & (flat < 1)
    cand = np.flatnonzero(iface & (cover > 0))
    # cells inside the most overlapping stencils, interface cells inside the
    # fewest, and the corner entries (+-1, +-1, +-1) of listed cells
    dense = cand[np.argsort(-cover[cand], kind="stable")[:20]]
    low = cand[cover[cand] <= np.sort(cover[cand])[40]]
    sparse = rng.choice(low, 15, replace=False)
    corner_off = [dx + nx * (dy + ny * dz) for dz in (-1, 1) for dy in (-1, 1) for dx in (-1, 1)]
    corners = []
    for k in rng.permutation(idx.size):
        j = int(idx[k]) + corner_off[len(corners) % 8]
        if iface[j]:
            corners.append(j)
        if len(corners) == 15:
            break
    probes = np.unique(np.concatenate([dense, sparse, np.array(corners)]))
    assert probes.size >= 45
    assert cover[dense].min() >= 16 and cover[sparse].max() <= 11
    gscale = np.abs(g).max()
    worst = 0.0
    for j in probes:
        q = flat.copy()
        q[j] = np.float32(flat[j] + h)
        sp = float(q[j])
        kp, *_ = orc.curvature(q.reshape(p.shape), idx)
        q[j] = np.float32(flat[j] - h)
        sm = float(q[j])
        km, *_ = orc.curvature(q.reshape(p.shape), idx)
        gq = float(np.dot(w, kp - km)) / (sp - sm)
        rel = abs(gq - g[j]) / max(abs(gq), 1e-3 * gscale)
        worst = max(worst, rel)
        assert rel <= 1e-6, (j, gq, g[j], cover[j])
    print("global difference quotient: %d probes, max rel %.2e" % (probes.size, worst))
