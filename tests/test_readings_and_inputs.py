"""Readings of printed constants, and the seeded input generators.

- The FP32 decimals printed in the listings of Sec. 2.3-2.4 are the closed
  forms of Eqs. 13-22 (and pi/6, 4 pi/3, 2^24, FLT_MIN) rounded to FP32; the
  GPU kernels derive their FP32 and FP64 constants from those closed forms.
- The generators are deterministic for a seed and hold the recipe's shapes.
"""
import math
import os

import numpy as np

from paper_2006_12838_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_listing_constants_are_fp32_roundings_of_closed_forms():
    with open(os.path.join(GOLD, "listing_constants.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for dec, expr in rows:
        exact = eval(expr, {"math": math})
        printed = np.float32(float(dec))
        assert abs(float(printed) - exact) <= 2 * float(np.spacing(np.float32(exact))), (dec, expr)


def test_frame_vector_is_unit():
    with open(os.path.join(GOLD, "frame_r.txt")) as f:
        r = [float(v) for l in f if l.strip() and not l.startswith("#") for v in l.split()]
    assert abs(math.sqrt(sum(v * v for v in r)) - 1.0) < 1e-7


def test_plic_cells_recipe():
    a = synth.plic_cells(20000, seed=1, edge_frac=0.02)
    b = synth.plic_cells(20000, seed=1, edge_frac=0.02)
    np.testing.assert_array_equal(a["n"], b["n"])
    np.testing.assert_array_equal(a["V0"], b["V0"])
    np.testing.assert_allclose(np.linalg.norm(a["n"], axis=0), 1.0, atol=1e-15)
    tail = a["V0"][-400:]
    assert ((tail == 0) | (tail == 1) | (tail == 0.5)).sum() > 80
    c = synth.plic_cells(20000, seed=2, vertex_frac=0.1)
    v = c["vertex"]
    assert abs(v.mean() - 0.1) < 1e-2
    assert np.isnan(c["V0"][v]).all() and not np.isnan(c["V0"][~v]).any()
    # the vertex offsets are n.s/2 + O(1e-6) for a sign pattern s in {+-1}^3
    n = c["n"][:, v].T
    d0 = c["d0_vertex"][v]
    best = np.min(np.stack([np.abs(0.5 * (n * np.array(s)).sum(1) - d0)
                            for s in np.ndindex(2, 2, 2)
                            for s in [tuple(1 - 2 * np.array(s))]]), 0)
    assert best.max() <= 1e-6
    h = 0.5 * np.abs(n).sum(1)
    assert np.all(np.abs(d0) < h)


def test_paper_normals_counts():
    n = synth.paper_normals(4096, seed=6).T
    assert np.allclose(n[0], [1, 0, 0]) and np.allclose(n[1], [0.5 ** 0.5, 0.5 ** 0.5, 0])
    assert np.sum(n[:, 2] == 0) == 512          # 2 special + 510 random 2D
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-15)


def test_fill_fields_exact_quantised():
    phi = synth.fill_spheres((24, 24, 24), [(11.3, 12.6, 11.9, 7.4)]).numpy()
    assert np.all(phi * 4096 == np.round(phi * 4096))
    assert abs(phi.sum() - 4 / 3 * math.pi * (round(7.4 * 32) / 32) ** 3) < 0.5
    p2 = synth.fill_spheres((24, 24, 24), [(11.3, 12.6, 11.9, 7.4), (11.3, 12.6, 11.9, 7.4)]).numpy()
    np.testing.assert_array_equal(phi, p2)       # union with itself
    e = synth.fill_ellipsoid((40, 40, 40), (20, 20, 20), (6, 9, 12)).numpy()
    assert abs(e.sum() - 4 / 3 * math.pi * 6 * 9 * 12) < 1.0


def test_boundary_cells_sit_on_case_boundaries(orc):
    # the throughput workload's boundary cells: the plane through the corner
    # that ends case (2) or starts case (4) / (5), whose volume must equal the
    # closed-form boundary volumes of the configuration (Eq. 10 at d = n2,
    # n3 and n1 + n2)
    from paper_2006_12838_gb300 import synth
    c = synth.plic_cells(40_000, seed=2, edge_frac=0.02, boundary_frac=0.1)
    b = c["boundary"]
    assert 0.08 < b.mean() < 0.12 and not b[-800:].any()
    n = c["n"][:, b]
    Vb = orc.volume(n[0], n[1], n[2], c["d0_boundary"][b])
    n1, n2, n3 = np.sort(np.abs(n), 0)
    V23 = (3 * n2 ** 2 - 3 * n1 * n2 + n1 ** 2) / (6 * n2 * n3)
    V34 = (n3 ** 3 - (n3 - n1) ** 3 - (n3 - n2) ** 3) / (6 * n1 * n2 * n3)
    V35 = (n1 + n2) / (2 * n3)
    other = np.where(n3 >= n1 + n2, V35, V34)
    at23 = np.abs(Vb - V23) < 1e-12
    assert np.all(at23 | (np.abs(Vb - other) < 1e-12))
    assert 0.4 < at23.mean() < 0.6
    V0 = synth.boundary_fill(Vb, c["dV"][b], c["mirror"][b])
    V = np.minimum(V0, 1 - V0)
    assert np.all(np.abs(V - np.clip(Vb, 0, 0.5)) <= 1e-6 + 1e-15)
