"""GPU parity of interface compaction and curvature against the oracle.

- Compaction is index work: bit-exact (same cells, same ascending order).
- Curvature: |kappa - kappa_ref| <= 1e-4 max(|kappa_ref|, 1/64) per cell for
  the adaptive, FP64 and double-float fits; the FP32 fit is reported with a
  looser gate.  Cells with a reduced fit are gated too (kappa_gate.py);
  stencils built with 1-4 interface neighbours and collinear neighbours
  exercise the reduced and near-singular fits directly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from kappa_gate import gate_kappa  # noqa: E402
from paper_2006_12838_gb300 import plic, synth  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_12838_gb300 import build
    build.build()
    plic.load()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def field(orc):
    phi, _ = synth.curvature_field(seed=3, edge=96, n_spheres=5, rmin=6, rmax=20)
    p = phi.numpy()
    idx = orc.interface_cells(p)
    return p, idx


def _compact(dev, p):
    phid = torch.tensor(p, device=dev)
    idx, cnt = plic.interface_compact(phid)
    k = int(cnt.item())
    return phid, idx[:k].cpu().numpy(), idx, cnt


@pytest.mark.parametrize("shape", [(96, 96, 96), (29, 41, 37), (3, 3, 3), (5, 70, 13), (7, 9, 100),
                                   (5, 6, 260), (6, 5, 4), (4, 33, 8), (3, 17, 516),
                                   # rows of 32 cells (one bit word), of 8192 cells (one row
                                   # per tile) and beyond, a 44-cell row (two words)
                                   (6, 7, 32), (3, 4, 8192), (3, 3, 8196), (3, 40, 44),
                                   # > 4096 tiles: the separate scan launch, with the vector
                                   # loads and with the scalar ones (odd nx), and with rows of
                                   # 30 cells, which keep no bits (the recounting write pass)
                                   (520, 256, 256), (500, 257, 257), (2000, 600, 30),
                                   # rows of more than 512 cells (the count pass cuts them into
                                   # 512-cell segments): two, four and a partial last segment,
                                   # then with the scan launch, then 32 769 tiles (two scan rounds)
                                   (5, 9, 1024), (4, 6, 2048), (7, 5, 1540), (300, 120, 1024),
                                   (3, 10923, 4100),
                                   # the ballot layout of the bits (rows of >= 64 cells, nx % 4
                                   # == 0): one partial chunk, tiles spanning many z planes
                                   # (ny = 5 and 3 with 128 rows per tile), an exact chunk
                                   (40, 5, 64), (9, 11, 68), (130, 3, 64), (6, 50, 128),
                                   # the slot count pass (rows of 128 * 2^k cells) with tiles
                                   # that wrap over several z planes (ny = 3, 5)
                                   (7, 3, 512), (9, 5, 128), (5, 7, 256)])
def test_compaction_bit_exact(dev, orc, shape):
    rng = np.random.default_rng(sum(shape))
    p = rng.random(shape).astype(np.float32)
    p[p < 0.4] = 0.0
    p[p > 0.8] = 1.0
    _, got, _, _ = _compact(dev, p)
    np.testing.assert_array_equal(got, orc.interface_cells(p))


def test_compaction_edge_fields(dev, orc, field):
    p, idx = field
    _, got, _, _ = _compact(dev, p)
    np.testing.assert_array_equal(got, idx)
    for fill in (0.0, 1.0, 0.5):
        q = np.full((17, 18, 19), fill, np.float32)
        _, got, _, _ = _compact(dev, q)
        np.testing.assert_array_equal(got, orc.interface_cells(q))
    # capacity smaller than the count: count is the full count, prefix written
    phid = torch.tensor(p, device=dev)
    small = torch.full((100,), -1, dtype=torch.int32, device=dev)
    _, cnt = plic.interface_compact(phid, idx=small)
    assert int(cnt.item()) == idx.size
    np.testing.assert_array_equal(small.cpu().numpy(), idx[:100])


def _check(kappa, kref, dim, tol, label, cond=None):
    return gate_kappa(kappa, kref, dim, label, tol, cond)


@pytest.mark.parametrize("method", list(plic.METHODS))
def test_curvature_methods_default_fit(dev, orc, field, method):
    p, idx = field
    kref, dim, _, cond = orc.curvature(p, idx, with_cond=True)
    phid = torch.tensor(p, device=dev)
    k = plic.curvature(phid, torch.tensor(idx, device=dev), method=method).cpu().numpy()
    _check(k.astype(np.float64), kref, dim, TOL, method + " adaptive fit", cond)


@pytest.mark.parametrize("fit,tol", [(plic.FLAG_FIT_DF32, TOL), (plic.FLAG_FIT_FP64, TOL),
                                     (plic.FLAG_FIT_FP32, 1e-3)])
def test_curvature_fit_precisions(dev, orc, field, fit, tol):
    p, idx = field
    kref, dim, _, cond = orc.curvature(p, idx, with_cond=True)
    phid = torch.tensor(p, device=dev)
    k = plic.curvature(phid, torch.tensor(idx, device=dev), flags=fit).cpu().numpy()
    _check(k.astype(np.float64), kref, dim, tol, "fit flag %d" % fit, cond)


def test_curvature_flags(dev, orc, field):
    p, idx = field
    phid = torch.tensor(p, device=dev)
    it = torch.tensor(idx, device=dev)
    kref, dim, _, cond = orc.curvature(p, idx, orc.POINT_CENTROID, with_cond=True)
    k = plic.curvature(phid, it, flags=plic.FLAG_POINT_CENTROID).cpu().numpy()
    _check(k.astype(np.float64), kref, dim, TOL, "centroid points", cond)
    k0 = plic.curvature(phid, it)
    k1 = plic.curvature(phid, it, flags=plic.FLAG_KAPPA_PAPER_SIGN)
    assert torch.equal(k0, -k1)


def test_device_count_path_and_sphere(dev, orc):
    R = 14.0
    e = 40
    phi = synth.fill_spheres((e, e, e), [(19.6, 20.3, 19.8, R)])
    phid = phi.to(dev)
    idx, cnt = plic.interface_compact(phid)
    # curvature driven by the device-side count (no host round trip)
    kap = torch.full((idx.numel(),), 7.0, device=dev)
    plic.curvature(phid, idx, n_iface=idx.numel(), count=cnt, kappa=kap)
    k = int(cnt.item())
    assert torch.all(kap[k:] == 7.0)
    kd = kap[:k].cpu().numpy()
    kh = plic.curvature(phid, idx[:k].contiguous()).cpu().numpy()
    np.testing.assert_array_equal(kd, kh)
    assert abs(kd.mean() * R - 1) < 0.03


def test_batched_matches_single(dev, orc):
    fields = synth.batched_fields(seed=5, n_fields=6, edges=(32, 48, 64), device="cpu")
    args, singles = [], []
    for phi, _ in fields:
        phid = phi.to(dev)
        idx, cnt = plic.interface_compact(phid)
        k = int(cnt.item())
        it = idx[:k].contiguous()
        kap = torch.empty(max(k, 1), device=dev)
        args.append((phid, it, k, kap))
        singles.append(plic.curvature(phid, it).cpu().numpy() if k else np.zeros(0, np.float32))
    big = max(range(len(args)), key=lambda i: args[i][2])
    kref, dim, _, cond = orc.curvature(args[big][0].cpu().numpy(), args[big][1].cpu().numpy(), with_cond=True)
    # one thread per cell (the default and lanes_per_cell = 1): the single-field
    # kernel's arithmetic, so the same values
    for tuning in (None, (128, 64, 1), (128, 7, 2), (128, 1000, 0), (128, 96, 0, 1), (128, 32, 3, 0)):
        plic.curvature_batched(args, tuning=tuning)
        for (phid, it, k, kap), s in zip(args, singles):
            np.testing.assert_array_equal(kap[:k].cpu().numpy(), s)
    # eight lanes per cell: other summation orders; against the oracle, per
    # cell, on every field
    refs = [orc.curvature(a[0].cpu().numpy(), a[1].cpu().numpy(), with_cond=True) if a[2] else None
            for a in args]
    for tuning in ((128, 64, 1, 8), (128, 7, 2, 8), (128, 1000, 0, 8)):
        plic.curvature_batched(args, tuning=tuning)
        for j, ((phid, it, k, kap), r) in enumerate(zip(args, refs)):
            if k:
                _check(kap[:k].cpu().numpy().astype(np.float64), r[0], r[1], TOL,
                       "batched, 8 lanes %s, field %d" % (tuning, j), r[3])
    plic.curvature_batched(args)
    phid, it, k, kap = args[big]
    _check(kap[:k].cpu().numpy().astype(np.float64), kref, dim, TOL, "batched", cond)
    # the prepared descriptor table, reused: same values
    batch = plic.BatchedFields(args)
    for _ in range(2):
        for a in args:
            a[3].fill_(7.0)
        plic.curvature_batched(batch)
        for (phid, it, k, kap), s in zip(args, singles):
            np.testing.assert_array_equal(kap[:k].cpu().numpy(), s)


def _stencil_field(stencils):
    """A field of shape (3, 3, 4 S) holding S given 3^3 stencils (arrays
    indexed [dz+1, dy+1, dx+1]) side by side, their centres at x = 4 s + 1,
    y = z = 1, with a spacer column between them; returns (field, centres)."""
    S = len(stencils)
    phi = np.zeros((3, 3, 4 * S), np.float32)
    for s_, st in enumerate(stencils):
        phi[:, :, 4 * s_:4 * s_ + 3] = st
    nx = 4 * S
    return phi, np.array([4 * s_ + 1 + nx * (1 + 3) for s_ in range(S)], np.int32)


def _reduced_stencils(orc, rng):
    """Stencils of a nearly horizontal interface (fluid below) whose set of
    interface neighbours is chosen: 1-4 random neighbours (fits of dimension
    1-4), and collinear or symmetric sets that make the normal matrix
    (nearly) singular."""
    e = orc.d3q27()
    out = []

    def make(sel):
        st = np.zeros((3, 3, 3), np.float32)
        for i in range(1, 27):
            ex, ey, ez = e[i]
            st[ez + 1, ey + 1, ex + 1] = 1.0 if (ez < 0 or (ez == 0 and ex + 2 * ey < 0)) else 0.0
        for i in sel:
            ex, ey, ez = e[i]
            st[ez + 1, ey + 1, ex + 1] = rng.uniform(0.05, 0.95)
        st[1, 1, 1] = rng.uniform(0.2, 0.8)
        return st

    for m in (1, 2, 3, 4):
        for _ in range(25):
            out.append(make(rng.choice(np.arange(1, 27), m, replace=False)))
    lut = {tuple(v): i for i, v in enumerate(e)}
    lines = [[(1, 0, 0), (-1, 0, 0)], [(0, 1, 0), (0, -1, 0)], [(1, 1, 0), (-1, -1, 0)],
             [(1, 0, 0), (-1, 0, 0), (0, 0, 1)], [(1, -1, 0), (1, 0, 0), (1, 1, 0)],
             [(1, -1, 0), (1, 0, 0), (1, 1, 0), (-1, -1, 0), (-1, 0, 0), (-1, 1, 0)],
             [(0, 1, 0), (0, -1, 0), (0, 1, 1), (0, -1, -1), (0, 0, 1)]]
    for ln in lines:
        for _ in range(6):
            out.append(make([lut[v] for v in ln]))
    return out


@pytest.mark.parametrize("fit", [0, plic.FLAG_FIT_FP64, plic.FLAG_FIT_DF32])
def test_reduced_and_near_singular_fits(dev, orc, fit):
    rng = np.random.default_rng(61)
    phi, idx = _stencil_field(_reduced_stencils(orc, rng))
    kref, dim, npt, cond = orc.curvature(phi, idx, with_cond=True)
    print("oracle fit dimensions:", np.bincount(dim, minlength=6))
    for d in (1, 2, 3, 4):
        assert (dim == d).any(), d
    k = plic.curvature(torch.tensor(phi, device=dev), torch.tensor(idx, device=dev),
                       flags=fit).cpu().numpy()
    _check(k.astype(np.float64), kref, dim, TOL, "reduced / near-singular fits, flag %d" % fit, cond)
