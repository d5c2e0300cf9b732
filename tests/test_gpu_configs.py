"""GPU parity on the workloads the benchmark times, element by element against
the oracle, in the launch configurations the benchmark uses.

- Curvature, 256^3 field with 8 spheres R ~ U[6, 40] (seed 3): every one of
  its interface cells, compaction bit-exact, curvature per cell within
  1e-4 max(|kappa_ref|, 1/64).
- Batched curvature, 64 fields with edges from {32, ..., 256} and 1-20
  droplets each (seed 5): every field, with the autotuned launch shape and
  with an eight-lane shape.
- PLIC adjoints, 2^26 FP32 cells of the parity distribution (2 % edge cases):
  2^17 sampled cells against the oracle's area/centroid adjoints.

Curvature cells with a reduced fit are gated like the others (kappa_gate.py:
only cells where the GPU's and the oracle's pivots fall on opposite sides of
the reduction threshold may differ, counted and bounded).
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


def test_curvature_256_all_cells(dev, orc):
    phi, _ = synth.curvature_field(seed=3, edge=256, device=dev)
    p = phi.cpu().numpy()
    ref_idx = orc.interface_cells(p)
    idx, cnt = plic.interface_compact(phi)
    k = int(cnt.item())
    assert k == ref_idx.size and k > 50_000
    np.testing.assert_array_equal(idx[:k].cpu().numpy(), ref_idx)
    kref, dim, npt, cond = orc.curvature(p, ref_idx, with_cond=True)
    # the benchmark's call: the device-side count, the list as compacted
    kap = torch.full((idx.numel(),), 7.0, device=dev)
    plic.curvature(phi, idx, n_iface=idx.numel(), count=cnt, kappa=kap)
    assert torch.all(kap[k:] == 7.0)
    gate_kappa(kap[:k].cpu().numpy(), kref, dim, "256^3, 8 spheres", cond=cond)
    # FP64 fit, and the Young-Laplace epilogue, on the same list
    k64 = plic.curvature(phi, idx[:k].contiguous(), flags=plic.FLAG_FIT_FP64).cpu().numpy()
    gate_kappa(k64, kref, dim, "256^3, FP64 fit", cond=cond)
    dp = plic.laplace_pressure(phi, idx[:k].contiguous(), 0.0728).cpu().numpy()
    np.testing.assert_array_equal(dp, np.float32(2 * 0.0728) * kap[:k].cpu().numpy())


@pytest.fixture(scope="module")
def batch64(dev, orc):
    fields = synth.batched_fields(seed=5, n_fields=64, device=dev)
    args, refs = [], []
    for phi, _ in fields:
        idx, cnt = plic.interface_compact(phi)
        k = int(cnt.item())
        it = idx[:k].contiguous()
        args.append((phi, it, k, torch.full((max(k, 1),), 7.0, device=dev)))
        p = phi.cpu().numpy()
        ri = orc.interface_cells(p)
        assert ri.size == k
        np.testing.assert_array_equal(it.cpu().numpy(), ri)
        refs.append(orc.curvature(p, ri, with_cond=True) if k else
                    (np.zeros(0), np.zeros(0, np.int32), None, np.zeros(0)))
    return args, refs


def _gate_batch(args, refs, label):
    kk = np.concatenate([a[3][:a[2]].cpu().numpy() for a in args if a[2]])
    kr = np.concatenate([r[0] for a, r in zip(args, refs) if a[2]])
    dm = np.concatenate([r[1] for a, r in zip(args, refs) if a[2]])
    cd = np.concatenate([r[3] for a, r in zip(args, refs) if a[2]])
    return gate_kappa(kk, kr, dm, label, cond=cd)


def test_batched_64_fields_autotuned(dev, batch64):
    from paper_2006_12838_gb300 import autotune
    args, refs = batch64
    batch = plic.BatchedFields(args)
    shape, _ = autotune.tune(batch, flags=0, force=True)
    for a in args:
        a[3].fill_(7.0)
    plic.curvature_batched(batch, tuning=shape)
    assert sum(a[2] for a in args) > 1_000_000
    _gate_batch(args, refs, "64 fields, autotuned %s" % (tuple(shape),))


@pytest.mark.parametrize("tuning", [(128, 64, 0, 8), (128, 256, 3, 1)])
def test_batched_64_fields_layouts(dev, batch64, tuning):
    args, refs = batch64
    for a in args:
        a[3].fill_(7.0)
    plic.curvature_batched(args, tuning=tuning)
    _gate_batch(args, refs, "64 fields, tuning %s" % (tuning,))


def test_plic_adjoints_2p26_sampled(dev, orc):
    # the adjoint workload: 2^26 FP32 cells of the parity distribution, the
    # full launch; 2^17 cells sampled at a fixed stride against the oracle
    n_cells = 1 << 26
    t = [torch.empty(n_cells, device=dev) for _ in range(4)]
    for start, c in synth.plic_cells_chunks(n_cells, 4, edge_frac=0.02):
        k = c["V0"].size
        for j in range(3):
            t[j][start:start + k] = torch.from_numpy(c["n"][j]).to(dev, torch.float32)
        t[3][start:start + k] = torch.from_numpy(c["V0"]).to(dev, torch.float32)
    g = torch.randn(n_cells, device=dev, generator=torch.Generator(device=dev).manual_seed(44))
    d0 = plic.offset(*t, method="sz_opt", precision="fp32p")
    gV, gx, gy, gz = plic.offset_backward(t[0], t[1], t[2], d0, g)
    vd, vx, vy, vz = plic.volume_backward(t[0], t[1], t[2], d0, g)
    sel = torch.arange(0, n_cells, n_cells >> 17, device=dev)
    f = lambda x: x[sel].cpu().numpy().astype(np.float64)  # noqa: E731
    nx, ny, nz, dd, gg = f(t[0]), f(t[1]), f(t[2]), f(d0), f(g)
    rV, rx, ry, rz = orc.offset_grad(nx, ny, nz, dd, gg)
    sd, sx, sy, sz = orc.volume_grad(nx, ny, nz, dd, gg)
    A, *_ = orc.area_centroid(nx, ny, nz, dd)
    V0s = f(t[3])
    # dd0/dV0 = |n|/A grows without bound as the cut area A -> 0 (V0 -> 0 or 1,
    # and the edge cases' corners): there the relative error of A in FP32 is
    # what matters, so g_V0 is gated where A > 0.02 and its sign elsewhere.
    # At V0 in {0, 1} the plane only touches the cube (a face, an edge or a
    # vertex): the derivative is one-sided there; the kernel returns +-inf
    # with the sign of g (the documented convention), checked apart.
    ends = (V0s == 0) | (V0s == 1)
    keep = (A > 0.02) & ~ends
    tol = 2e-4
    # the touching plane's polygon degenerates (a face, an edge or a vertex)
    # and its centroid is a one-sided limit: the normal and volume adjoints
    # are gated on 0 < V0 < 1 and required finite at the ends
    inner = ~ends
    for name, a, b, mask in (("g_V0", f(gV), rV, keep), ("g_nx", f(gx), rx, inner),
                             ("g_ny", f(gy), ry, inner), ("g_nz", f(gz), rz, inner),
                             ("vol g_d0", f(vd), sd, inner), ("vol g_nx", f(vx), sx, inner),
                             ("vol g_ny", f(vy), sy, inner), ("vol g_nz", f(vz), sz, inner)):
        m = mask
        assert np.all(np.isfinite(a[ends])) or name == "g_V0", name
        fin = np.isfinite(b) & m
        rel = np.abs(a - b)[fin] / np.maximum(np.abs(b[fin]), np.abs(gg[fin]))
        print("%s: cells %d, max rel %.3e, p99.9 %.3e" % (name, fin.sum(), rel.max(), np.percentile(rel, 99.9)))
        assert rel.max() <= tol, name
    a = f(gV)
    small = ~keep & ~ends & np.isfinite(rV) & (rV != 0)
    assert np.all(np.sign(a[small]) == np.sign(rV[small]))
    assert ends.sum() > 0
    assert np.all(np.isinf(a[ends]) & (np.sign(a[ends]) == np.sign(gg[ends])))


def test_pipe_probes_run(dev):
    # the probes of the compute rooflines: positive rates of the right order
    # (FP32 FMA: 128 lanes per SM, at most the maximum clock)
    sink = torch.zeros(1, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rates = {}
    for kind in plic.PROBES:
        ops = plic.pipe_probe(kind, 64, sink)          # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ops = plic.pipe_probe(kind, 2048, sink)
        b.record()
        torch.cuda.synchronize()
        rates[kind] = ops / (a.elapsed_time(b) / 1e3)
    print({k: "%.3g" % v for k, v in rates.items()})
    assert 0.2 * sms * 128 * 1.0e9 < rates["ffma"] <= 1.05 * sms * 128 * 2.2e9
    assert rates["ffma2"] >= 0.8 * rates["ffma"]
    assert all(v > 0 for v in rates.values())
    assert float(sink.item()) == 0.0


def test_read_probe_runs(dev):
    # the plain streaming read of the memory rooflines: a 256 MiB buffer (twice
    # the L2) at a positive rate below twice the nominal HBM bandwidth; odd
    # lengths take the tail loads
    sink = torch.zeros(1, device=dev)
    for n in (1 << 26, (1 << 20) + 3, 1, 5):
        buf = torch.rand(n, device=dev)
        plic.read_probe(buf, sink)
        torch.cuda.synchronize()
    buf = torch.rand(1 << 26, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    plic.read_probe(buf, sink)
    b.record()
    torch.cuda.synchronize()
    gbs = buf.numel() * 4 / (a.elapsed_time(b) / 1e3) / 1e9
    print("read probe %.0f GB/s" % gbs)
    assert 500.0 < gbs < 16000.0
    assert float(sink.item()) == 0.0
