"""GPU parity on the throughput workload's adversarial cells and at full size.

- Vertex cells: the plane passes within 1e-6 of a cube vertex, i.e. at the
  boundaries of the five intersection cases (Sec. 2.2); V0 is computed by the
  oracle's forward volume from the same float/double inputs.
- Full size: 2^28 FP32 cells in the bench's launch configuration, compared
  with the oracle on a sample of outputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2006_12838_gb300 import plic, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_12838_gb300 import build
    build.build()
    plic.load()
    return torch.device("cuda:0")


def _inputs(orc, m, seed, dtype, vertex_frac):
    c = synth.plic_cells(m, seed=seed, vertex_frac=vertex_frac)
    npd = np.float32 if dtype == torch.float32 else np.float64
    n = c["n"].astype(npd).astype(np.float64)
    V0 = c["V0"].copy()
    vm = c["vertex"]
    V0[vm] = orc.volume(n[0][vm], n[1][vm], n[2][vm], c["d0_vertex"][vm].astype(npd).astype(np.float64))
    V0 = V0.astype(npd).astype(np.float64)
    return n, V0, vm


def _report(tag, err, n, V0, ref, d0, k=5):
    worst = np.argsort(err)[::-1][:k]
    print("%s max %.3e p99.99 %.3e" % (tag, err.max(), np.percentile(err, 99.99)))
    for i in worst:
        print("   n=(%.9g, %.9g, %.9g) V0=%.9g d0=%.9g ref=%.12g" % (n[0][i], n[1][i], n[2][i], V0[i], d0[i], ref[i]))


@pytest.mark.parametrize("method", list(plic.METHODS))
@pytest.mark.parametrize("precision", ["fp32p", "fp64", "fp64r"])
def test_vertex_cells(dev, orc, method, precision):
    dtype = torch.float64 if precision.startswith("fp64") else torch.float32
    n, V0, vm = _inputs(orc, 1 << 20, 12, dtype, 0.5)
    ref = orc.offset(n[0], n[1], n[2], V0)
    t = [torch.tensor(a, dtype=dtype, device=dev) for a in (n[0], n[1], n[2], V0)]
    d0t = plic.offset(*t, method=method, precision=precision)
    d0 = d0t.cpu().numpy().astype(np.float64)
    err = np.abs(d0 - ref)
    _report("%s %s vertex-cells" % (method, precision), err, n, V0, ref, d0)
    Vb = plic.volume(t[0], t[1], t[2], d0t).cpu().numpy().astype(np.float64)
    rt = np.abs(Vb - V0)
    print("   round trip max %.3e" % rt.max())
    tol = 1e-12 if precision.startswith("fp64") else 2e-6
    assert err.max() <= tol
    if precision == "fp32p":
        assert rt.max() <= 1e-6


def test_full_size_sampled(dev, orc):
    """2^28 FP32 cells, SZ-opt with polish (the bench's headline call), 10 %
    vertex cells; 2^17 sampled outputs against the oracle."""
    N = 1 << 28
    t = [torch.empty(N, dtype=torch.float32, device=dev) for _ in range(4)]
    rng = np.random.default_rng(99)
    samp = []
    for start, c in synth.plic_cells_chunks(N, 2, vertex_frac=0.1):
        k = c["V0"].size
        n = c["n"].astype(np.float32).astype(np.float64)
        V0 = c["V0"].copy()
        vm = c["vertex"]
        V0[vm] = orc.volume(n[0][vm], n[1][vm], n[2][vm],
                            c["d0_vertex"][vm].astype(np.float32).astype(np.float64))
        for j in range(3):
            t[j][start:start + k] = torch.from_numpy(n[j].astype(np.float32))
        t[3][start:start + k] = torch.from_numpy(V0.astype(np.float32))
        # sample: 2048 random cells per chunk, all of them vertex cells for half
        pick = np.concatenate([rng.choice(k, 1024, replace=False),
                               rng.choice(np.flatnonzero(vm), 1024, replace=False)])
        samp.append((start + pick, n[:, pick], V0.astype(np.float32).astype(np.float64)[pick]))
    d0 = plic.offset(*t, method="sz_opt", precision="fp32p")
    Vb = plic.volume(t[0], t[1], t[2], d0)
    # the fused round trip (the bench's step) gives the same d0 and a V0_rt
    # within the rounding of two FP32 evaluations of plic_volume's
    d0f, vrt = plic.offset_roundtrip(*t, method="sz_opt", precision="fp32p")
    assert torch.equal(d0f, d0)
    assert (vrt - Vb).abs().max().item() <= 5e-7
    assert (vrt - t[3]).abs().max().item() <= 1e-6
    del d0f, vrt
    idx = np.concatenate([s[0] for s in samp])
    nn = np.concatenate([s[1] for s in samp], axis=1)
    VV = np.concatenate([s[2] for s in samp])
    ref = orc.offset(nn[0], nn[1], nn[2], VV)
    it = torch.tensor(idx, device=dev)
    got = d0[it].cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    _report("full-size sampled", err, nn, VV, ref, got)
    rt = (Vb - t[3]).abs()
    print("full-size round trip max %.3e mean %.3e" % (rt.max().item(), rt.double().mean().item()))
    assert err.max() <= 2e-6
    assert rt.max().item() <= 1e-6
