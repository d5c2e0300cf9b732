"""GPU parity of the plane-sphere kernels (Sec. 3) against the oracle.

Inputs: V0 ~ U[0, 1] plus the ends, values within 1e-30..1e-3 of 0 and 1,
and invalid values; d0 ~ U[-1.1 r, 1.1 r].  Gates: |d0 - d0_ref| <= 2e-7 (FP32)
and 2e-15 (FP64) absolute (the FP32 bound is 3 ulp of r; the kernel's FP32
Newton root is within 1e-7 of u in units of r); volume within 4 ulp of 1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2006_12838_gb300 import plic  # noqa: E402

R = (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_12838_gb300 import build
    build.build()
    plic.load()
    return torch.device("cuda:0")


def _V0(m, seed):
    rng = np.random.default_rng(seed)
    tiny = np.logspace(-30, -3, 200)
    return np.concatenate([rng.uniform(0, 1, m), [0.0, 0.5, 1.0], tiny, 1 - tiny,
                           0.5 + rng.uniform(-1e-6, 1e-6, 50)])


@pytest.mark.parametrize("precision", ["fp32", "fp32p", "fp64", "fp64r"])
def test_sphere_offset_parity(dev, orc, precision):
    dt = torch.float64 if precision.startswith("fp64") else torch.float32
    npd = np.float64 if dt == torch.float64 else np.float32
    V0 = _V0(1 << 20, 81).astype(npd)
    ref = orc.sphere_offset(V0.astype(np.float64))
    d0 = plic.sphere_offset(torch.tensor(V0, device=dev), precision=precision).cpu().numpy()
    err = np.abs(d0.astype(np.float64) - ref)
    print("%s sphere offset max|dd0| %.3e" % (precision, err.max()))
    assert err.max() <= (2e-15 if dt == torch.float64 else 2e-7)
    # the two ends are mirror images
    i0 = np.flatnonzero(V0 == 0.0)
    i1 = np.flatnonzero(V0 == 1.0)
    assert np.all(d0[i0] == -d0[i1])


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_sphere_volume_parity_and_round_trip(dev, orc, dt):
    npd = np.float64 if dt == torch.float64 else np.float32
    rng = np.random.default_rng(82)
    d = rng.uniform(-1.1 * R, 1.1 * R, 1 << 20).astype(npd)
    ref = orc.sphere_volume(d.astype(np.float64))
    V = plic.sphere_volume(torch.tensor(d, device=dev)).cpu().numpy().astype(np.float64)
    tol = 1e-15 if dt == torch.float64 else 4e-7
    assert np.abs(V - ref).max() <= tol
    assert np.all(V[d <= -R] == 0.0) and np.all(V[d >= R] == 1.0)
    # round trip V0 -> d0 -> V0
    V0 = _V0(1 << 20, 83).astype(npd)
    t = torch.tensor(V0, device=dev)
    back = plic.sphere_volume(plic.sphere_offset(t)).cpu().numpy().astype(np.float64)
    rt = np.abs(back - V0)
    print("%s sphere round trip max %.3e" % (dt, rt.max()))
    assert rt.max() <= (4e-15 if dt == torch.float64 else 4e-7)


def test_sphere_invalid_and_ragged(dev, orc):
    bad = torch.tensor([-0.1, 1.5, float("nan"), 0.3], device=dev)
    d = plic.sphere_offset(bad).cpu().numpy()
    assert np.isnan(d[:3]).all() and np.isfinite(d[3])
    v = plic.sphere_volume(torch.tensor([float("nan"), -5.0, 5.0], device=dev)).cpu().numpy()
    assert np.isnan(v[0]) and v[1] == 0.0 and v[2] == 1.0
    # ragged lengths and a misaligned start (scalar path)
    V0 = np.random.default_rng(84).uniform(0, 1, 1031).astype(np.float32)
    base = torch.tensor(np.concatenate([[0.5], V0]), device=dev)
    for n in (1, 3, 5, 1030):
        a = plic.sphere_offset(base[1:1 + n].clone()).cpu().numpy()     # fresh, aligned
        b = plic.sphere_offset(base[1:1 + n]).cpu().numpy()      # offset by 4 bytes
        np.testing.assert_array_equal(a, b)
        ref = orc.sphere_offset(V0[:n].astype(np.float64))
        assert np.abs(a - ref).max() <= 2e-7


def test_sphere_full_size_sampled(dev, orc):
    """2^28 FP32 cells in the bench's launch configuration; 2^16 sampled."""
    N = 1 << 28
    g = torch.Generator(device=dev)
    g.manual_seed(85)
    V0 = torch.rand(N, device=dev, generator=g)
    d0 = plic.sphere_offset(V0)
    idx = torch.randint(0, N, (1 << 16,), device=dev, generator=g)
    v = V0[idx].cpu().numpy().astype(np.float64)
    ref = orc.sphere_offset(v)
    err = np.abs(d0[idx].cpu().numpy().astype(np.float64) - ref)
    assert err.max() <= 2e-7
    back = plic.sphere_volume(d0)
    assert (back - V0).abs().max().item() <= 4e-7
