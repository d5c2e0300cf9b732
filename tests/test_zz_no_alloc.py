"""The allocation-free compaction entry point, called through the C ABI.

vof_interface_compact_noalloc serves callers that cannot allocate device
memory themselves (a simulation that owns the whole GPU through its own pool,
a real-time loop or callback where cudaMalloc is not allowed).  It must give
exactly the list and count of vof_interface_compact (index work: bit-exact),
also on a second call in a row that reuses the library's built-in scratch,
and the list must be the oracle's interface set.  Fields of more than 4096
tiles take the path with a separate scan launch, which is covered too.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LIMIT = 1 << 28          # PLIC_NOALLOC_MAX_CELLS


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_12838_gb300 import build, plic
    build.build()
    return plic.load()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _compact_both(lib, phi, orc=None):
    """Both entry points on one field; returns the count.  The list and count
    must agree bit for bit, and with the oracle's interface set if given."""
    from paper_2006_12838_gb300 import plic
    nz, ny, nx = phi.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = phi.numel()
    ws = torch.empty(plic.workspace_bytes(plic.WS_COMPACT, n), dtype=torch.uint8, device=phi.device)
    idx_a = torch.full((n,), -7, dtype=torch.int32, device=phi.device)
    cnt_a = torch.full((1,), -7, dtype=torch.int64, device=phi.device)
    assert lib.vof_interface_compact(_ptr(phi), nx, ny, nz, _ptr(idx_a), n, _ptr(cnt_a),
                                     _ptr(ws), ws.numel(), stream) == 0
    idx_b = torch.full((n,), -7, dtype=torch.int32, device=phi.device)
    cnt_b = torch.full((1,), -7, dtype=torch.int64, device=phi.device)
    assert lib.vof_interface_compact_noalloc(_ptr(phi), nx, ny, nz, _ptr(idx_b), n,
                                             _ptr(cnt_b), stream) == 0
    torch.cuda.synchronize()
    k = int(cnt_a.item())
    assert int(cnt_b.item()) == k
    assert torch.equal(idx_a[:k], idx_b[:k])
    if orc is not None:
        ref = orc.interface_cells(phi.cpu().numpy())
        assert ref.size == k
        assert np.array_equal(idx_b[:k].cpu().numpy(), ref)
    return k


def _tiles(nx, ny, nz):
    # whole x-rows per tile: as many as fit in 8192 cells (at least one)
    r = max(1, min(8192 // nx, 4096))
    return -(-(ny * nz) // r)


def test_noalloc_matches_workspace_version_twice(lib, orc):
    from paper_2006_12838_gb300 import synth
    dev = torch.device("cuda:0")
    big, _ = synth.curvature_field(seed=3, edge=160, n_spheres=6, rmin=6, rmax=30, device=dev)
    rng = np.random.default_rng(5)
    small = torch.tensor(rng.random((37, 29, 41)).astype(np.float32), device=dev)
    small[small < 0.3] = 0.0
    k1 = _compact_both(lib, big, orc)      # first call: large field fills many tiles
    k2 = _compact_both(lib, small, orc)    # second call in a row: fewer tiles, stale scratch beyond
    assert k1 > 1000 and k2 > 100


def test_noalloc_beyond_4096_tiles_twice(lib, orc):
    # 512 x 256 x 320 cells (about 42 M, 168 MB): 5120 tiles, so the per-tile
    # counts go through the separate scan launch, and the write pass re-reads
    # the field (the built-in scratch keeps no interface bits)
    dev = torch.device("cuda:0")
    nz, ny, nx = 320, 256, 512
    assert _tiles(nx, ny, nz) > 4096
    g = torch.Generator(device=dev)
    g.manual_seed(17)
    phi = torch.rand((nz, ny, nx), device=dev, generator=g)
    phi[phi < 0.45] = 0.0
    phi[phi > 0.55] = 1.0
    k1 = _compact_both(lib, phi, orc)
    phi2 = phi[:, :, :480].contiguous()       # second call: a narrower field, 4800 tiles
    assert _tiles(480, ny, nz) > 4096
    k2 = _compact_both(lib, phi2, orc)
    assert k1 > 1_000_000 and k2 > 1_000_000


def test_noalloc_size_limit(lib):
    P = ctypes.c_void_p
    dev = torch.device("cuda:0")
    cnt = torch.full((1,), -7, dtype=torch.int64, device=dev)
    # 2^28 + 1 = 17 x 15790321 cells: one cell over the limit, refused before any launch
    st = lib.vof_interface_compact_noalloc(P(256), 17, 15790321, 1, P(256), 10, _ptr(cnt), None)
    assert st == 1
    assert b"limit" in lib.plic_last_error()
    # exactly 2^28 cells (1 GiB) is accepted: a field of zeros with three
    # interior interface cells
    nz, ny, nx = 1024, 512, 512
    assert nz * ny * nx == LIMIT
    phi = torch.zeros((nz, ny, nx), device=dev)
    cells = [(1, 1, 1), (500, 300, 7), (1022, 510, 510)]
    for z, y, x in cells:
        phi[z, y, x] = 0.5
    phi[0, 5, 5] = 0.5                         # boundary layer: not a curvature cell
    idx = torch.full((8,), -7, dtype=torch.int32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.vof_interface_compact_noalloc(_ptr(phi), nx, ny, nz, _ptr(idx), 8, _ptr(cnt),
                                             stream) == 0
    torch.cuda.synchronize()
    assert int(cnt.item()) == 3
    want = sorted(x + nx * (y + ny * z) for z, y, x in cells)
    assert idx[:3].cpu().tolist() == want
    assert idx[3:].cpu().tolist() == [-7] * 5
