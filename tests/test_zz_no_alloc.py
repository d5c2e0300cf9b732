"""The allocation-free compaction entry point, called through the C ABI.

vof_interface_compact_noalloc serves callers that cannot allocate device
memory themselves (a simulation that owns the whole GPU through its own pool,
a real-time loop or callback where cudaMalloc is not allowed).  It must give
exactly the list and count of vof_interface_compact (index work: bit-exact),
also on a second call in a row that reuses the library's built-in scratch.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_12838_gb300 import build, plic
    build.build()
    return plic.load()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _compact_both(lib, phi):
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
    return k


def test_noalloc_matches_workspace_version_twice(lib):
    from paper_2006_12838_gb300 import synth
    dev = torch.device("cuda:0")
    big, _ = synth.curvature_field(seed=3, edge=160, n_spheres=6, rmin=6, rmax=30, device=dev)
    rng = np.random.default_rng(5)
    small = torch.tensor(rng.random((37, 29, 41)).astype(np.float32), device=dev)
    small[small < 0.3] = 0.0
    k1 = _compact_both(lib, big)      # first call: large field fills many tiles
    k2 = _compact_both(lib, small)    # second call in a row: fewer tiles, stale scratch beyond
    assert k1 > 1000 and k2 > 100


def test_noalloc_rejects_fields_beyond_limit(lib):
    P = ctypes.c_void_p
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    # 2^28 + 4096 cells: one tile over the limit; rejected before any launch
    st = lib.vof_interface_compact_noalloc(P(256), 4096, 4096, 16 + 1, P(256), 10, _ptr(cnt), None)
    assert st == 1
    assert b"limit" in lib.plic_last_error()
