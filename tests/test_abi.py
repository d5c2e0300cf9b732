"""The C ABI library: it builds, loads, exports every symbol that
``include/plic.h`` declares, and validates arguments on the host (these calls
return before any CUDA work, so they run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2006_12838_gb300 import build as B
from paper_2006_12838_gb300 import plic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plic.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return plic.load()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:plic_status|size_t|char|int)\s*\*?\s*(\w+)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("plic_volume", "plic_offset", "plic_offset_backward", "plic_volume_backward",
              "vof_interface_compact", "vof_curvature", "vof_curvature_backward",
              "vof_curvature_batched", "plic_workspace_bytes", "plic_status_string"):
        assert n in names, n


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


# entry points with no counterpart in the paper (sizes, status text, version,
# host-memory addressing)
PLUMBING = {"plic_workspace_bytes", "plic_curv_bwd_workspace_bytes", "plic_status_string",
            "plic_last_error", "plic_abi_version", "plic_host_device_pointer", "plic_pipe_probe",
            "plic_read_probe"}


# deployment variants of a compute entry: no passage of the paper defines
# them, and their comment says so instead of citing one
DEPLOYMENT = {"vof_interface_compact_noalloc"}


def test_every_compute_entry_cites_its_passage():
    txt = open(HEADER).read()
    blocks = re.findall(r"/\*(.*?)\*/", txt, flags=re.S)
    cite = re.compile(r"\b(Sec\.\s*\d|Eqs?\.\s*\d|Appendix\s+[A-Z])")
    for name in DEPLOYMENT:
        heads = [b for b in blocks if re.match(r"\s*%s\b" % name, b)]
        flat = " ".join(heads[0].replace("*", " ").split()) if heads else ""
        assert "no counterpart" in flat and not cite.search(flat), name
    for name in declared_functions():
        if name in PLUMBING or name in DEPLOYMENT:
            continue
        heads = [b for b in blocks if re.match(r"\s*(\w+\s*/\s*)?%s\b" % name, b)]
        assert heads, "%s has no doc block naming it" % name
        assert any(cite.search(b) for b in heads), "%s cites no passage" % name
    assert PLUMBING <= set(declared_functions())
    assert DEPLOYMENT <= set(declared_functions())


def test_status_strings_and_version(lib):
    assert lib.plic_abi_version() == 1
    for s in range(6):
        assert lib.plic_status_string(s).startswith(b"PLIC_")
    assert lib.plic_status_string(99) == b"unknown plic_status"


def test_workspace_sizes(lib):
    # one int per tile (tiles of whole rows, >= 8192 cells each) + 1 bit per cell, 256-byte rounded
    r256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    # tile counts + interface bits
    assert lib.plic_workspace_bytes(plic.WS_COMPACT, 256 ** 3) == (
        r256((2 * 2048 + 1) * 4) + r256((256 ** 3 // 16 + 1) * 4))
    assert lib.plic_workspace_bytes(plic.WS_COMPACT, 1) == 512
    assert lib.plic_workspace_bytes(plic.WS_BATCHED, 64) >= 64 * (ctypes.sizeof(plic.VofField) + 8)
    assert lib.plic_workspace_bytes(77, 10) == 0
    assert lib.plic_curv_bwd_workspace_bytes(128 ** 3, 1000) == 128 ** 3 * 4 + (27 * 4 * 1000 + 255) // 256 * 256


def test_host_side_argument_checks(lib):
    P = ctypes.c_void_p
    ok = P(256)                      # never dereferenced: every call below fails validation
    ERR_ARG, ERR_ALIGN = 1, 2
    # negative size, bad enum, bad flags, NULL pointers
    assert lib.plic_offset(ok, ok, ok, ok, ok, -1, 2, 1, 0, None, None) == ERR_ARG
    assert lib.plic_offset(ok, ok, ok, ok, ok, 10, 7, 1, 0, None, None) == ERR_ARG
    assert lib.plic_offset(ok, ok, ok, ok, ok, 10, 2, 5, 0, None, None) == ERR_ARG
    assert lib.plic_offset(ok, ok, ok, ok, ok, 10, 2, 1, 0x100, None, None) == ERR_ARG
    assert lib.plic_offset(None, ok, ok, ok, ok, 10, 2, 1, 0, None, None) == ERR_ARG
    # misaligned element pointers
    assert lib.plic_offset(P(258), ok, ok, ok, ok, 10, 2, 1, 0, None, None) == ERR_ALIGN
    assert lib.plic_offset(P(260), ok, ok, ok, ok, 10, 2, 2, 0, None, None) == ERR_ALIGN
    assert lib.plic_volume(ok, ok, ok, ok, None, 10, 0, None) == ERR_ARG
    # empty work is a no-op
    assert lib.plic_offset(None, None, None, None, None, 0, 2, 1, 0, None, None) == 0
    assert lib.plic_volume(None, None, None, None, None, 0, 0, None) == 0
    assert lib.plic_offset_backward(None, None, None, None, None, None, None, None, None, 0, 0, None) == 0
    # curvature: too small a field, bad method, conflicting fit flags
    assert lib.vof_curvature(ok, 2, 8, 8, ok, 5, None, ok, 2, 0, None) == ERR_ARG
    assert lib.vof_curvature(ok, 8, 8, 8, ok, 5, None, ok, 9, 0, None) == ERR_ARG
    assert lib.vof_curvature(ok, 8, 8, 8, ok, 5, None, ok, 2, 8 | 16, None) == ERR_ARG
    assert lib.vof_curvature(ok, 8, 8, 8, ok, 5, None, ok, 2, 8 | 32, None) == ERR_ARG
    assert lib.vof_curvature(ok, 8, 8, 8, ok, 0, None, ok, 2, 0, None) == 0
    assert lib.vof_curvature(ok, 2048, 2048, 513, ok, 5, None, ok, 2, 0, None) == ERR_ARG   # > 2^31 - 1 cells
    # compaction: workspace too small, unaligned workspace, oversized field
    assert lib.vof_interface_compact(ok, 64, 64, 64, ok, 10, ok, ok, 4, None) == ERR_ARG
    assert lib.vof_interface_compact(ok, 64, 64, 64, ok, 10, ok, P(264), 1 << 20, None) == ERR_ALIGN
    assert lib.vof_interface_compact(ok, 2048, 2048, 1024, ok, 10, ok, ok, 1 << 30, None) == ERR_ARG
    # allocation-free compaction: 2^28 + 1 = 17 x 15790321 cells, one cell over
    # the built-in scratch's limit, is refused before any CUDA call
    assert lib.vof_interface_compact_noalloc(ok, 17, 15790321, 1, ok, 10, ok, None) == ERR_ARG
    assert b"limit" in lib.plic_last_error()
    assert lib.vof_interface_compact_noalloc(ok, -1, 8, 8, ok, 10, ok, None) == ERR_ARG
    assert lib.vof_interface_compact_noalloc(ok, 8, 8, 8, ok, 10, None, None) == ERR_ARG
    # read probe: negative size, null sink, unaligned buffer (no launch)
    assert lib.plic_read_probe(ok, -1, ok, None) == ERR_ARG
    assert lib.plic_read_probe(ok, 16, None, None) == ERR_ARG
    assert lib.plic_read_probe(None, 16, ok, None) == ERR_ARG
    assert lib.plic_read_probe(P(260), 16, ok, None) == ERR_ALIGN
    assert lib.plic_read_probe(ok, 0, ok, None) == 0
    # host-mapped address query: null arguments
    out = ctypes.c_void_p()
    assert lib.plic_host_device_pointer(None, ctypes.byref(out)) == ERR_ARG
    assert lib.plic_host_device_pointer(ok, None) == ERR_ARG
    # batched: bad tuning
    tun = plic.VofTuning(48, 16, 1)
    f = (plic.VofField * 1)()
    assert lib.vof_curvature_batched(ctypes.cast(f, P), 1, ctypes.cast(ctypes.pointer(tun), P), 2, 0,
                                     ok, 1 << 20, None) == ERR_ARG
    for lanes in (2, 4, -1):                     # one thread or eight lanes per cell only
        tun = plic.VofTuning(128, 64, 0, lanes)
        assert lib.vof_curvature_batched(ctypes.cast(f, P), 1, ctypes.cast(ctypes.pointer(tun), P), 2,
                                         0, ok, 1 << 20, None) == ERR_ARG
    # plane-sphere: bad n, precision, null, misaligned; empty is a no-op
    assert lib.plic_sphere_offset(ok, ok, -1, 0, None) == ERR_ARG
    assert lib.plic_sphere_offset(ok, ok, 10, 4, None) == ERR_ARG
    assert lib.plic_sphere_volume(None, ok, 10, 0, None) == ERR_ARG
    assert lib.plic_sphere_volume(ok, P(258), 10, 0, None) == ERR_ALIGN
    assert lib.plic_sphere_offset(P(260), ok, 10, 2, None) == ERR_ALIGN
    assert lib.plic_sphere_offset(None, None, 0, 0, None) == 0
    # paper harness: L < 2, bad precision, null accumulator
    assert lib.plic_paper_benchmark(ok, ok, ok, 10, 1, 2, 1, 0, ok, None) == ERR_ARG
    assert lib.plic_paper_benchmark(ok, ok, ok, 10, 256, 2, 3, 0, ok, None) == ERR_ARG
    assert lib.plic_paper_benchmark(ok, ok, ok, 10, 256, 2, 1, 0, None, None) == ERR_ARG
    assert lib.plic_paper_benchmark(ok, ok, ok, 10, 256, 2, 1, 0, P(260), None) == ERR_ALIGN


def test_binding_refuses_cpu_tensors(lib):
    import torch
    x = torch.zeros(8)
    with pytest.raises(plic.PlicError):
        plic.offset(x, x, x, x)
    with pytest.raises(plic.PlicError):
        plic.volume(x, x, x, x)
