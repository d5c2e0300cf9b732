"""ctypes binding of the PLIC C ABI (``include/plic.h``, ``libplic.so``).

Argument marshalling only: every function takes CUDA tensors, checks their
dtype/device/contiguity, passes raw device pointers and the current CUDA
stream to the library, and raises :class:`PlicError` on a non-zero status.
All arithmetic runs in the library's kernels; there is no CPU path, and a
missing library is an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

METHODS = {"analytic": 0, "sz_orig": 1, "sz_opt": 2, "newton": 3, "nested": 4}
PRECISIONS = {"fp32": 0, "fp32p": 1, "fp64": 2, "fp64r": 3}
FLAG_FAITHFUL = 1
FLAG_POINT_CENTROID = 2
FLAG_KAPPA_PAPER_SIGN = 4
FLAG_FIT_FP32 = 8
FLAG_FIT_DF32 = 16
FLAG_FIT_FP64 = 32
FLAG_NORMAL_CM = 64
FLAG_NEIGHBOR_NORMAL = 128
WS_COMPACT = 0
WS_BATCHED = 2

_lock = threading.Lock()
_lib = None


class PlicError(RuntimeError):
    pass


class VofField(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_void_p), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("idx", ctypes.c_void_p), ("n_iface", ctypes.c_int64),
                ("kappa", ctypes.c_void_p)]


class VofTuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("cells_per_chunk", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("lanes_per_cell", ctypes.c_int)]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libplic.so (built by ``paper_2006_12838_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise PlicError("libplic.so is not built (%s); run paper_2006_12838_gb300.build.build()"
                            % path)
        L = ctypes.CDLL(path)
        P, I64, I32, U32, SZ = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                ctypes.c_size_t)
        sigs = {
            "plic_volume": [P, P, P, P, P, I64, I32, P],
            "plic_offset": [P, P, P, P, P, I64, I32, I32, U32, P, P],
            "plic_offset_backward": [P, P, P, P, P, P, P, P, P, I64, I32, P],
            "plic_volume_backward": [P, P, P, P, P, P, P, P, P, I64, I32, P],
            "vof_interface_compact": [P, I32, I32, I32, P, I64, P, P, SZ, P],
            "vof_interface_compact_noalloc": [P, I32, I32, I32, P, I64, P, P],
            "vof_curvature": [P, I32, I32, I32, P, I64, P, P, I32, U32, P],
            "vof_laplace_pressure": [P, I32, I32, I32, P, I64, P, ctypes.c_float, P, I32, U32, P],
            "vof_normal": [P, I32, I32, I32, P, I64, P, P, P, P, U32, P],
            "vof_curvature_backward": [P, I32, I32, I32, P, I64, P, P, P, I32, U32, P, SZ, P],
            "vof_curvature_batched": [P, I32, P, I32, U32, P, SZ, P],
            "plic_paper_benchmark": [P, P, P, I64, I32, I32, I32, I32, P, P],
            "plic_sphere_volume": [P, P, I64, I32, P],
            "plic_offset_roundtrip": [P, P, P, P, P, P, I64, I32, I32, U32, P, P],
            "plic_sphere_offset": [P, P, I64, I32, P],
            "plic_pipe_probe": [I32, I32, P, ctypes.POINTER(I64), P],
            "plic_read_probe": [P, I64, P, P],
        }
        for name, args in sigs.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = ctypes.c_int
        L.plic_workspace_bytes.argtypes = [I32, I64]
        L.plic_workspace_bytes.restype = SZ
        L.plic_curv_bwd_workspace_bytes.argtypes = [I64, I64]
        L.plic_curv_bwd_workspace_bytes.restype = SZ
        L.plic_status_string.argtypes = [I32]
        L.plic_status_string.restype = ctypes.c_char_p
        L.plic_last_error.argtypes = []
        L.plic_last_error.restype = ctypes.c_char_p
        L.plic_abi_version.restype = ctypes.c_int
        L.plic_host_device_pointer.argtypes = [P, ctypes.POINTER(ctypes.c_void_p)]
        L.plic_host_device_pointer.restype = ctypes.c_int
        if L.plic_abi_version() != 1:
            raise PlicError("libplic.so ABI version mismatch")
        _lib = L
        return L


def _check(status: int, what: str):
    if status != 0:
        L = load()
        raise PlicError("%s: %s %s" % (what, L.plic_status_string(status).decode(),
                                       L.plic_last_error().decode()))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(t, stream):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _cuda(*ts, dtype=None):
    ref = ts[0]
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise PlicError("tensors must be CUDA tensors (there is no CPU path)")
        if t.device != ref.device:
            raise PlicError("tensors must be on one device")
        if not t.is_contiguous():
            raise PlicError("tensors must be contiguous")
        if dtype is not None and t.dtype != dtype:
            raise PlicError("expected dtype %s, got %s" % (dtype, t.dtype))


def _prec(dtype, precision):
    if precision is None:
        return 2 if dtype == torch.float64 else 1
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    want = torch.float64 if p >= 2 else torch.float32
    if dtype != want:
        raise PlicError("precision %s needs %s tensors" % (precision, want))
    return p


def host_device_pointer(t) -> int:
    """Device address of a page-locked (pinned) CPU tensor's storage, for the
    zero-copy entry points; raises PlicError for any other tensor."""
    if t.is_cuda or not t.is_contiguous():
        raise PlicError("expected a contiguous pinned CPU tensor")
    out = ctypes.c_void_p()
    _check(load().plic_host_device_pointer(ctypes.c_void_p(t.data_ptr()), ctypes.byref(out)),
           "plic_host_device_pointer (is the tensor pinned?)")
    return int(out.value)


def volume(nx, ny, nz, d0, out=None, stream=None):
    """V0 = plic_volume(n, d0) (Sec. 2.2, Eq. 10)."""
    _cuda(nx, ny, nz, d0, out, dtype=d0.dtype)
    p = 2 if d0.dtype == torch.float64 else 0
    out = torch.empty_like(d0) if out is None else out
    _check(load().plic_volume(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(d0), _ptr(out), d0.numel(), p,
                              _stream(d0, stream)), "plic_volume")
    return out


def offset(nx, ny, nz, V0, method="sz_opt", precision=None, faithful=False, out=None,
           invalid=None, stream=None):
    """d0 = plic_offset(n, V0) (Sec. 2, Eq. 1).  ``invalid``: optional CUDA int64
    tensor of one element that accumulates the number of invalid cells."""
    _cuda(nx, ny, nz, V0, out, dtype=V0.dtype)
    p = _prec(V0.dtype, precision)
    m = METHODS[method] if isinstance(method, str) else int(method)
    if invalid is not None:
        _cuda(V0, invalid, dtype=None)
        if invalid.dtype != torch.int64:
            raise PlicError("invalid counter must be int64")
    out = torch.empty_like(V0) if out is None else out
    _check(load().plic_offset(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(V0), _ptr(out), V0.numel(), m, p,
                              FLAG_FAITHFUL if faithful else 0, _ptr(invalid),
                              _stream(V0, stream)), "plic_offset")
    return out


def offset_roundtrip(nx, ny, nz, V0, method="sz_opt", precision=None, faithful=False, out=None,
                     out_rt=None, invalid=None, stream=None):
    """(d0, V0_rt): plic_offset and the forward volume of its result in one
    call (Sec. 2.5 round trip); one fused kernel for SZ-opt and the analytic solution in FP32."""
    _cuda(nx, ny, nz, V0, out, out_rt, dtype=V0.dtype)
    p = _prec(V0.dtype, precision)
    m = METHODS[method] if isinstance(method, str) else int(method)
    if invalid is not None:
        _cuda(V0, invalid, dtype=None)
        if invalid.dtype != torch.int64:
            raise PlicError("invalid counter must be int64")
    out = torch.empty_like(V0) if out is None else out
    out_rt = torch.empty_like(V0) if out_rt is None else out_rt
    _check(load().plic_offset_roundtrip(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(V0), _ptr(out),
                                        _ptr(out_rt), V0.numel(), m, p,
                                        FLAG_FAITHFUL if faithful else 0, _ptr(invalid),
                                        _stream(V0, stream)), "plic_offset_roundtrip")
    return out, out_rt


def offset_backward(nx, ny, nz, d0, g_d0, stream=None, need=(True, True)):
    """(g_V0, g_nx, g_ny, g_nz) of plic_offset at its solution d0 (implicit
    function theorem on Eq. 1: g/A and g c, A and c the cut polygon's area and
    centroid)."""
    _cuda(nx, ny, nz, d0, g_d0, dtype=d0.dtype)
    p = 2 if d0.dtype == torch.float64 else 0
    gV = torch.empty_like(d0) if need[0] else None
    gx, gy, gz = ((torch.empty_like(d0) for _ in range(3)) if need[1] else (None, None, None))
    _check(load().plic_offset_backward(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(d0), _ptr(g_d0),
                                       _ptr(gV), _ptr(gx), _ptr(gy), _ptr(gz), d0.numel(), p,
                                       _stream(d0, stream)), "plic_offset_backward")
    return gV, gx, gy, gz


def volume_backward(nx, ny, nz, d0, g_V0, stream=None, need=(True, True)):
    """(g_d0, g_nx, g_ny, g_nz) of plic_volume (derivatives of Eq. 10: g A and
    -g A c)."""
    _cuda(nx, ny, nz, d0, g_V0, dtype=d0.dtype)
    p = 2 if d0.dtype == torch.float64 else 0
    gd = torch.empty_like(d0) if need[0] else None
    gx, gy, gz = ((torch.empty_like(d0) for _ in range(3)) if need[1] else (None, None, None))
    _check(load().plic_volume_backward(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(d0), _ptr(g_V0),
                                       _ptr(gd), _ptr(gx), _ptr(gy), _ptr(gz), d0.numel(), p,
                                       _stream(d0, stream)), "plic_volume_backward")
    return gd, gx, gy, gz


def workspace_bytes(op: int, arg: int) -> int:
    return int(load().plic_workspace_bytes(op, arg))


def curv_bwd_workspace_bytes(cells: int, n_iface: int) -> int:
    return int(load().plic_curv_bwd_workspace_bytes(cells, n_iface))


def interface_compact(phi, idx=None, count=None, workspace=None, stream=None):
    """Interface-cell list of a (nz, ny, nx) float32 field (Sec. 4.1, Eq. 33).

    Returns (idx, count) as device tensors; idx has capacity phi.numel() unless
    given; count is a one-element int64 tensor (no host synchronisation)."""
    _cuda(phi, dtype=torch.float32)
    nz, ny, nx = phi.shape
    if idx is None:
        idx = torch.empty(phi.numel(), dtype=torch.int32, device=phi.device)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=phi.device)
    ws_n = workspace_bytes(WS_COMPACT, phi.numel())
    if workspace is None:
        workspace = torch.empty(max(ws_n, 1), dtype=torch.uint8, device=phi.device)
    _cuda(phi, idx, count, workspace)
    _check(load().vof_interface_compact(_ptr(phi), nx, ny, nz, _ptr(idx), idx.numel(), _ptr(count),
                                        _ptr(workspace), workspace.numel(),
                                        _stream(phi, stream)), "vof_interface_compact")
    return idx, count


def curvature(phi, idx, n_iface=None, count=None, kappa=None, method="sz_opt", flags=0,
              stream=None):
    """kappa per interface cell (Sec. 4.2, Appendix B)."""
    _cuda(phi, dtype=torch.float32)
    _cuda(phi, idx, dtype=None)
    nz, ny, nx = phi.shape
    n = idx.numel() if n_iface is None else int(n_iface)
    if kappa is None:
        kappa = torch.empty(max(n, 1), dtype=torch.float32, device=phi.device)
    m = METHODS[method] if isinstance(method, str) else int(method)
    _check(load().vof_curvature(_ptr(phi), nx, ny, nz, _ptr(idx), n, _ptr(count), _ptr(kappa), m,
                                flags, _stream(phi, stream)), "vof_curvature")
    return kappa[:n] if n_iface is not None or kappa.numel() != n else kappa


def laplace_pressure(phi, idx, sigma, n_iface=None, count=None, dp=None, method="sz_opt",
                     flags=0, stream=None):
    """Young-Laplace pressure jump dp = 2 sigma kappa per interface cell (Sec. 4.1)."""
    _cuda(phi, dtype=torch.float32)
    _cuda(phi, idx, dtype=None)
    nz, ny, nx = phi.shape
    n = idx.numel() if n_iface is None else int(n_iface)
    if dp is None:
        dp = torch.empty(max(n, 1), dtype=torch.float32, device=phi.device)
    m = METHODS[method] if isinstance(method, str) else int(method)
    _check(load().vof_laplace_pressure(_ptr(phi), nx, ny, nz, _ptr(idx), n, _ptr(count),
                                       float(sigma), _ptr(dp), m, flags, _stream(phi, stream)),
           "vof_laplace_pressure")
    return dp[:n] if n_iface is not None or dp.numel() != n else dp


def normals(phi, idx, n_iface=None, count=None, out=None, flags=0, stream=None):
    """Interface normals (Appendix B: Parker-Youngs, or CM with FLAG_NORMAL_CM),
    returned as a (3, n) float tensor (rows n_x, n_y, n_z)."""
    _cuda(phi, dtype=torch.float32)
    _cuda(phi, idx, dtype=None)
    nz, ny, nx = phi.shape
    n = idx.numel() if n_iface is None else int(n_iface)
    if out is None:
        out = torch.empty((3, max(n, 1)), dtype=torch.float32, device=phi.device)
    _cuda(phi, out, dtype=None)
    _check(load().vof_normal(_ptr(phi), nx, ny, nz, _ptr(idx), n, _ptr(count), _ptr(out[0]),
                             _ptr(out[1]), _ptr(out[2]), flags, _stream(phi, stream)),
           "vof_normal")
    return out[:, :n]


def curvature_backward(phi, idx, g_kappa, n_iface=None, count=None, g_phi=None,
                       method="sz_opt", flags=0, workspace=None, stream=None):
    """g_phi = d(sum g_kappa * kappa)/d phi (dense, same shape as phi): the
    adjoint of the curvature step of Sec. 4.2 and Appendix B."""
    _cuda(phi, g_kappa, dtype=torch.float32)
    nz, ny, nx = phi.shape
    n = idx.numel() if n_iface is None else int(n_iface)
    if g_phi is None:
        g_phi = torch.empty_like(phi)
    ws_n = curv_bwd_workspace_bytes(phi.numel(), n)
    if workspace is None:
        workspace = torch.empty(max(ws_n, 1), dtype=torch.uint8, device=phi.device)
    m = METHODS[method] if isinstance(method, str) else int(method)
    _check(load().vof_curvature_backward(_ptr(phi), nx, ny, nz, _ptr(idx), n, _ptr(count),
                                         _ptr(g_kappa), _ptr(g_phi), m, flags, _ptr(workspace),
                                         workspace.numel(), _stream(phi, stream)),
           "vof_curvature_backward")
    return g_phi


class BatchedFields:
    """The descriptor table of a list of fields for vof_curvature_batched, built
    and checked once: ``fields`` is a list of (phi, idx, n_iface, kappa) with
    device tensors.  Reusing it saves the per-call Python work of building the
    table (a few microseconds per field), which for many fields would otherwise
    exceed the kernel's own time."""

    def __init__(self, fields, workspace=None):
        self.fields = list(fields)
        self.arr = (VofField * len(self.fields))()
        dev = self.fields[0][0].device
        for i, (phi, idx, n, kappa) in enumerate(self.fields):
            _cuda(phi, kappa, dtype=torch.float32)
            _cuda(idx, dtype=torch.int32)
            if idx.device != phi.device or phi.device != dev:
                raise PlicError("tensors must be on one device")
            nz, ny, nx = phi.shape
            self.arr[i] = VofField(phi.data_ptr(), nx, ny, nz, idx.data_ptr(), int(n),
                                   kappa.data_ptr())
        ws_n = workspace_bytes(WS_BATCHED, len(self.fields))
        if workspace is None:
            workspace = torch.empty(max(ws_n, 1), dtype=torch.uint8, device=dev)
        elif workspace.numel() < ws_n:
            raise PlicError("workspace too small")
        self.workspace = workspace
        self.ptr = ctypes.cast(self.arr, ctypes.c_void_p)

    def __len__(self):
        return len(self.fields)


def curvature_batched(fields, method="sz_opt", flags=0, tuning=None, workspace=None,
                      stream=None):
    """The curvature step (Sec. 4.2, Appendix B) over many fields in one
    persistent launch.  ``fields``: a BatchedFields, or a list of (phi, idx,
    n_iface, kappa) with device tensors; ``tuning``: optional (block_threads,
    cells_per_chunk, blocks_per_sm[, lanes_per_cell]) with lanes_per_cell 8
    (cooperative groups), 1 (one thread per cell) or 0 (the library's
    default)."""
    if not isinstance(fields, BatchedFields):
        fields = BatchedFields(fields, workspace)
    tun = None
    if tuning is not None:
        t = [int(v) for v in tuning]
        if len(t) not in (3, 4):
            raise PlicError("tuning: (block_threads, cells_per_chunk, blocks_per_sm[, lanes_per_cell])")
        tun = VofTuning(*(t + [0] * (4 - len(t))))
    m = METHODS[method] if isinstance(method, str) else int(method)
    ws = fields.workspace
    _check(load().vof_curvature_batched(fields.ptr, len(fields),
                                        None if tun is None else ctypes.cast(ctypes.pointer(tun), ctypes.c_void_p),
                                        m, flags, _ptr(ws), ws.numel(),
                                        _stream(fields.fields[0][0], stream)), "vof_curvature_batched")


def paper_benchmark(nx, ny, nz, L=256, method="sz_opt", precision=None, blank=False, err_sum=None,
                    stream=None):
    """Sec. 2.5 harness: sum over normals and L fill levels of the round-trip
    error; returns the device accumulator (double, one element)."""
    _cuda(nx, ny, nz, dtype=nx.dtype)
    p = _prec(nx.dtype, precision)
    m = METHODS[method] if isinstance(method, str) else int(method)
    if err_sum is None:
        err_sum = torch.zeros(1, dtype=torch.float64, device=nx.device)
    _check(load().plic_paper_benchmark(_ptr(nx), _ptr(ny), _ptr(nz), nx.numel(), int(L), m, p,
                                       1 if blank else 0, _ptr(err_sum), _stream(nx, stream)),
           "plic_paper_benchmark")
    return err_sum


def sphere_volume(d0, precision=None, out=None, stream=None):
    """Sec. 3: cap volume of the unit-volume ball below a plane at distance d0."""
    _cuda(d0, out, dtype=d0.dtype)
    p = _prec(d0.dtype, precision)
    if out is None:
        out = torch.empty_like(d0)
    _check(load().plic_sphere_volume(_ptr(d0), _ptr(out), d0.numel(), p, _stream(d0, stream)),
           "plic_sphere_volume")
    return out


def sphere_offset(V0, precision=None, out=None, stream=None):
    """Sec. 3: plane distance d0 that cuts volume V0 off the unit-volume ball."""
    _cuda(V0, out, dtype=V0.dtype)
    p = _prec(V0.dtype, precision)
    if out is None:
        out = torch.empty_like(V0)
    _check(load().plic_sphere_offset(_ptr(V0), _ptr(out), V0.numel(), p, _stream(V0, stream)),
           "plic_sphere_offset")
    return out


PROBES = {"ffma": 0, "ffma2": 1, "dfma": 2, "mufu_ex2_lg2": 3, "mufu_rsqrt": 4, "mufu_sin": 5,
          "d_sqrt": 6, "d_div": 7, "d_cbrt": 8, "d_sin": 9, "d_cos": 10, "d_asin": 11,
          "d_acos": 12, "d_atan2": 13}


def pipe_probe(kind, iters, sink, stream=None) -> int:
    """Launch the pipe-throughput probe ``kind`` (a key of PROBES) on the
    current device; returns the number of operations (or calls) the launch
    performs.  ``sink``: a CUDA float tensor of at least one element."""
    L = load()
    _cuda(sink, dtype=torch.float32)
    ops = ctypes.c_int64(0)
    _check(L.plic_pipe_probe(PROBES[kind], int(iters), _ptr(sink), ctypes.byref(ops),
                             _stream(sink, stream)), "plic_pipe_probe")
    return int(ops.value)


def read_probe(buf, sink, stream=None):
    """Launch the plain streaming read of the float32 tensor ``buf`` (the
    fastest one-pass read from the cache state it finds; time it with CUDA
    events).  ``sink``: a CUDA float tensor of at least one element."""
    _cuda(buf, sink, dtype=torch.float32)
    _check(load().plic_read_probe(_ptr(buf), buf.numel(), _ptr(sink), _stream(buf, stream)),
           "plic_read_probe")
