"""Host-buffer entry points: PLIC offsets for arrays that live in (pinned) host
memory.

Two ways, the same C ABI call as :func:`plic.offset` / :func:`plic.offset_roundtrip`:

- :class:`MappedHostOffset` (zero copy): the kernel is given the device
  addresses of the pinned host arrays (``plic_host_device_pointer``) and reads
  its inputs and writes its results over the host link itself, one launch per
  pass, no staging buffers.  On a Grace-Blackwell node the link is NVLink-C2C
  and the kernel's streaming loads keep it busy in both directions at once.
- :class:`HostOffsetPipeline` (staged): chunk i is copied host->device on one
  stream while chunk i-1 is solved on a second and chunk i-2 is copied back on a
  third, so the copies and the kernels overlap; ``capture`` turns a whole pass
  into one CUDA graph.  For hosts whose memory the device cannot map.
"""
from __future__ import annotations

import ctypes

import torch

from . import plic


class MappedHostOffset:
    """Zero-copy solve of pinned host arrays: ``run(nx, ny, nz, V0, d0_out,
    V_out=None)`` launches plic_offset (or plic_offset_roundtrip when V_out is
    given) on the device addresses of the host tensors, on the current stream.
    Every tensor must be a contiguous pinned CPU tensor of the same length (the
    address query raises PlicError otherwise, before anything is launched)."""

    def __init__(self, device="cuda", method="sz_opt", precision=None):
        self.device = torch.device(device)
        self.method = method
        self.precision = precision
        self.launches = 0

    def run(self, nx, ny, nz, V0, d0_out, V_out=None):
        n = V0.numel()
        ts = [nx, ny, nz, V0, d0_out] + ([V_out] if V_out is not None else [])
        for t in ts:
            if t.numel() != n or t.dtype != V0.dtype:
                raise plic.PlicError("host arrays must have one length and dtype")
        ptrs = [plic.host_device_pointer(t) for t in ts]
        p = plic._prec(V0.dtype, self.precision)
        m = plic.METHODS[self.method] if isinstance(self.method, str) else int(self.method)
        stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        P = ctypes.c_void_p
        if V_out is not None:
            st = plic.load().plic_offset_roundtrip(*[P(x) for x in ptrs], n, m, p, 0, None, stream)
            plic._check(st, "plic_offset_roundtrip (host-mapped)")
        else:
            st = plic.load().plic_offset(*[P(x) for x in ptrs], n, m, p, 0, None, stream)
            plic._check(st, "plic_offset (host-mapped)")
        self.launches = 1


class HostOffsetPipeline:
    """Reusable device staging buffers and streams for host-resident batches.

    ``run(nx, ny, nz, V0, d0_out, V0_roundtrip_out=None)`` solves
    d0 = plic_offset(n, V0) for host tensors (pinned) and, if
    ``V0_roundtrip_out`` is given, also the forward volume of the result
    (plic_offset_roundtrip)."""

    def __init__(self, chunk: int, dtype=torch.float32, device="cuda", method="sz_opt",
                 precision=None, depth: int = 3):
        self.chunk = int(chunk)
        self.dtype = dtype
        self.device = torch.device(device)
        self.method = method
        self.precision = precision
        self.depth = depth
        mk = lambda: torch.empty(self.chunk, dtype=dtype, device=self.device)  # noqa: E731
        self.bufs = [[mk() for _ in range(6)] for _ in range(depth)]
        self.h2d = torch.cuda.Stream(self.device)
        self.comp = torch.cuda.Stream(self.device)
        self.d2h = torch.cuda.Stream(self.device)
        self.launches = 0

    def run(self, nx, ny, nz, V0, d0_out, V_out=None):
        n = V0.numel()
        ev_in = [torch.cuda.Event() for _ in range(self.depth)]
        ev_done = [torch.cuda.Event() for _ in range(self.depth)]
        ev_free = [None] * self.depth
        cur = torch.cuda.current_stream(self.device)
        for s in (self.h2d, self.comp, self.d2h):
            s.wait_stream(cur)
        self.launches = 0
        for j, start in enumerate(range(0, n, self.chunk)):
            k = min(self.chunk, n - start)
            b = j % self.depth
            bx, by, bz, bv, bd, bw = (t[:k] for t in self.bufs[b])
            if ev_free[b] is not None:
                self.h2d.wait_event(ev_free[b])
            with torch.cuda.stream(self.h2d):
                for dst, src in ((bx, nx), (by, ny), (bz, nz), (bv, V0)):
                    dst.copy_(src[start:start + k], non_blocking=True)
                ev_in[b].record(self.h2d)
            self.comp.wait_event(ev_in[b])
            if V_out is not None:
                plic.offset_roundtrip(bx, by, bz, bv, method=self.method, precision=self.precision,
                                      out=bd, out_rt=bw, stream=self.comp)
            else:
                plic.offset(bx, by, bz, bv, method=self.method, precision=self.precision, out=bd,
                            stream=self.comp)
            self.launches += 1
            ev_done[b].record(self.comp)
            self.d2h.wait_event(ev_done[b])
            with torch.cuda.stream(self.d2h):
                d0_out[start:start + k].copy_(bd, non_blocking=True)
                if V_out is not None:
                    V_out[start:start + k].copy_(bw, non_blocking=True)
                e = torch.cuda.Event()
                e.record(self.d2h)
                ev_free[b] = e
        for s in (self.h2d, self.comp, self.d2h):
            cur.wait_stream(s)

    def capture(self, nx, ny, nz, V0, d0_out, V_out=None):
        """A CUDA graph of ``run`` for these host buffers: every chunk's copies and
        kernel launches become one graph, so a step is one ``replay()`` with no
        per-chunk host work.  The buffers must stay alive while the graph is used."""
        cur = torch.cuda.current_stream(self.device)
        self.run(nx, ny, nz, V0, d0_out, V_out)          # warm-up outside the capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(nx, ny, nz, V0, d0_out, V_out)
        cur.wait_stream(torch.cuda.current_stream(self.device))
        return g
