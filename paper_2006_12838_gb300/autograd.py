"""torch.autograd.Function wrappers over the forward/backward C ABI pairs.

* :func:`offset`    -- d0 = plic_offset(n, V0); backward plic_offset_backward
  (g_V0 = g/A, g_n = g c, implicit function theorem on Eq. 1).
* :func:`volume`    -- V0 = plic_volume(n, d0); backward plic_volume_backward
  (g_d0 = g A, g_n = -g A c).
* :func:`curvature` -- kappa = vof_curvature(phi, idx); backward
  vof_curvature_backward (dense g_phi, interface set held fixed).

All arithmetic runs in the library's kernels; these classes only route
tensors.  The interface list ``idx`` is an integer input without gradient.
"""
from __future__ import annotations

import torch

from . import plic


class PlicOffset(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nx, ny, nz, V0, method="sz_opt", precision=None):
        d0 = plic.offset(nx.contiguous(), ny.contiguous(), nz.contiguous(), V0.contiguous(),
                         method=method, precision=precision)
        ctx.save_for_backward(nx, ny, nz, d0)
        return d0

    @staticmethod
    def backward(ctx, g):
        nx, ny, nz, d0 = ctx.saved_tensors
        need_n = any(ctx.needs_input_grad[:3])
        gV, gx, gy, gz = plic.offset_backward(nx.contiguous(), ny.contiguous(), nz.contiguous(), d0,
                                              g.contiguous(), need=(ctx.needs_input_grad[3], need_n))
        return gx, gy, gz, gV, None, None


class PlicVolume(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nx, ny, nz, d0):
        V0 = plic.volume(nx.contiguous(), ny.contiguous(), nz.contiguous(), d0.contiguous())
        ctx.save_for_backward(nx, ny, nz, d0)
        return V0

    @staticmethod
    def backward(ctx, g):
        nx, ny, nz, d0 = ctx.saved_tensors
        need_n = any(ctx.needs_input_grad[:3])
        gd, gx, gy, gz = plic.volume_backward(nx.contiguous(), ny.contiguous(), nz.contiguous(),
                                              d0.contiguous(), g.contiguous(),
                                              need=(ctx.needs_input_grad[3], need_n))
        return gx, gy, gz, gd


class VofCurvature(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, idx, method="sz_opt", flags=0):
        phi = phi.contiguous()
        kappa = plic.curvature(phi, idx, method=method, flags=flags)
        ctx.save_for_backward(phi, idx)
        ctx.method = method
        ctx.flags = flags
        return kappa

    @staticmethod
    def backward(ctx, g):
        phi, idx = ctx.saved_tensors
        g_phi = plic.curvature_backward(phi, idx, g.contiguous(), method=ctx.method, flags=ctx.flags)
        return g_phi, None, None, None


def offset(nx, ny, nz, V0, method="sz_opt", precision=None):
    """d0(n, V0) of Eq. 1, differentiable in n and V0 (implicit function theorem)."""
    return PlicOffset.apply(nx, ny, nz, V0, method, precision)


def volume(nx, ny, nz, d0):
    """V0(n, d0) of Eq. 10, differentiable in n and d0."""
    return PlicVolume.apply(nx, ny, nz, d0)


def curvature(phi, idx, method="sz_opt", flags=0):
    """kappa of the listed interface cells (Sec. 4.2, Appendix B), differentiable
    in phi with the interface set held fixed."""
    return VofCurvature.apply(phi, idx, method, flags)
