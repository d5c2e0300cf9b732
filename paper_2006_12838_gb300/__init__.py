"""GB300-native PLIC hot path (Lehmann & Gekle, arXiv 2006.12838).

Batched plane-cube offset inversion with five solvers, the forward plane-cube
volume, the PLIC-based VOF curvature step, and their adjoints, as hand-written
CUDA kernels for sm_103a behind a C ABI (``include/plic.h``).

Submodules:

* ``plic``     -- ctypes binding of the C ABI (argument marshalling only).
* ``autograd`` -- torch.autograd.Function wrappers over the forward/backward calls.
* ``synth``    -- seeded synthetic inputs shaped like the paper's workloads.
* ``build``    -- nvcc build of the shared library.

Importing the package loads nothing; the GPU library is loaded on first use and
its absence is an error (there is no CPU fallback).
"""
__all__ = ["plic", "autograd", "synth", "build"]
