"""FP64 CPU oracle for the PLIC hot path (Lehmann & Gekle, arXiv 2006.12838).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library and its
Python binding never import it, and it shares no code with them: the
arithmetic lives in ``plic_oracle.c`` (plain C, compiled with gcc, no fast
math, no FMA contraction) and this module only marshals numpy arrays.

Functions and the passages they follow:

* :func:`volume`          -- Sec. 2 problem statement (Eq. 1) via Eqs. 2-10.
* :func:`offset`          -- the inverse of Eq. 1 by bisection to adjacent doubles.
* :func:`area_centroid`   -- cut polygon of the plane and the cube (clipping);
  the adjoints of Eq. 1 follow from it by the implicit function theorem.
* :func:`offset_grad`, :func:`volume_grad` -- those adjoints.
* :func:`interface_cells` -- Eq. 33 (0 < phi < 1), interior cells only.
* :func:`curvature`       -- Sec. 4.2 with Appendix B (Eqs. 36, 38, 42, 43-48).
* :func:`curvature_grad_fd` -- central differences of sum_k w_k kappa_k.
* :func:`lsq_paraboloid`, :func:`paraboloid_kappa`, :func:`py_normal` -- the
  individual curvature steps, exposed for the pins.
* :func:`cm_normal`, :func:`normals` -- the centre-of-mass normal of Appendix B
  and batched PY/CM normals.
* :func:`sphere_volume`, :func:`sphere_offset` -- the plane-sphere problem of
  Sec. 3 (spherical cap; inverse by bisection).

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, brute force, high-precision re-evaluation and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plic_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

POINT_CENTROID = 2
KAPPA_PAPER_SIGN = 4
NORMAL_CM = 64
NEIGHBOR_NORMAL = 128


def build(force: bool = False) -> str:
    """Compile ``plic_oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        D, P, I64, I32, U = (ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_int, ctypes.c_uint)
        lib.oracle_volume.restype = D
        lib.oracle_volume.argtypes = [D, D, D, D]
        lib.oracle_offset.restype = D
        lib.oracle_offset.argtypes = [D, D, D, D]
        lib.oracle_volume_batch.argtypes = [P, P, P, P, P, I64]
        lib.oracle_offset_batch.argtypes = [P, P, P, P, P, I64]
        lib.oracle_area_centroid_batch.argtypes = [P, P, P, P, P, P, P, P, I64]
        lib.oracle_num_threads.restype = I32
        lib.oracle_set_num_threads.argtypes = [I32]
        lib.oracle_d3q27.argtypes = [P]
        lib.oracle_py_normal.restype = I32
        lib.oracle_py_normal.argtypes = [P, P]
        lib.oracle_lsq_paraboloid.restype = I32
        lib.oracle_lsq_paraboloid.argtypes = [I32, P, P, P, P]
        lib.oracle_paraboloid_kappa.restype = D
        lib.oracle_paraboloid_kappa.argtypes = [P]
        lib.oracle_curvature_cell.restype = D
        lib.oracle_curvature_cell.argtypes = [P, P, P, U, P, P]
        lib.oracle_cm_normal.restype = I32
        lib.oracle_cm_normal.argtypes = [P, P]
        lib.oracle_normal_batch.argtypes = [P, I32, I32, I32, P, I64, U, P, P, P]
        lib.oracle_sphere_volume.restype = D
        lib.oracle_sphere_volume.argtypes = [D]
        lib.oracle_sphere_offset.restype = D
        lib.oracle_sphere_offset.argtypes = [D]
        lib.oracle_sphere_volume_batch.argtypes = [P, P, I64]
        lib.oracle_sphere_offset_batch.argtypes = [P, P, I64]
        lib.oracle_curvature_batch.argtypes = [P, I32, I32, I32, P, I64, U, P, P, P, P]
        lib.oracle_curvature_grad_fd.argtypes = [P, I32, I32, I32, P, I64, P, D, U, P]
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the batched oracle functions use."""
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Set the OpenMP threads of the batched oracle functions."""
    _load().oracle_set_num_threads(int(n))


def volume(nx, ny, nz, d0):
    """V0(n, d0) = vol{x in [-1/2,1/2]^3 : n.x <= d0} (Sec. 2, Eq. 1), FP64."""
    lib = _load()
    nx, ny, nz, d0 = (_f64(a).ravel() for a in np.broadcast_arrays(nx, ny, nz, d0))
    out = np.empty(nx.shape, np.float64)
    lib.oracle_volume_batch(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(d0), _ptr(out), out.size)
    return out


def offset(nx, ny, nz, V0):
    """d0 with V0(n, d0) = V0 on [-L/2, L/2] (Sec. 2, Eq. 1), bisection, FP64."""
    lib = _load()
    nx, ny, nz, V0 = (_f64(a).ravel() for a in np.broadcast_arrays(nx, ny, nz, V0))
    out = np.empty(nx.shape, np.float64)
    lib.oracle_offset_batch(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(V0), _ptr(out), out.size)
    return out


def area_centroid(nx, ny, nz, d0):
    """Area and centroid (cube-centred coordinates) of the cut polygon of the
    plane n.x = d0 (Eq. 1) with the cell."""
    lib = _load()
    nx, ny, nz, d0 = (_f64(a).ravel() for a in np.broadcast_arrays(nx, ny, nz, d0))
    A, cx, cy, cz = (np.empty(nx.shape, np.float64) for _ in range(4))
    lib.oracle_area_centroid_batch(_ptr(nx), _ptr(ny), _ptr(nz), _ptr(d0), _ptr(A),
                                   _ptr(cx), _ptr(cy), _ptr(cz), nx.size)
    return A, cx, cy, cz


def offset_grad(nx, ny, nz, d0, g):
    """Vector-Jacobian product of d0(n, V0) at the solution d0 (implicit
    function theorem on Eq. 1).

    Returns (g_V0, g_nx, g_ny, g_nz) = g * (|n|/A, c_x, c_y, c_z)."""
    nx, ny, nz, d0, g = (_f64(a).ravel() for a in np.broadcast_arrays(nx, ny, nz, d0, g))
    A, cx, cy, cz = area_centroid(nx, ny, nz, d0)
    nn = np.sqrt(nx * nx + ny * ny + nz * nz)
    return g * nn / A, g * cx, g * cy, g * cz


def volume_grad(nx, ny, nz, d0, g):
    """Vector-Jacobian product of V0(n, d0) (derivatives of Eq. 10: slice area
    and first moment of the cut polygon).

    Returns (g_d0, g_nx, g_ny, g_nz) = g * (A/|n|, -A c/|n|)."""
    nx, ny, nz, d0, g = (_f64(a).ravel() for a in np.broadcast_arrays(nx, ny, nz, d0, g))
    A, cx, cy, cz = area_centroid(nx, ny, nz, d0)
    s = A / np.sqrt(nx * nx + ny * ny + nz * nz)
    return g * s, -g * s * cx, -g * s * cy, -g * s * cz


def d3q27() -> np.ndarray:
    """The 27 stencil directions e_0..e_26 (Appendix B order), shape (27, 3)."""
    e = np.empty(81, np.int32)
    _load().oracle_d3q27(_ptr(e))
    return e.reshape(27, 3).astype(np.int64)


def py_normal(phi27):
    """Parker-Youngs normal (Eq. 38) of one 27-value stencil; None if undefined."""
    s = _f64(phi27).ravel()
    assert s.size == 27
    n = np.empty(3, np.float64)
    ok = _load().oracle_py_normal(_ptr(s), _ptr(n))
    return n if ok else None


def lsq_paraboloid(px, py, pz):
    """Least-squares (A, B, C, H, I) of Appendix B; returns (x5, fit_dim)."""
    px, py, pz = (_f64(a).ravel() for a in (px, py, pz))
    x5 = np.zeros(5, np.float64)
    dim = _load().oracle_lsq_paraboloid(px.size, _ptr(px), _ptr(py), _ptr(pz), _ptr(x5))
    return x5, int(dim)


def paraboloid_kappa(x5) -> float:
    """Eq. 42 for the parameters (A, B, C, H, I)."""
    x5 = _f64(x5).ravel()
    return float(_load().oracle_paraboloid_kappa(_ptr(x5)))


def curvature_cell(phi27, flags: int = 0, iface27=None, nn=None):
    """Curvature of one stencil (Sec. 4.2, Appendix B: Eqs. 36, 38, 42);
    returns (kappa, fit_dim, n_points).

    ``nn`` (27 x 3, optional, used with NEIGHBOR_NORMAL): the normal of each
    neighbour's PLIC plane; zero rows mean the centre normal."""
    s = _f64(phi27).ravel()
    dim = ctypes.c_int(0)
    npt = ctypes.c_int(0)
    mask = None
    if iface27 is not None:
        mask = np.ascontiguousarray(np.asarray(iface27, dtype=np.int32).ravel())
    nn81 = None if nn is None else _f64(nn).ravel()
    k = _load().oracle_curvature_cell(_ptr(s), None if mask is None else _ptr(mask),
                                      None if nn81 is None else _ptr(nn81),
                                      flags, ctypes.byref(dim), ctypes.byref(npt))
    return float(k), dim.value, npt.value


def cm_normal(phi27):
    """Centre-of-mass normal (Appendix B, unit weights); None if undefined."""
    s = _f64(phi27).ravel()
    assert s.size == 27
    n = np.empty(3, np.float64)
    ok = _load().oracle_cm_normal(_ptr(s), _ptr(n))
    return n if ok else None


def normals(phi, idx, flags: int = 0):
    """PY (Eq. 38; or the CM normal of Appendix B with NORMAL_CM) normals of
    the listed cells, shape (3, k)."""
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32))
    nz, ny, nx = phi.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    out = np.empty((3, idx.size), np.float64)
    _load().oracle_normal_batch(_ptr(phi), nx, ny, nz, _ptr(idx), idx.size, flags,
                                _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
    return out


def sphere_radius() -> float:
    """Radius of the unit-volume ball of Sec. 3."""
    return (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)


def sphere_volume(d0):
    """Sec. 3: volume of the unit-volume ball below a plane at distance d0."""
    d0 = _f64(d0).ravel()
    out = np.empty(d0.shape, np.float64)
    _load().oracle_sphere_volume_batch(_ptr(d0), _ptr(out), d0.size)
    return out


def sphere_offset(V0):
    """Sec. 3: the inverse of :func:`sphere_volume` by bisection, FP64."""
    V0 = _f64(V0).ravel()
    out = np.empty(V0.shape, np.float64)
    _load().oracle_sphere_offset_batch(_ptr(V0), _ptr(out), V0.size)
    return out


def interface_cells(phi) -> np.ndarray:
    """Linear indices (x + nx*(y + ny*z)) of curvature cells, ascending.

    A curvature cell is an interface cell (0 < phi < 1, Eq. 33) whose 26
    neighbours all lie inside the field.  ``phi`` has shape (nz, ny, nx)."""
    phi = np.asarray(phi)
    mask = (phi > 0) & (phi < 1)
    mask[0, :, :] = mask[-1, :, :] = False
    mask[:, 0, :] = mask[:, -1, :] = False
    mask[:, :, 0] = mask[:, :, -1] = False
    return np.flatnonzero(mask.ravel()).astype(np.int32)


def curvature(phi, idx, flags: int = 0, with_cond: bool = False):
    """kappa (FP64) for the curvature cells ``idx`` of the FP32 field ``phi``
    (the curvature step of Sec. 4.2 and Appendix B).

    ``phi`` has shape (nz, ny, nx).  Returns (kappa, fit_dim, n_points), and
    with ``with_cond`` also the fit's conditioning: the smallest leading pivot
    of its normal matrix divided by the matrix's trace (1 without a fit)."""
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32))
    nz, ny, nx = phi.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    kappa = np.empty(idx.size, np.float64)
    dim = np.empty(idx.size, np.int32)
    npt = np.empty(idx.size, np.int32)
    cond = np.empty(idx.size, np.float64) if with_cond else None
    _load().oracle_curvature_batch(_ptr(phi), nx, ny, nz, _ptr(idx), idx.size, flags,
                                   _ptr(kappa), _ptr(dim), _ptr(npt),
                                   None if cond is None else _ptr(cond))
    return (kappa, dim, npt, cond) if with_cond else (kappa, dim, npt)


def curvature_grad_fd(phi, idx, w, h: float = 1e-4, flags: int = 0):
    """Central-difference gradient of sum_k w_k kappa_k w.r.t. the dense field
    (the adjoint of the curvature step of Sec. 4.2, by brute force)."""
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32))
    nz, ny, nx = phi.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    w = _f64(w).ravel()
    assert w.size == idx.size
    g = np.empty(phi.size, np.float64)
    _load().oracle_curvature_grad_fd(_ptr(phi), nx, ny, nz, _ptr(idx), idx.size, _ptr(w),
                                     float(h), flags, _ptr(g))
    return g.reshape(phi.shape)
