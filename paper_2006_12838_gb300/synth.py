"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random draws and geometry only -- no PLIC arithmetic (no
volume, offset, normal or curvature formula).  It serves both the GPU path
(bench, tests) and the oracle side (tests, CPU baseline), which is why it is a
module of its own and imports neither.

Recipes (seeds fixed per workload):

* :func:`plic_cells` -- unit normals n = g/|g|, g ~ N(0, I3), fill fractions
  V0 ~ U[0, 1], optionally with a tail of edge cases (V0 in {0, 1, 1/2},
  axis-aligned normals, one or two zero components, |nx| = |ny| = |nz|) and a
  share of "vertex" cells whose plane offset d0 passes within 1e-6 of a cube
  vertex.  A vertex crossing is exactly where the intersection polygon changes
  shape, i.e. where the five intersection cases of Sec. 2.2 meet; the caller
  turns those d0 into V0 with its own forward volume.
* :func:`paper_normals` -- the normal sets of the paper's CPU and GPU
  benchmarks (Sec. 2.5: one axis normal, one diagonal 2D normal, random 2D
  normals in the x-y plane, random 3D normals).
* :func:`fill_spheres`, :func:`fill_ellipsoid`, :func:`fill_cylinder` -- VOF
  fill fields phi (Eq. 33) by exact sub-cell integration: the fraction of the
  16^3 midpoints of a cell that lie strictly inside the shape.  Centres and
  radii are quantised to 1/32 of a cell, so every inside test is exact integer
  arithmetic and the field is the same on any device; fills are multiples of
  1/4096.
* :func:`curvature_field`, :func:`adjoint_field`, :func:`batched_fields` --
  the curvature workloads (8 spheres in 256^3; one noisy ellipsoid in 128^3;
  64 uneven fields with 1-20 droplets each).
"""
from __future__ import annotations

import math

import numpy as np
import torch

SUB = 16            # sub-samples per cell edge
Q = 32              # quantum: coordinates are integers in units of 1/Q cell


# ---------------------------------------------------------------------------
# PLIC cell batches
# ---------------------------------------------------------------------------
def gaussian_normals(rng: np.random.Generator, m: int) -> np.ndarray:
    """m unit normals g/|g|, g ~ N(0, I3) (uniform on the sphere), shape (3, m)."""
    g = rng.standard_normal((3, m))
    r2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2]
    r2[r2 == 0] = 1.0
    g *= 1.0 / np.sqrt(r2)
    return g


def edge_case_cells(rng: np.random.Generator, m: int):
    """m edge-case cells in five equal parts: V0 in {0, 1, 1/2} with random n;
    axis-aligned n with random V0 (including 0 and 1); one zero component; two
    zero components; |nx| = |ny| = |nz| with all 8 sign patterns.
    Returns (n of shape (3, m), V0)."""
    parts = np.array_split(np.arange(m), 5)
    n = np.empty((3, m))
    V0 = np.empty(m)
    # (a) special V0, random n
    i = parts[0]
    n[:, i] = gaussian_normals(rng, i.size)
    V0[i] = rng.choice([0.0, 1.0, 0.5], i.size)
    # (b) axis-aligned n, random V0 with 0/1 included
    i = parts[1]
    ax = rng.integers(0, 3, i.size)
    n[:, i] = 0.0
    n[ax, i] = rng.choice([-1.0, 1.0], i.size)
    V0[i] = rng.random(i.size)
    V0[i[::7]] = 0.0
    V0[i[3::7]] = 1.0
    # (c) one zero component (random 2D normal in a coordinate plane)
    i = parts[2]
    g = gaussian_normals(rng, i.size)
    g[rng.integers(0, 3, i.size), np.arange(i.size)] = 0.0
    n[:, i] = g / np.sqrt((g * g).sum(0))
    V0[i] = rng.random(i.size)
    # (d) two zero components
    i = parts[3]
    ax = rng.integers(0, 3, i.size)
    n[:, i] = 0.0
    n[ax, i] = rng.choice([-1.0, 1.0], i.size)
    V0[i] = rng.random(i.size)
    V0[i[::5]] = rng.choice([0.0, 1.0], i[::5].size)
    # (e) |nx| = |ny| = |nz| = 1/sqrt 3, all sign patterns
    i = parts[4]
    signs = np.array([[sx, sy, sz] for sx in (1, -1) for sy in (1, -1) for sz in (1, -1)], float)
    n[:, i] = (signs[np.arange(i.size) % 8] / math.sqrt(3.0)).T
    V0[i] = rng.random(i.size)
    return n, V0


def plic_cells(m: int, seed, edge_frac: float = 0.0, vertex_frac: float = 0.0,
               vertex_eps: float = 1e-6, boundary_frac: float = 0.0, boundary_eps: float = 1e-6):
    """Normals and fill fractions for m PLIC cells (FP64 numpy arrays).

    Returns dict(n=(3, m) [rows nx, ny, nz], V0=(m,), vertex=(m,) bool,
    d0_vertex=(m,)).  For ``vertex`` cells V0 is NaN and ``d0_vertex`` holds a
    plane offset that passes within ``vertex_eps`` of a cube vertex (other
    than the two extreme vertices where V0 is 0 or 1); the caller computes
    V0 = V0(n, d0_vertex) with its own forward volume.  Edge cases occupy the
    last ``edge_frac`` share; each other cell is a vertex cell with probability
    ``vertex_frac``.

    ``boundary`` cells (probability ``boundary_frac`` among the cells that are
    neither edge nor vertex cells) sit at the boundaries of cases (3), (4) and
    (5) in V rather than in d: with the components of |n| sorted,
    n1 <= n2 <= n3, the plane through the cube corner at the far end of the
    n2 axis ends case (2) and starts case (3); the one at the end of the n3
    axis ends case (3) and starts case (4) when n3 < n1 + n2, else the plane
    through the corner n1 + n2 ends case (3) and starts case (5).  One of the
    two boundaries is drawn with probability 1/2; ``d0_boundary`` is that
    plane's offset, ``dV`` ~ U[-boundary_eps, boundary_eps] and ``mirror`` a
    fair coin.  The caller forms V = V0(n, d0_boundary) with its own forward
    volume, then V0 = clip(V + dV, 0, 1/2), mirrored to 1 - V0 where
    ``mirror`` is set; V0 of these cells is NaN here."""
    rng = np.random.default_rng(seed)
    n = gaussian_normals(rng, m)
    V0 = rng.random(m)
    m_edge = int(round(edge_frac * m))
    if m_edge:
        ne, Ve = edge_case_cells(rng, m_edge)
        n[:, m - m_edge:] = ne
        V0[m - m_edge:] = Ve
    vertex = np.zeros(m, bool)
    d0v = np.full(m, np.nan)
    if vertex_frac > 0:
        pool = m - m_edge
        vertex[:pool] = rng.random(pool) < vertex_frac
        pick = np.flatnonzero(vertex)
        k = pick.size
        npk = n[:, pick]
        sgn_n = np.where(npk >= 0, 1.0, -1.0)
        # vertex v = s/2 with a sign pattern s that is neither +sign(n) nor -sign(n)
        pat = rng.integers(1, 7, k)                   # 3-bit patterns 1..6
        flips = np.stack([(pat >> b) & 1 for b in range(3)], 0).astype(float)
        s = sgn_n * (1.0 - 2.0 * flips)
        d0v[pick] = 0.5 * (npk * s).sum(0) + rng.uniform(-vertex_eps, vertex_eps, k)
        V0[pick] = np.nan
    boundary = np.zeros(m, bool)
    d0b = np.full(m, np.nan)
    dV = np.zeros(m)
    mirror = np.zeros(m, bool)
    if boundary_frac > 0:
        pool = m - m_edge
        boundary[:pool] = (~vertex[:pool]) & (rng.random(pool) < boundary_frac)
        pick = np.flatnonzero(boundary)
        k = pick.size
        a = np.abs(n[:, pick])
        order = np.argsort(a, axis=0, kind="stable")        # axes of n1, n2, n3
        srt = np.take_along_axis(a, order, 0)
        cols = np.arange(k)
        # vertex offsets from the corner -sign(n)/2 (where V0 = 0): a corner
        # reached by moving along the chosen axes
        upper = rng.random(k) < 0.5
        tall = srt[2] >= srt[0] + srt[1]
        move = np.zeros((3, k), bool)
        move[order[1], cols] = ~upper                        # case (2)/(3): the n2 axis
        move[order[2], cols] = upper & ~tall                 # case (3)/(4): the n3 axis
        move[order[0], cols] |= upper & tall                 # case (3)/(5): n1 and n2
        move[order[1], cols] |= upper & tall
        sgn = np.where(n[:, pick] >= 0, 1.0, -1.0)
        x = -0.5 * sgn + np.where(move, sgn, 0.0)
        d0b[pick] = (n[:, pick] * x).sum(0)
        dV[pick] = rng.uniform(-boundary_eps, boundary_eps, k)
        mirror[pick] = rng.random(k) < 0.5
        V0[pick] = np.nan
    return {"n": n, "V0": V0, "vertex": vertex, "d0_vertex": d0v,
            "boundary": boundary, "d0_boundary": d0b, "dV": dV, "mirror": mirror}


def boundary_fill(Vb, dV, mirror):
    """V0 of boundary cells from the forward volume Vb of their plane
    (see :func:`plic_cells`): clip(Vb + dV, 0, 1/2), mirrored where asked."""
    V = np.clip(Vb + dV, 0.0, 0.5)
    return np.where(mirror, 1.0 - V, V)


def plic_cells_chunks(m: int, seed: int, chunk: int = 1 << 22, **kw):
    """The recipe of :func:`plic_cells` for large m, generated in chunks of
    ``chunk`` cells; chunk i uses its own generator seeded with (seed, i), so
    any chunk can be regenerated alone.  Yields (start, cells_dict)."""
    for i, start in enumerate(range(0, m, chunk)):
        k = min(chunk, m - start)
        yield start, plic_cells(k, seed=np.random.SeedSequence([seed, i]), **kw)


def paper_normals(m: int, seed: int) -> np.ndarray:
    """Normal set (shape (3, m)) of the paper's benchmarks (Sec. 2.5): (1,0,0),
    (1/sqrt2, 1/sqrt2, 0), then one eighth minus two random 2D normals in the
    x-y plane (510 of 4096; 8 388 606 of 67 108 864), the rest random 3D."""
    rng = np.random.default_rng(seed)
    n = np.empty((3, m))
    n[:, 0] = [1.0, 0.0, 0.0]
    n[:, 1] = [1 / math.sqrt(2), 1 / math.sqrt(2), 0.0]
    m2 = m // 8 - 2
    phi = rng.uniform(0, 2 * math.pi, m2)
    n[:, 2:2 + m2] = np.stack([np.cos(phi), np.sin(phi), np.zeros(m2)], 0)
    n[:, 2 + m2:] = gaussian_normals(rng, m - 2 - m2)
    return n


# ---------------------------------------------------------------------------
# Fill fields by exact sub-cell integration
# ---------------------------------------------------------------------------
def _popcount16(x: torch.Tensor) -> torch.Tensor:
    x = x - ((x >> 1) & 0x5555)
    x = (x & 0x3333) + ((x >> 2) & 0x3333)
    x = (x + (x >> 4)) & 0x0F0F
    return (x + (x >> 8)) & 0x1F


def _isqrt(q: torch.Tensor) -> torch.Tensor:
    """floor(sqrt(q)) for 0 <= q < 2**24, exact (float estimate + correction)."""
    s = torch.floor(torch.sqrt(q.to(torch.float32))).to(torch.int64)
    s = torch.where((s + 1) * (s + 1) <= q, s + 1, s)
    s = torch.where(s * s > q, s - 1, s)
    return s


def _quantise(x) -> int:
    return int(round(float(x) * Q))


def fill_spheres(shape, spheres, device="cpu") -> torch.Tensor:
    """Fill field of the union of spheres.

    ``shape`` = (nz, ny, nx); cell (x, y, z) has its centre at (x, y, z).
    ``spheres`` = iterable of (cx, cy, cz, R) in cell units (quantised to 1/32).
    phi = (number of the 16^3 sub-cell midpoints strictly inside the union)/4096.
    Per sub-column (sx, sy) the inside z-range of a sphere is an integer
    interval, kept as a 16-bit mask; masks of overlapping spheres are OR-ed."""
    nz, ny, nx = shape
    dev = torch.device(device)
    phi = torch.zeros(shape, dtype=torch.float32, device=dev)
    sph = [tuple(_quantise(v) for v in s) for s in spheres]
    off = (2 * torch.arange(SUB, device=dev, dtype=torch.int64) + 1 - SUB)   # in 1/32 units
    half = SUB - 1                                                            # 15/32
    pair_cells, pair_sph = [], []
    for si, (cx, cy, cz, R) in enumerate(sph):
        lo = [max(0, (c - R) // Q - 1) for c in (cx, cy, cz)]
        hi = [min(e - 1, (c + R) // Q + 1) for c, e in zip((cx, cy, cz), (nx, ny, nz))]
        if any(h < l for l, h in zip(lo, hi)):
            continue
        zs = torch.arange(lo[2], hi[2] + 1, device=dev)
        ys = torch.arange(lo[1], hi[1] + 1, device=dev)
        xs = torch.arange(lo[0], hi[0] + 1, device=dev)
        Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
        dx = (X * Q - cx).abs()
        dy = (Y * Q - cy).abs()
        dz = (Z * Q - cz).abs()
        R2 = R * R
        full = (dx + half) ** 2 + (dy + half) ** 2 + (dz + half) ** 2 < R2
        near = ((dx - half).clamp(min=0) ** 2 + (dy - half).clamp(min=0) ** 2
                + (dz - half).clamp(min=0) ** 2) < R2
        part = near & ~full
        sub = phi[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        sub[full] = 1.0
        lin = (Z * ny + Y) * nx + X
        pc = lin[part]
        pair_cells.append(pc)
        pair_sph.append(torch.full_like(pc, si))
    if not pair_cells:
        return phi
    cells = torch.cat(pair_cells)
    sids = torch.cat(pair_sph)
    flat = phi.view(-1)
    keep = flat[cells] < 1.0
    cells, sids = cells[keep], sids[keep]
    if cells.numel() == 0:
        return phi
    order = torch.argsort(cells, stable=True)
    cells, sids = cells[order], sids[order]
    ucell, inv, counts = torch.unique_consecutive(cells, return_inverse=True, return_counts=True)
    start = torch.cumsum(counts, 0) - counts
    rank = torch.arange(cells.numel(), device=dev) - start[inv]
    sph_t = torch.tensor(sph, dtype=torch.int64, device=dev)
    masks = torch.zeros((ucell.numel(), SUB, SUB), dtype=torch.int64, device=dev)
    chunk = 1 << 18
    for r in range(int(counts.max().item())):
        sel = torch.nonzero(rank == r).squeeze(1)
        for c0 in range(0, sel.numel(), chunk):
            s = sel[c0:c0 + chunk]
            c = cells[s]
            cx, cy, cz, R = sph_t[sids[s]].unbind(1)
            x = c % nx
            y = (c // nx) % ny
            z = c // (nx * ny)
            DX = x[:, None] * Q + off[None, :] - cx[:, None]          # (k, 16) sub-x
            DY = y[:, None] * Q + off[None, :] - cy[:, None]
            q = (R * R)[:, None, None] - DX[:, :, None] ** 2 - DY[:, None, :] ** 2
            pos = q > 0
            srt = _isqrt((q - 1).clamp(min=0))                        # |dz| <= srt  <=>  dz^2 < q
            base = (z * Q - cz)[:, None, None]                        # dz of sub-z = base + off
            # sub index j has dz = base + 2j + 1 - 16; need -srt <= dz <= srt
            jlo = torch.div(-srt - base + SUB - 1 + 1, 2, rounding_mode="floor")
            jhi = torch.div(srt - base + SUB - 1, 2, rounding_mode="floor")
            jlo = jlo.clamp(0, SUB)
            jhi = jhi.clamp(-1, SUB - 1)
            ok = pos & (jhi >= jlo)
            m = ((1 << (jhi + 1).clamp(min=0)) - 1) & ~((1 << jlo) - 1)
            m = torch.where(ok, m, torch.zeros_like(m))
            masks[inv[s]] |= m
    cnt = _popcount16(masks).sum(dim=(1, 2))
    flat[ucell] = cnt.to(torch.float32) / float(SUB ** 3)
    return phi


def fill_ellipsoid(shape, center, semi, device="cpu", chunk=4096) -> torch.Tensor:
    """Fill field of an axis-aligned ellipsoid (exact integer sub-sampling)."""
    nz, ny, nx = shape
    dev = torch.device(device)
    c = [_quantise(v) for v in center]
    a = [_quantise(v) for v in semi]
    w = [(a[1] * a[2]) ** 2, (a[0] * a[2]) ** 2, (a[0] * a[1]) ** 2]
    rhs = (a[0] * a[1] * a[2]) ** 2
    phi = torch.zeros(shape, dtype=torch.float32, device=dev)
    zs, ys, xs = (torch.arange(e, device=dev) for e in (nz, ny, nx))
    Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
    d = [(X * Q - c[0]).abs(), (Y * Q - c[1]).abs(), (Z * Q - c[2]).abs()]
    half = SUB - 1
    far = sum(wk * (dk + half) ** 2 for wk, dk in zip(w, d)) < rhs
    near = sum(wk * (dk - half).clamp(min=0) ** 2 for wk, dk in zip(w, d)) < rhs
    phi[far] = 1.0
    part = torch.nonzero((near & ~far).view(-1)).squeeze(1)
    off = (2 * torch.arange(SUB, device=dev, dtype=torch.int64) + 1 - SUB)
    flat = phi.view(-1)
    for c0 in range(0, part.numel(), chunk):
        p = part[c0:c0 + chunk]
        x = p % nx
        y = (p // nx) % ny
        z = p // (nx * ny)
        DX = (x[:, None] * Q + off - c[0])[:, :, None, None]
        DY = (y[:, None] * Q + off - c[1])[:, None, :, None]
        DZ = (z[:, None] * Q + off - c[2])[:, None, None, :]
        inside = w[0] * DX ** 2 + w[1] * DY ** 2 + w[2] * DZ ** 2 < rhs
        flat[p] = inside.sum(dim=(1, 2, 3)).to(torch.float32) / float(SUB ** 3)
    return phi


def fill_cylinder(shape, axis: int, center2, R, device="cpu") -> torch.Tensor:
    """Fill field of an infinite circular cylinder along ``axis`` (0=x, 1=y,
    2=z) through the point ``center2`` of the perpendicular plane (ordered as
    the two remaining axes in x, y, z order).  Exact integer sub-sampling."""
    nz, ny, nx = shape
    dev = torch.device(device)
    other = [k for k in range(3) if k != axis]
    cu, cv = (_quantise(v) for v in center2)
    Rq = _quantise(R)
    idx = torch.meshgrid(*(torch.arange(e, device=dev) for e in (nz, ny, nx)), indexing="ij")
    coord = [idx[2], idx[1], idx[0]]                    # x, y, z
    U, V = coord[other[0]], coord[other[1]]
    off = (2 * torch.arange(SUB, device=dev, dtype=torch.int64) + 1 - SUB)
    DU = (U[..., None] * Q + off - cu)[..., :, None]
    DV = (V[..., None] * Q + off - cv)[..., None, :]
    inside = DU ** 2 + DV ** 2 < Rq * Rq
    return inside.sum(dim=(-1, -2)).to(torch.float32) / float(SUB * SUB)


def curvature_field(seed: int = 3, edge: int = 256, n_spheres: int = 8,
                    rmin: float = 6.0, rmax: float = 40.0, device="cpu"):
    """Curvature workload: ``n_spheres`` spheres with R ~ U[rmin, rmax] and
    centres ~ U[R+2, edge-2-R] per axis, union fill on an edge^3 FP32 field."""
    rng = np.random.default_rng(seed)
    spheres = []
    for _ in range(n_spheres):
        R = rng.uniform(rmin, rmax)
        c = rng.uniform(R + 2, edge - 2 - R, 3)
        spheres.append((c[0], c[1], c[2], R))
    phi = fill_spheres((edge, edge, edge), spheres, device=device)
    return phi, spheres


def adjoint_field(seed: int = 4, edge: int = 128, semi=(12.0, 18.0, 24.0),
                  noise: float = 1e-3, device="cpu"):
    """Adjoint workload: one ellipsoid centred in an edge^3 field, with
    noise * N(0,1) added to the interface cells only and the result clamped to
    [2e-4, 1 - 2e-4] so that no interface flag flips under +-1e-4 steps.
    Returns (phi, w) with w ~ N(0,1) per curvature cell (ascending index)."""
    c = (edge / 2, edge / 2, edge / 2)
    phi = fill_ellipsoid((edge, edge, edge), c, semi, device="cpu")
    rng = np.random.default_rng(seed)
    p = phi.numpy()
    iface = (p > 0) & (p < 1)
    p[iface] = np.clip(p[iface] + noise * rng.standard_normal(int(iface.sum())),
                       2e-4, 1 - 2e-4).astype(np.float32)
    inner = np.zeros_like(iface)
    inner[1:-1, 1:-1, 1:-1] = iface[1:-1, 1:-1, 1:-1]
    w = rng.standard_normal(int(inner.sum()))
    return torch.from_numpy(p).to(device), w


def batched_fields(seed: int = 5, n_fields: int = 64, edges=(32, 64, 96, 128, 192, 256),
                   device="cpu", max_fields=None):
    """Batched workload: ``n_fields`` cubic fields with edge drawn from
    ``edges``, each with 1-20 droplets of radius U[4, 40] and centres
    U[0, edge)^3 (overlap and clipping by the field boundary allowed)."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(n_fields):
        e = int(rng.choice(edges))
        k = int(rng.integers(1, 21))
        spheres = []
        for _ in range(k):
            R = rng.uniform(4.0, 40.0)
            c = rng.uniform(0, e, 3)
            spheres.append((c[0], c[1], c[2], R))
        if max_fields is not None and f >= max_fields:
            continue
        out.append((fill_spheres((e, e, e), spheres, device=device), spheres))
    return out
