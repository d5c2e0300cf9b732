"""The per-cell curvature gate shared by the GPU curvature tests.

Every cell is gated: |kappa - kappa_ref| <= tol_c max(|kappa_ref|, 1/64) with
tol_c = max(tol, 4e-6 / cond_c), where cond_c is the conditioning of the
cell's least-squares fit as the oracle reports it (the smallest leading pivot
of the 5x5 normal matrix divided by its trace, Appendix B).  The kernels form
the normal, the frame and the points in FP32: the normal carries a relative
error of about 2e-6 (the parity of vof_normal), and the fit amplifies it by
up to 1/cond.  Cells with cond >= 0.04 -- nearly all of them -- keep the
plain tolerance; the nearly singular fits of a few cells (cond down to 1e-5
on the 64-field workload) get the amplified bound.  Cells whose fit has fewer
than 5 parameters (fewer than 5 interface neighbours, or a pivot at or below
1e-6 of the trace: the reduced-dimension reading of Appendix B) are gated the
same way.  Where the GPU's FP32 pivots and the oracle's FP64 ones fall on
opposite sides of that reduction threshold the two fits have different
dimensions and kappa differs by design, so a few cells over their tolerance
are allowed: they are counted and printed, and their number is bounded by 3,
or 1 in 10^4 of the cells.
"""
import numpy as np


COND_AMP = 4e-6


def gate_kappa(kappa, kref, dim, label, tol=1e-4, cond=None, max_straddle=None):
    kappa = np.asarray(kappa, np.float64)
    rel = np.abs(kappa - kref) / np.maximum(np.abs(kref), 1 / 64)
    tol_c = np.full(rel.size, tol) if cond is None else np.maximum(tol, COND_AMP / cond)
    full = dim == 5
    bad = rel > tol_c
    print("%s: cells %d (reduced fit %d, tolerance above %.0e: %d), max rel %.3e, p99.9 %.3e, "
          "max rel / tolerance %.3f, over tolerance %d" % (
              label, rel.size, (~full).sum(), tol, (tol_c > tol).sum(), rel.max() if rel.size else 0.0,
              np.percentile(rel, 99.9) if rel.size else 0.0,
              (rel / tol_c).max() if rel.size else 0.0, bad.sum()))
    for i in np.flatnonzero(bad)[:10]:
        print("   cell %d: kappa %.6e ref %.6e dim %d cond %s" % (
            i, kappa[i], kref[i], dim[i], "-" if cond is None else "%.2e" % cond[i]))
    limit = max(3, rel.size // 10000) if max_straddle is None else max_straddle
    assert bad.sum() <= limit, label
    return rel
