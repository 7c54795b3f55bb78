"""Hierarchical active-cell prediction (Algorithm 1) run level by level over octree cubes, and the
dense ground truth it is measured against.  float64.

Test infrastructure: see the package docstring.

Algorithm 1 bounds a node, culls it when the iso-value lies outside its bound
(upper < c or lower > c), returns it as an active cell at the maximum depth, and otherwise splits
it.  The paper splits k-d style along the widest axis and keeps depths a multiple of three so the
leaves are cubes (Sec. IV-D); here the tree is visited breadth first and only cube nodes
(every third k-d depth, i.e. octree levels) are bounded.  Level ``l`` has cells ``(i, j, k)`` in
``[0, 2^l)^3`` with box ``lo = -1 + 2 (i, j, k) / 2^l``, ``hi = lo + 2 / 2^l``.  Several
iso-values are handled at once: a cell carries a bit set of the iso-values it may contain, a
child inherits its parent's set, and the bound (which does not depend on the iso-value) is read
once per cell.  Equality with a bound endpoint keeps the cell (the cull test is strict).
"""
from __future__ import annotations

import numpy as np

from . import affine


def cell_box(ijk, level):
    ijk = np.asarray(ijk, dtype=np.float64).reshape(-1, 3)
    size = 2.0 / float(1 << level)
    lo = -1.0 + ijk * size
    return lo, lo + size


CHILD_OFF = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.int64)


def children(ijk):
    """The 8 children of each cell, child ``c`` at ``2 (i, j, k) + (c & 1, c >> 1 & 1, c >> 2 & 1)``."""
    ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
    return (2 * ijk[:, None, :] + CHILD_OFF[None, :, :]).reshape(-1, 3)


def iso_bits(lower, upper, isos):
    """Bit q set iff lower <= iso_q <= upper (not culled by Algorithm 1's test)."""
    isos = np.asarray(isos, dtype=np.float64)
    keep = (lower[:, None] <= isos[None, :]) & (isos[None, :] <= upper[:, None])
    return (keep.astype(np.int64) << np.arange(isos.shape[0])[None, :]).sum(axis=1)


def extract_active(layers, max_level, isos, mode, k=3.0, batch=64, start_level=0, start_cells=None,
                   start_masks=None, act="relu"):
    """Run the level loop.  Returns a list with one dict per level:
    ``ijk`` (n, 3) cells bounded at that level, ``mask_in`` their inherited iso sets, ``lower``,
    ``upper`` their bounds, ``mask`` the surviving sets.  The last level's surviving cells are the
    predicted active cells."""
    isos = np.asarray(isos, dtype=np.float64)
    full = (1 << isos.shape[0]) - 1
    if start_cells is None:
        ijk = np.zeros((1, 3), dtype=np.int64)
        masks = np.array([full], dtype=np.int64)
    else:
        ijk = np.asarray(start_cells, dtype=np.int64).reshape(-1, 3)
        masks = np.asarray(start_masks, dtype=np.int64) if start_masks is not None else \
            np.full(ijk.shape[0], full, dtype=np.int64)
    levels = []
    for level in range(start_level, max_level + 1):
        lo, hi = cell_box(ijk, level)
        if ijk.shape[0]:
            centre, spread = affine.bound(layers, lo, hi, mode, batch=batch, act=act)
        else:
            centre = spread = np.zeros(0)
        lower, upper = affine.interval(centre, spread, mode, k)
        new = masks & iso_bits(lower, upper, isos)
        levels.append(dict(level=level, ijk=ijk, mask_in=masks, centre=centre, spread=spread,
                           lower=lower, upper=upper, mask=new))
        keep = new != 0
        if level < max_level:
            ijk = children(ijk[keep])
            masks = np.repeat(new[keep], 8)
    return levels


def kd_box(ijk, depth):
    """Box of k-d cells at ``depth`` of Algorithm 1: the widest side is bisected at every depth (x, then
    y, then z on ties, starting from the cube [-1, 1]^3), so axis a has been split
    ``(depth + 2 - a) // 3`` times and the cell ``(i, j, k)`` spans ``-1 + 2 i_a / 2^splits_a`` onwards."""
    ijk = np.asarray(ijk, dtype=np.float64).reshape(-1, 3)
    splits = np.array([(depth + 2 - a) // 3 for a in range(3)])
    size = 2.0 / (2.0 ** splits)
    lo = -1.0 + ijk * size[None, :]
    return lo, lo + size[None, :]


def kd_extract_active(layers, max_level, isos, mode, k=3.0, batch=64):
    """Algorithm 1 literally, breadth first: every node of depths 0 .. 3 max_level is bounded, a node
    keeps the iso-values whose value lies inside its bound, and a surviving node below the maximum
    depth is split in two along its widest side (``depth mod 3`` is that axis).  The leaves at depth
    3 max_level are the cubes of the octree's finest level.  Returns one dict per depth as
    extract_active does."""
    isos = np.asarray(isos, dtype=np.float64)
    full = (1 << isos.shape[0]) - 1
    ijk = np.zeros((1, 3), dtype=np.int64)
    masks = np.array([full], dtype=np.int64)
    depths = []
    D = 3 * max_level
    for depth in range(D + 1):
        lo, hi = kd_box(ijk, depth)
        if ijk.shape[0]:
            centre, spread = affine.bound(layers, lo, hi, mode, batch=batch)
        else:
            centre = spread = np.zeros(0)
        lower, upper = affine.interval(centre, spread, mode, k)
        new = masks & iso_bits(lower, upper, isos)
        depths.append(dict(depth=depth, ijk=ijk, mask_in=masks, centre=centre, spread=spread,
                           lower=lower, upper=upper, mask=new))
        keep = new != 0
        if depth < D:
            axis = depth % 3
            par = ijk[keep]
            kids = np.repeat(par, 2, axis=0)
            kids[:, axis] = 2 * kids[:, axis] + np.tile(np.array([0, 1]), par.shape[0])
            ijk = kids
            masks = np.repeat(new[keep], 2)
    return depths


def active_cells(levels):
    last = levels[-1]
    keep = last["mask"] != 0
    return last["ijk"][keep], last["mask"][keep]


def lattice_points(R):
    """All (R+1)^3 lattice points of the finest grid, x fastest, as coordinates -1 + 2 i / R."""
    t = -1.0 + 2.0 * np.arange(R + 1) / R
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def fpr_fnr(pred_ijk, true_ijk, R):
    """False-positive and false-negative rates of predicted active cells (Sec. V-A.3):
    FPR = FP / (FP + TN), FNR = FN / (FN + TP) over the R^3 cells."""
    def key(a):
        a = np.asarray(a, dtype=np.int64).reshape(-1, 3)
        return (a[:, 2] * R + a[:, 1]) * R + a[:, 0]
    p = np.unique(key(pred_ijk))
    t = np.unique(key(true_ijk))
    tp = np.intersect1d(p, t).size
    fp = p.size - tp
    fn = t.size - tp
    tn = R ** 3 - tp - fp - fn
    fpr = fp / (fp + tn) if fp + tn else 0.0
    fnr = fn / (fn + tp) if fn + tp else 0.0
    return fpr, fnr
