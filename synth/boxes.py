"""Seeded random axis-aligned boxes and octree cell lists inside [-1, 1]^3."""
from __future__ import annotations

import numpy as np


def random_boxes(n, seed, log2_half_min=-10.0, log2_half_max=-1.0):
    """``n`` boxes with log-uniform half-widths in ``[2^log2_half_min, 2^log2_half_max]`` per axis
    and centres uniform so that the box stays inside the domain.  Returns float32 ``lo, hi`` (n, 3)."""
    rng = np.random.default_rng(seed)
    h = 2.0 ** rng.uniform(log2_half_min, log2_half_max, size=(n, 3))
    c = rng.uniform(-1.0 + h, 1.0 - h)
    lo = (c - h).astype(np.float32)
    hi = (c + h).astype(np.float32)
    return lo, hi


def random_cubes(n, seed, level_min=1, level_max=9):
    """``n`` octree cells (i, j, k, level) with level uniform in [level_min, level_max];
    returns int arrays ``ijk`` (n, 3), ``level`` (n,) and their float32 ``lo, hi``."""
    rng = np.random.default_rng(seed)
    level = rng.integers(level_min, level_max + 1, size=n)
    ijk = np.floor(rng.uniform(0, 1, size=(n, 3)) * (1 << level)[:, None]).astype(np.int64)
    lo, hi = cell_boxes(ijk, level)
    return ijk, level, lo, hi


def cell_boxes(ijk, level):
    """Exact dyadic boxes of octree cells: lo = -1 + 2 i / 2^level, hi = lo + 2 / 2^level."""
    ijk = np.asarray(ijk, dtype=np.float64)
    size = 2.0 / (2.0 ** np.asarray(level, dtype=np.float64))
    size = np.broadcast_to(np.reshape(size, (-1, 1)) if np.ndim(size) else size, ijk.shape)
    lo = -1.0 + ijk * size
    hi = lo + size
    return lo.astype(np.float32), hi.astype(np.float32)


def pack_codes(ijk):
    """Cell code used by the C interface: i | j << 10 | k << 20 (levels up to 10)."""
    ijk = np.asarray(ijk, dtype=np.uint32)
    return (ijk[:, 0] | (ijk[:, 1] << 10) | (ijk[:, 2] << 20)).astype(np.uint32)


def unpack_codes(codes):
    codes = np.asarray(codes, dtype=np.uint32)
    return np.stack([codes & 1023, (codes >> 10) & 1023, (codes >> 20) & 1023], axis=1).astype(np.int64)
