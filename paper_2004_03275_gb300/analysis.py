"""Host-side analysis of solver output (numpy; not part of the stage path).

``project_uniform`` maps a field on the leaves of a block tree to one uniform grid,
so that two runs whose trees differ (a float32 run may flag a block differently from
a float64 one) can be compared cell by cell: leaves coarser than the target grid are
replicated (piecewise constant), finer ones averaged.
"""
from __future__ import annotations

import numpy as np


def project_uniform(level, coords, field, ndim: int, block_nx: int, base, level_of_grid: int):
    """Project a per-leaf field onto the uniform grid of tree level ``level_of_grid``.

    level, coords: the leaves (levels from 1, integer block coordinates at the leaf's level);
    field: (nleaves, block_nx**ndim), x fastest within a block; base: blocks per dimension
    on level 1.  Returns an array of shape (N_z, N_y, N_x) (last ndim axes), N_d = base[d] *
    block_nx * 2**(level_of_grid - 1).
    """
    level = np.asarray(level)
    coords = np.asarray(coords).reshape(len(level), -1)
    field = np.asarray(field, dtype=np.float64).reshape(len(level), *([block_nx] * ndim))
    shape = tuple(int(base[d]) * block_nx * 2 ** (level_of_grid - 1) for d in reversed(range(ndim)))
    out = np.zeros(shape)
    filled = np.zeros(shape, dtype=bool)
    for l, c, f in zip(level, coords, field):
        if l <= level_of_grid:
            r = 2 ** (level_of_grid - l)  # target cells per leaf cell and dimension
            blk = f
            for ax in range(ndim):
                blk = np.repeat(blk, r, axis=ax)
            n = block_nx * r
            sl = tuple(slice(int(c[d]) * n, int(c[d]) * n + n) for d in reversed(range(ndim)))
        else:
            r = 2 ** (l - level_of_grid)  # leaf cells per target cell and dimension
            m = block_nx // r
            blk = f.reshape(*sum(([m, r] for _ in range(ndim)), [])).mean(axis=tuple(range(1, 2 * ndim, 2)))
            sl = tuple(slice(int(c[d]) * m, int(c[d]) * m + m) for d in reversed(range(ndim)))
        if filled[sl].any():
            raise ValueError("leaves overlap")
        out[sl] = blk
        filled[sl] = True
    if not filled.all():
        raise ValueError("leaves do not cover the domain")
    return out


def l1_relative(a, ref):
    """sum |a - ref| / sum |ref| (the normalised L1 error)."""
    a, ref = np.asarray(a, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float(np.abs(a - ref).sum() / np.abs(ref).sum())
