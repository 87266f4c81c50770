"""Helpers shared by the GPU parity tests."""
import numpy as np

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs

# FP64 GPU path vs the FP64 oracle, per cell: |a-b| <= RTOL * max(|b|, 1e-12 * max|b| of that variable)
RTOL64 = 1e-12


def rel_err(a, b):
    """Per-cell relative difference with the near-zero guard, max over everything."""
    a = np.asarray(a)
    b = np.asarray(b)
    # scale per variable (axis 1 of [leaf][var][cell])
    vmax = np.max(np.abs(b), axis=(0, 2), keepdims=True) if b.ndim == 3 else np.max(np.abs(b))
    den = np.maximum(np.abs(b), 1e-12 * np.maximum(vmax, 1e-300))
    return float(np.max(np.abs(a - b) / den))


def assert_parity(a, b, rtol=RTOL64, what=""):
    e = rel_err(a, b)
    assert e <= rtol, f"{what}: max relative difference {e:.3e} > {rtol:.1e}"
    return e


def pair(precision="fp64", **kw):
    """A GPU solver and an oracle grid with the same configuration."""
    s = amrvac.AmrSolver(precision=precision, **kw)
    okw = {k: v for k, v in kw.items() if k not in ("max_blocks",)}
    g = O.Grid(**okw)
    return s, g


def centres_for(lev, crd, kw):
    base = list(kw["base"]) + [1] * (3 - len(kw["base"]))
    xmin = list(kw.get("xmin", (0, 0, 0))) + [0] * 3
    xmax = list(kw.get("xmax", (1, 1, 1))) + [1] * 3
    return inputs.cell_centres(lev, crd, kw["ndim"], kw["block_nx"], base, xmin[:3], xmax[:3])


def assert_parity_scaled(a, b, rtol=RTOL64, floor=1e-3, what=""):
    """Trees with level jumps: the GPU adds the reflux correction after the stage
    update while the oracle uses the mean fine flux directly, so the two differ by
    round-off of O(1) terms.  Check |a-b| <= rtol * max|b_var| everywhere, and the
    per-cell relative bound for cells with |b| >= floor * max|b_var|."""
    a, b = np.asarray(a), np.asarray(b)
    vmax = np.max(np.abs(b), axis=(0, 2), keepdims=True)
    d = np.abs(a - b)
    e_abs = float(np.max(d / vmax))
    big = np.abs(b) >= floor * vmax
    e_rel = float(np.max(np.where(big, d / np.maximum(np.abs(b), 1e-300), 0.0)))
    assert e_abs <= rtol and e_rel <= rtol, f"{what}: scaled {e_abs:.3e}, relative (|b| large) {e_rel:.3e}"
    return e_abs, e_rel
