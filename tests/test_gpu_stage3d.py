"""GPU parity of the float32 3D stage for 16^3 leaves (xy march + z march kernels)
against the FP64 oracle.

Tolerances as for the 2D float32 kernels: after one step, per-cell difference
<= 1e-5 of each variable's max norm (float32 rounding of O(1) flux terms makes a
per-cell relative bound meaningless near zero momenta); after several steps the
normalised L1 of the density <= 1e-5.  On trees with level jumps both sides must
also keep the conserved totals to float32 round-off."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from gpu_util import centres_for, pair
from treeutil import random_balanced_tree

pytestmark = pytest.mark.gpu


def bump_state(x, nl, nc):
    V = np.zeros((nl, 5, nc))
    c = np.array([0.3, 0.45, 0.55])
    r2 = sum((x[:, d] - c[d]) ** 2 for d in range(3))
    V[:, 0] = 1.0 + 0.2 * np.sin(2 * np.pi * (x[:, 0] + 2 * x[:, 2]))
    V[:, 1] = 0.15 * np.cos(2 * np.pi * x[:, 1])
    V[:, 2] = -0.1 * np.sin(2 * np.pi * x[:, 2])
    V[:, 3] = 0.05 + 0.1 * np.cos(2 * np.pi * x[:, 0])
    V[:, 4] = np.where(r2 < 0.03, 8.0, 1.0)
    return V


def scaled_err(a, b):
    return float(np.max(np.abs(a - b) / np.max(np.abs(b), axis=(0, 2), keepdims=True)))


@pytest.mark.parametrize("flux", ["tvdlf", "hll", "hllc"])
@pytest.mark.parametrize("limiter", ["minmod", "vanleer", "koren", "none", "mc", "cada"])
def test_3d_fp32_schemes(flux, limiter):
    base = [2, 1, 1]
    kw = dict(ndim=3, block_nx=16, base=base, gamma=5.0 / 3.0, cfl=0.8, flux=flux, limiter=limiter, rk=3,
              bc="periodic", xmax=(1.0, 0.5, 0.5))
    s, g = pair(precision="fp32", **kw)
    lev, crd = s.leaves()
    x, _ = centres_for(lev, crd, kw)
    s.set_prim(bump_state(x, len(lev), 16 ** 3))
    g.set_cons(s.read_state())  # same (float-rounded) initial state on both sides
    s.step()
    g.step()
    e1 = scaled_err(s.read_state(), g.get_cons())
    assert e1 <= 1e-5, e1
    for _ in range(3):
        s.step()
        g.step()
    a, b = s.read_state()[:, 0], g.get_cons()[:, 0]
    assert np.sum(np.abs(a - b)) / np.sum(np.abs(b)) <= 1e-5


def test_3d_fp32_totals_and_dt():
    """Last-stage reductions of the 3D kernels on a uniform grid (no level jumps):
    float-float totals equal the float64 sum of the float32 state; the CFL step
    matches the oracle on the same state."""
    base = [2, 2, 1]
    kw = dict(ndim=3, block_nx=16, base=base, gamma=5.0 / 3.0, cfl=0.8, flux="hllc", limiter="koren", rk=3,
              bc="periodic", xmax=(1.0, 1.0, 0.5))
    s, g = pair(precision="fp32", **kw)
    lev, crd = s.leaves()
    x, _ = centres_for(lev, crd, kw)
    s.set_prim(bump_state(x, len(lev), 16 ** 3))
    s.run(3)
    s.sync()
    U = s.read_state()
    dV = (1.0 / 32) ** 3
    want = U.sum(axis=(0, 2)) * dV
    got = s.totals()
    assert np.all(np.abs(got - want) <= 1e-11 * np.maximum(np.abs(want), 1.0)), (got, want)
    g.set_cons(U)
    g.t = s.t
    dt_next = s.step()
    assert dt_next == pytest.approx(g.dt(), rel=1e-5)


@pytest.mark.parametrize("flux", ["hll", "hllc"])
def test_3d_fp32_amr_tree(flux):
    """Level jumps: slab ghosts and refluxing through both march kernels."""
    rng = np.random.default_rng(77)
    base = [2, 2, 2]
    lev, crd = random_balanced_tree(3, base, 3, rng, 3)
    kw = dict(ndim=3, block_nx=16, base=base, max_level=3, gamma=1.4, cfl=0.6, flux=flux, limiter="koren", rk=3,
              bc="periodic", refine_tol=0.2, coarsen_frac=0.5, wavefilter=0.01)
    s = amrvac.AmrSolver(precision="fp32", max_blocks=4096, **kw)
    g = O.Grid(**kw)
    s.set_leaves(lev, crd)
    g.set_leaves(lev, crd)
    l2, c2 = s.leaves()
    assert np.any(l2 != l2[0]), "the tree must have level jumps"
    x, _ = centres_for(l2, c2, kw)
    s.set_prim(bump_state(x, len(l2), 16 ** 3))
    g.set_cons(s.read_state())
    t0 = g.totals()
    s.step()
    g.step()
    e1 = scaled_err(s.read_state(), g.get_cons())
    assert e1 <= 1e-5, e1
    s.step()
    g.step()
    a, b = s.read_state()[:, 0], g.get_cons()[:, 0]
    assert np.sum(np.abs(a - b)) / np.sum(np.abs(b)) <= 1e-5
    t1 = s.totals()
    assert np.all(np.abs(t1 - t0)[[0, 4]] <= 1e-6 * np.abs(t0)[[0, 4]]), (t0, t1)


def test_3d_fp32_blast_full_size_step():
    """The blast configuration's tree (4^3 base blocks of 16^3, 4 levels) takes a step
    with the march kernels and keeps density and energy to float32 round-off."""
    base = [4, 4, 4]
    kw = dict(ndim=3, block_nx=16, base=base, max_level=4, gamma=5.0 / 3.0, cfl=0.8, flux="hllc", limiter="koren",
              rk=3, bc="periodic", refine_tol=0.2, coarsen_frac=0.5, wavefilter=0.01, var_mask=1 | (1 << 4))
    s = amrvac.AmrSolver(precision="fp32", max_blocks=8192, **kw)
    for _ in range(4):
        lev, crd = s.leaves()
        x, _ = centres_for(lev, crd, kw)
        s.set_prim(inputs.blast(x, seed=7, ndim=3))
        s.regrid()
    lev, crd = s.leaves()
    assert len(np.unique(lev)) >= 3
    t0 = s.totals()
    s.run(2)
    s.sync()
    t1 = s.totals()
    assert np.all(np.isfinite(s.read_state()))
    assert np.all(np.abs(t1 - t0)[[0, 4]] <= 1e-5 * np.abs(t0)[[0, 4]]), (t0, t1)
