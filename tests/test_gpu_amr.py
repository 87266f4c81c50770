"""GPU parity of the block-tree (AMR) parts: face-neighbour tables, ghost
filling across level jumps, refluxing, the refinement estimator and regrid.

Integer work (trees, neighbour tables) must match bit for bit; the FP64
estimator, computed in the same operation order without FMA contraction on
both sides, must match bit for bit on identical input; FP64 states within
1e-12 relative per cell.
"""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from gpu_util import assert_parity, assert_parity_scaled, centres_for, rel_err
from treeutil import random_balanced_tree, touching

pytestmark = pytest.mark.gpu


def make_pair(ndim, bnx, base, max_level, lev=None, crd=None, precision="fp64", **over):
    kw = dict(ndim=ndim, block_nx=bnx, base=base, max_level=max_level, gamma=1.4, cfl=0.6, flux="hllc",
              limiter="koren", rk=3, bc="periodic", refine_tol=0.2, coarsen_frac=0.5, wavefilter=0.01)
    kw.update(over)
    s = amrvac.AmrSolver(precision=precision, max_blocks=4096, **kw)
    g = O.Grid(**kw)
    if lev is not None:
        s.set_leaves(lev, crd)
        g.set_leaves(lev, crd)
    return s, g, kw


def smooth_state(x, ndim, seed=0):
    nl, _, nc = x.shape
    V = np.zeros((nl, ndim + 2, nc))
    ph = sum(x[:, d] * (d + 1) for d in range(ndim))
    V[:, 0] = 1.0 + 0.3 * np.sin(2 * np.pi * ph + seed)
    for d in range(ndim):
        V[:, 1 + d] = 0.4 * np.cos(2 * np.pi * x[:, (d + 1) % ndim])
    V[:, ndim + 1] = 1.0 + 0.2 * np.cos(2 * np.pi * ph)
    return V


def brute_face_neighbors(lev, crd, ndim, base, max_level, periodic=True):
    """Face neighbour (kind, index) from the definition: look for the leaf that
    covers the block-sized region across the face on the same, coarser or finer level."""
    idx = {(int(l), tuple(int(c) for c in crd[i][:3])): i for i, l in enumerate(lev)}
    n = len(lev)
    kind = np.full((n, 2 * ndim), -1)
    nbr = np.full((n, 2 * ndim), -1)
    for i in range(n):
        l = int(lev[i])
        for f in range(2 * ndim):
            d, side = f // 2, f % 2
            c = [int(v) for v in crd[i][:3]]
            c[d] += 1 if side else -1
            N = base[d] << (l - 1)
            if c[d] < 0 or c[d] >= N:
                if not periodic:
                    continue
                c[d] %= N
            if (l, tuple(c)) in idx:
                kind[i, f], nbr[i, f] = 0, idx[(l, tuple(c))]
                continue
            pc = tuple(v >> 1 for v in c)
            if l > 1 and (l - 1, pc) in idx:
                kind[i, f], nbr[i, f] = 1, idx[(l - 1, pc)]
                continue
            ch = [2 * v for v in c]
            ch[d] += 0 if side else 1
            kind[i, f], nbr[i, f] = 2, idx[(l + 1, tuple(ch))]
    return kind, nbr


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_neighbor_tables_bit_exact(ndim, seed):
    rng = np.random.default_rng(100 + seed + 10 * ndim)
    base = [2, 3, 2][:ndim] + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 5)
    s, g, kw = make_pair(ndim, 8, base, 3, lev, crd)
    l2, c2 = s.leaves()
    lo, co = g.leaves()
    assert np.array_equal(l2, lo) and np.array_equal(c2, co)  # same Morton order
    kind, nbr = s.face_neighbors()
    bk, bn = brute_face_neighbors(l2, c2, ndim, base, 3)
    assert np.array_equal(kind, bk)
    assert np.array_equal(nbr, bn)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_face_ghosts_match_oracle(ndim):
    rng = np.random.default_rng(7 + ndim)
    base = [3, 2, 2][:ndim] + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 5)
    s, g, kw = make_pair(ndim, 8, base, 3, lev, crd)
    l2, c2 = s.leaves()
    x, _ = centres_for(l2, c2, kw)
    V = smooth_state(x, ndim)
    V[:, 0] += 0.5 * (x[:, 0] > 0.5)  # a jump so that limiters act
    s.set_prim(V)
    g.set_prim(V)
    worst = 0.0
    for b in range(s.nleaves):
        a, o = s.face_ghosts(b), g.face_ghosts(b)
        worst = max(worst, float(np.max(np.abs(a - o))))
    assert worst == 0.0, worst


@pytest.mark.parametrize("ndim,bnx", [(2, 8), (2, 16), (3, 8)])
@pytest.mark.parametrize("flux", ["hll", "hllc"])
def test_amr_steps_parity_and_conservation(ndim, bnx, flux):
    rng = np.random.default_rng(50 + ndim + bnx)
    base = [2] * ndim + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 4)
    s, g, kw = make_pair(ndim, bnx, base, 3, lev, crd, flux=flux)
    l2, c2 = s.leaves()
    x, _ = centres_for(l2, c2, kw)
    V = smooth_state(x, ndim, seed=1)
    s.set_prim(V)
    g.set_prim(V)
    t0 = g.totals()
    for _ in range(5):
        dg, do = s.step(), g.step()
        assert dg == pytest.approx(do, rel=1e-14)
    assert_parity_scaled(s.read_state(), g.get_cons(), what="AMR steps")
    tg = s.totals()
    assert np.all(np.abs(tg - t0) <= 5e-13 * np.maximum(np.abs(t0), 1.0)), (t0, tg)


@pytest.mark.parametrize("ndim,bnx,allvars", [(2, 8, False), (3, 8, False), (3, 16, False), (2, 16, True),
                                              (3, 8, True), (3, 16, True)])
def test_estimator_bit_exact(ndim, bnx, allvars):
    """The staged estimator (primitive values in a shared tile; 2D and 3D) and the per-cell one
    (3D 16^3 with all five variables, whose tile would not fit) against the oracle."""
    rng = np.random.default_rng(60 + ndim)
    base = [2] * ndim + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 4)
    mask = (1 << (ndim + 2)) - 1 if allvars else 1 | (1 << (ndim + 1))
    s, g, kw = make_pair(ndim, bnx, base, 3, lev, crd, var_mask=mask)
    l2, c2 = s.leaves()
    x, _ = centres_for(l2, c2, kw)
    V = smooth_state(x, ndim, seed=2)
    r2 = sum((x[:, d] - 0.4) ** 2 for d in range(ndim))
    V[:, ndim + 1] = np.where(r2 < 0.05, 20.0, V[:, ndim + 1])
    s.set_prim(V)
    g.set_prim(V)
    assert np.array_equal(s.estimate(), g.lohner())


@pytest.mark.parametrize("ndim,bnx,allvars", [(2, 16, False), (3, 8, True), (3, 16, False), (3, 16, True)])
def test_estimator_fp32_state(ndim, bnx, allvars):
    """A float32 state is evaluated in float32: per leaf within 1e-5 (relative, or 1e-6 absolute)
    of the oracle's float64 estimator on the same (widened) state."""
    rng = np.random.default_rng(70 + ndim)
    base = [2] * ndim + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 4)
    mask = (1 << (ndim + 2)) - 1 if allvars else 1 | (1 << (ndim + 1))
    s, g, kw = make_pair(ndim, bnx, base, 3, lev, crd, precision="fp32", var_mask=mask)
    l2, c2 = s.leaves()
    x, _ = centres_for(l2, c2, kw)
    V = smooth_state(x, ndim, seed=3)
    r2 = sum((x[:, d] - 0.4) ** 2 for d in range(ndim))
    V[:, ndim + 1] = np.where(r2 < 0.05, 20.0, V[:, ndim + 1])
    s.set_prim(V)
    g.set_cons(s.read_state())
    e32, e64 = s.estimate(), g.lohner()
    assert np.all(np.abs(e32 - e64) <= 1e-5 * np.abs(e64) + 1e-6), np.max(np.abs(e32 - e64))


def blast_setup(ndim, bnx, base, max_level, precision="fp64", cycles=None):
    s, g, kw = make_pair(ndim, bnx, base, max_level, precision=precision, gamma=5.0 / 3.0, cfl=0.8,
                         var_mask=1 | (1 << (ndim + 1)))
    cycles = max_level - 1 if cycles is None else cycles
    for _ in range(cycles + 1):  # sample the initial condition on the current tree, then regrid
        l2, c2 = s.leaves()
        x, _ = centres_for(l2, c2, kw)
        V = inputs.blast(x, seed=7, ndim=ndim, radius=0.2, p_in=100.0)
        s.set_prim(V)
        lo, co = g.leaves()
        assert np.array_equal(lo, l2) and np.array_equal(co, c2)
        g.set_prim(V)
        s.regrid()
        g.regrid()
    l2, c2 = s.leaves()
    x, _ = centres_for(l2, c2, kw)
    V = inputs.blast(x, seed=7, ndim=ndim, radius=0.2, p_in=100.0)
    s.set_prim(V)
    g.set_prim(V)
    return s, g, kw


@pytest.mark.parametrize("ndim", [2, 3])
def test_regrid_tree_and_state_match_oracle(ndim):
    """Initial refinement of a blast, then steps with regrids: the trees stay
    identical and the states agree to 1e-12."""
    base = [2] * ndim + [1] * (3 - ndim)
    s, g, kw = blast_setup(ndim, 8, base, 3)
    lev, _ = s.leaves()
    assert lev.max() == 3
    for cyc in range(3):
        for _ in range(3):
            s.step()
            g.step()
        assert_parity_scaled(s.read_state(), g.get_cons(), what=f"before regrid {cyc}")
        s.regrid()
        g.regrid()
        l2, c2 = s.leaves()
        lo, co = g.leaves()
        assert np.array_equal(l2, lo) and np.array_equal(c2, co), f"trees differ after regrid {cyc}"
        assert_parity_scaled(s.read_state(), g.get_cons(), what=f"after regrid {cyc}")


def test_regrid_fp32_blast_runs_and_conserves():
    base = [2, 2, 2]
    s, _, kw = blast_setup(3, 8, base, 3, precision="fp32")
    t0 = s.totals()
    for _ in range(2):
        s.run(5)
        s.sync()
        s.regrid()
    t1 = s.totals()
    # float32 state: conservation to float32 round-off of the totals
    assert np.all(np.abs(t1 - t0)[[0, 4]] <= 1e-5 * np.abs(t0)[[0, 4]]), (t0, t1)


def test_set_leaves_rejects_unbalanced():
    s = amrvac.AmrSolver(ndim=2, block_nx=8, base=[2, 2], max_level=3, max_blocks=64)
    # a level-3 leaf next to a level-1 leaf
    lev = [1, 1, 1] + [2, 2, 2] + [3] * 4
    crd = [[1, 0, 0], [0, 1, 0], [1, 1, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 0], [1, 0, 0], [0, 1, 0],
           [1, 1, 0]]
    with pytest.raises(amrvac.AmrError) as ei:
        s.set_leaves(np.array(lev), np.array(crd))
    assert ei.value.code in (-8, -1)
    assert s.nleaves == 4  # unchanged


def test_regrid_capacity_error_leaves_tree_unchanged():
    kw = dict(ndim=2, block_nx=8, base=[2, 2], max_level=3, refine_tol=-1.0, coarsen_frac=0.5)
    s = amrvac.AmrSolver(max_blocks=10, **kw)
    V = np.zeros((4, 4, 64))
    V[:, 0] = 1.0
    V[:, 3] = 1.0
    s.set_prim(V)
    with pytest.raises(amrvac.AmrError) as ei:
        s.regrid()  # would need 16 leaves
    assert ei.value.code == -7
    assert s.nleaves == 4
