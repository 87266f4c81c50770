"""GPU parity of the float32 march stage kernels (16^2 and 16^3 leaves) on the paths
the uniform periodic tests do not reach: level jumps (slab ghosts and refluxed face
fluxes) in 2D, and outflow boundaries (ghosts copied from the leaf's own edge) in 2D
and 3D.  Tolerances as for the other float32 tests: per-cell difference <= 1e-5 of
each variable's max norm after one step; normalised L1 of the density <= 1e-5 after
a few; totals kept to float32 round-off on trees with jumps."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from gpu_util import centres_for
from treeutil import random_balanced_tree

pytestmark = pytest.mark.gpu


def scaled_err(a, b):
    return float(np.max(np.abs(a - b) / np.max(np.abs(b), axis=(0, 2), keepdims=True)))


def wave_state(x, ndim, nl, nc):
    V = np.zeros((nl, ndim + 2, nc))
    ph = sum(x[:, d] * (d + 1) for d in range(ndim))
    V[:, 0] = 1.0 + 0.3 * np.sin(2 * np.pi * ph)
    for d in range(ndim):
        V[:, 1 + d] = 0.3 * np.cos(2 * np.pi * x[:, (d + 1) % ndim])
    r2 = sum((x[:, d] - 0.4) ** 2 for d in range(ndim))
    V[:, ndim + 1] = np.where(r2 < 0.02, 6.0, 1.0)
    return V


def run_pair(kw, lev=None, crd=None, steps=3):
    s = amrvac.AmrSolver(precision="fp32", max_blocks=4096, **kw)
    g = O.Grid(**kw)
    if lev is not None:
        s.set_leaves(lev, crd)
        g.set_leaves(lev, crd)
    l2, c2 = s.leaves()
    x, _ = centres_for(l2, c2, kw)
    nc = kw["block_nx"] ** kw["ndim"]
    s.set_prim(wave_state(x, kw["ndim"], len(l2), nc))
    g.set_cons(s.read_state())  # same (float-rounded) initial state on both sides
    t0 = g.totals()
    s.step()
    g.step()
    e1 = scaled_err(s.read_state(), g.get_cons())
    for _ in range(steps - 1):
        s.step()
        g.step()
    a, b = s.read_state()[:, 0], g.get_cons()[:, 0]
    return e1, float(np.sum(np.abs(a - b)) / np.sum(np.abs(b))), t0, s.totals(), l2


@pytest.mark.parametrize("flux", ["hll", "hllc"])
@pytest.mark.parametrize("limiter", ["vanleer", "koren"])
def test_2d_fp32_march_amr_tree(flux, limiter):
    rng = np.random.default_rng(91)
    base = [3, 2]
    lev, crd = random_balanced_tree(2, base + [1], 3, rng, 4)
    kw = dict(ndim=2, block_nx=16, base=base, max_level=3, gamma=1.4, cfl=0.6, flux=flux, limiter=limiter, rk=3,
              bc="periodic", xmax=(1.0, 2.0 / 3.0, 1.0), refine_tol=0.2, coarsen_frac=0.5, wavefilter=0.01)
    e1, l1, t0, t1, l2 = run_pair(kw, lev, crd)
    assert len(np.unique(l2)) >= 2, "the tree must have level jumps"
    assert e1 <= 1e-5, e1
    assert l1 <= 1e-5, l1
    assert np.all(np.abs(t1 - t0)[[0, 3]] <= 1e-6 * np.abs(t0)[[0, 3]]), (t0, t1)


@pytest.mark.parametrize("ndim,base", [(2, [2, 3]), (3, [2, 1, 1])])
def test_fp32_march_outflow(ndim, base):
    kw = dict(ndim=ndim, block_nx=16, base=base, gamma=1.4, cfl=0.8, flux="hllc", limiter="koren", rk=3,
              bc="outflow", xmax=tuple(b / max(base) for b in base) + (1.0,) * (3 - ndim))
    e1, l1, _, _, _ = run_pair(kw)
    assert e1 <= 1e-5, e1
    assert l1 <= 1e-5, l1


@pytest.mark.parametrize("ndim,bnx,base,rk", [(2, 16, [3, 2], 3), (2, 16, [2, 2], 2), (2, 8, [3, 2], 3),
                                             (1, 16, [4], 3), (3, 16, [2, 1, 1], 3)])
def test_fp32_uniform_state_is_kept_exactly(ndim, bnx, base, rk):
    """Free-stream preservation: on a uniform periodic grid every face flux is the same, the
    flux differences are exactly zero, and the SSPRK combination must give back U^n bit for
    bit.  With the plain form alpha*U^n + beta*T the float coefficients 1/3 and 2/3 sum to
    1 + 3e-8, and states such as rho = 0.45 grow by an ulp per step."""
    kw = dict(ndim=ndim, block_nx=bnx, base=base, gamma=1.4, cfl=0.8, flux="hllc", limiter="koren", rk=rk,
              bc="periodic")
    s = amrvac.AmrSolver(precision="fp32", **kw)
    lev, _ = s.leaves()
    nc = bnx ** ndim
    V = np.zeros((len(lev), ndim + 2, nc))
    V[:, 0] = 0.45
    for d in range(ndim):
        V[:, 1 + d] = 0.3 - 0.2 * d
    V[:, ndim + 1] = 0.8
    s.set_prim(V)
    U0 = s.read_state()
    s.run(100)
    s.sync()
    U1 = s.read_state()
    assert np.array_equal(U0, U1), float(np.max(np.abs(U1 - U0)))


def test_stage_tuner_candidates_give_identical_states():
    """Every launch shape the stage-kernel tuner may pick (warps per CTA 2/4/8, grid or persistent,
    per stage kind) advances the state to the same bits; the tuner's own pick is one of them and
    reports a time per stage kind."""
    n = 256
    kw = dict(ndim=2, block_nx=16, base=[n // 16, n // 16], gamma=1.4, cfl=0.8, flux="hllc", limiter="vanleer",
              rk=3, bc="periodic")
    s0 = amrvac.AmrSolver(precision="fp32", **kw)
    lev, crd = s0.leaves()
    x, gi = inputs.cell_centres(lev, crd, 2, 16, kw["base"] + [1], [0, 0, 0], [1, 1, 1])
    V = inputs.kelvin_helmholtz(x, gi, n, seed=2004)
    choices = [[(4, 0), (4, 0), (4, 1)], [(2, 0), (8, 1), (4, 0)], [(8, 0), (2, 1), (4, 1)],
               [(2, 1), (4, 1), (4, 0)], [(8, 1), (8, 0), (4, 1)]]
    states = []
    for ch in choices:
        s = amrvac.AmrSolver(precision="fp32", **kw)
        s.set_prim(V)
        s.set_march_tuning(ch)
        s.run(5)
        s.sync()
        assert s.march_tuning()[0] == [tuple(c) for c in ch]
        states.append(s.read_state())
        s.close()
    for st in states[1:]:
        assert np.array_equal(st, states[0])
    s0.set_prim(V)
    s0.run(5)
    s0.sync()
    pick, us = s0.march_tuning()
    assert pick[2][0] == 4 and all(nw in (2, 4, 8) and p in (0, 1) for nw, p in pick)
    assert all(u > 0 for u in us)
    assert np.array_equal(s0.read_state(), states[0])
    with pytest.raises(amrvac.AmrError):
        s0.set_march_tuning([(3, 0), (4, 0), (4, 1)])


@pytest.mark.parametrize("ndim", [2, 3])
def test_fp32_step_after_set_time_takes_the_clipped_dt(ndim):
    """The float32 stage kernels read the step's dt from a float copy in the control block,
    rewritten by every writer of t, t_end and dt_cfl.  A step clipped to the end time 1 + h after
    amr_set_time(1) must use dt = h exactly as a step from t = 0 clipped to h does: same state
    bit for bit, and t lands on 1 + h (h = 2^-16, far below the CFL step, 1 + h exact)."""
    base = [4, 4] if ndim == 2 else [2, 2, 2]
    kw = dict(ndim=ndim, block_nx=16, base=base, gamma=1.4, cfl=0.8, flux="hllc",
              limiter="vanleer" if ndim == 2 else "koren", rk=3, bc="periodic")
    h = 2.0 ** -16
    runs = []
    for t0 in (0.0, 1.0):
        s = amrvac.AmrSolver(precision="fp32", **kw)
        lev, crd = s.leaves()
        x, gi = inputs.cell_centres(lev, crd, ndim, 16, base + [1] * (3 - ndim), [0, 0, 0], [1, 1, 1])
        s.set_prim(inputs.kelvin_helmholtz(x, gi, 16 * base[0], seed=3) if ndim == 2 else inputs.blast(x, seed=7))
        if t0:
            s.set_time(t0)
        assert s.step(t0 + h) == h
        assert s.t == t0 + h
        s.run(3, t0 + h)  # past the end time: device no-ops
        assert s.t == t0 + h
        runs.append(s.read_state())
        s.close()
    assert np.array_equal(runs[0], runs[1])
