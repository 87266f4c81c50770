"""GPU parity of the multigrid on a 2D block quadtree (float64) against the oracle.

The composite operator is the same arithmetic on both sides (no multiply-add contraction
on the GPU unit): within 1e-12 of max|Ax|.  The base-level correction solves run the uniform
multigrid on both sides (multiply-add contraction on the GPU's uniform unit, none in the
oracle) until the base residual has fallen by base_rtol; with base_rtol 1e-13 the iterates of
fixed V-cycle counts agree within 1e-12 of max|x| (measured: at most 1.9e-15), and so do the
converged solutions at rtol 1e-10 (measured: at most 4.9e-15), with the same cycle counts."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac
from test_oracle_amg import centres, patch_tree
from treeutil import random_balanced_tree

pytestmark = pytest.mark.gpu


def trees():
    out = [("patch", 4, 8) + patch_tree(4), ("patch16", 4, 16) + patch_tree(4)]
    for seed in (5, 6):
        lev, crd = random_balanced_tree(2, [4, 4, 1], 3, np.random.default_rng(seed), 7)
        out.append((f"random{seed}", 4, 8, lev, crd[:, :2]))
    return out


@pytest.mark.parametrize("case", trees(), ids=lambda c: c[0])
def test_composite_operator_matches_oracle(case):
    _, nb, B, lev, crd = case
    L, lam = 1.7, 3.5
    x = np.random.default_rng(1).standard_normal((len(lev), B * B))
    s = amrvac.TreeMgSolver(lev, crd, nb, B, L, lam)
    a = s.apply(x)
    o = O.amg_apply(lev, crd, x, nb, B, L, lam)
    assert np.max(np.abs(a - o)) <= 1e-12 * np.max(np.abs(o))


@pytest.mark.parametrize("case", trees(), ids=lambda c: c[0])
@pytest.mark.parametrize("ncyc", [1, 3])
def test_fixed_vcycles_match_oracle(case, ncyc):
    _, nb, B, lev, crd = case
    L, lam = 1.0, 40.0
    b = np.random.default_rng(2).standard_normal((len(lev), B * B))
    s = amrvac.TreeMgSolver(lev, crd, nb, B, L, lam, base_rtol=1e-13)
    x = np.zeros_like(b)
    cyc, rr = s.solve(b, x, fixed_cycles=ncyc)
    xo, co, ro = O.amg_solve(lev, crd, b, np.zeros_like(b), nb, B, L, lam, fixed_cycles=ncyc, base_rtol=1e-13)
    assert cyc == ncyc == co
    assert np.max(np.abs(x - xo)) <= 1e-12 * np.max(np.abs(xo))
    assert rr == pytest.approx(ro, rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("case", trees(), ids=lambda c: c[0])
def test_converged_solve_matches_oracle(case):
    _, nb, B, lev, crd = case
    L, lam = 1.0, 10.0
    X, Y, _ = centres(lev, crd, nb, B, L)
    xs = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    b = (lam + 8 * np.pi ** 2) * xs
    s = amrvac.TreeMgSolver(lev, crd, nb, B, L, lam, rtol=1e-10)
    x = np.zeros_like(b)
    cyc, rr = s.solve(b, x)
    xo, co, ro = O.amg_solve(lev, crd, b, np.zeros_like(b), nb, B, L, lam, rtol=1e-10)
    assert rr <= 1e-10 and cyc == co
    assert np.max(np.abs(x - xo)) <= 1e-12 * np.max(np.abs(xo))
    r = b - O.amg_apply(lev, crd, x, nb, B, L, lam)
    assert np.max(np.abs(r)) <= 1e-10 * np.max(np.abs(b)) * 1.0001


def test_device_arrays_and_launch_count():
    torch = pytest.importorskip("torch")
    lev, crd = patch_tree(4)
    B = 8
    b = np.random.default_rng(3).standard_normal((len(lev), B * B))
    s = amrvac.TreeMgSolver(lev, crd, 4, B, 1.0, 5.0)
    xh = np.zeros_like(b)
    s.solve(b, xh)
    n0 = s.kernel_launches()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    s.solve(bd, xd)
    assert np.array_equal(xd.cpu().numpy(), xh)
    assert s.kernel_launches() > n0


def test_invalid_trees_are_rejected():
    B = 8
    with pytest.raises(amrvac.AmrError) as ei:  # a base block missing
        amrvac.TreeMgSolver(np.array([1, 1, 1]), np.array([(0, 0), (1, 0), (0, 1)]), 2, B, 1.0, 1.0)
    assert ei.value.code == -1
    # level 3 next to level 1: not 2:1 balanced
    lev = [1, 1, 1] + [2, 2, 2] + [3, 3, 3, 3]
    crd = [(1, 0), (0, 1), (1, 1), (1, 0), (0, 1), (1, 1), (0, 0), (1, 0), (0, 1), (1, 1)]
    with pytest.raises(amrvac.AmrError) as ei:
        amrvac.TreeMgSolver(np.array(lev), np.array(crd), 2, B, 1.0, 1.0)
    assert ei.value.code == -1


# ------------------------------------------------------------ Gray-Scott on the tree --
def test_gray_scott_steps_match_oracle():
    from paper_2004_03275_gb300 import inputs
    nb, B, L = 4, 8, 2.0
    lev, crd = inputs.gray_scott_tree(nb=nb, L=L, radii=(0.5, 0.25))
    assert set(np.unique(lev)) == {1, 2, 3}
    X, Y = inputs.leaf_cell_centres(lev, crd, nb, B, L)
    u, v = inputs.gray_scott_gaussians(X, Y)
    p = dict(Du=2e-5, Dv=1e-5, F=0.046, k=0.063, dt=0.5)
    s = amrvac.TreeRdSolver(lev, crd, nb, B, L, **p)
    s.set_state(u.ravel(), v.ravel())
    cyc = s.step(3)
    ug, vg = s.read_state()
    uo, vo = u.ravel(), v.ravel()
    co = []
    for _ in range(3):
        uo, vo, c = O.amg_rd_step(lev, crd, uo, vo, nb, B, L, **p)
        co.append(c)
    assert np.array_equal(np.asarray(cyc).ravel(), np.asarray(co).ravel()), (cyc, co)
    assert np.max(np.abs(ug - uo)) <= 1e-12 * np.max(np.abs(uo)) and np.max(np.abs(vg - vo)) <= 1e-12 * np.max(np.abs(vo))


def test_gray_scott_tree_keeps_the_homogeneous_state():
    from paper_2004_03275_gb300 import inputs
    lev, crd = inputs.gray_scott_tree(nb=4, L=2.0, radii=(0.5, 0.25))
    n = len(lev) * 64
    s = amrvac.TreeRdSolver(lev, crd, 4, 8, 2.0, Du=2e-5, Dv=1e-5, F=0.046, k=0.063, dt=0.5)
    s.set_state(np.ones(n), np.zeros(n))
    cyc = s.step(2)
    u, v = s.read_state()
    assert np.array_equal(u, np.ones(n)) and np.array_equal(v, np.zeros(n)) and np.all(cyc == 0)


# ------------------------------------------------------------- regrid of the RD tree --
@pytest.mark.parametrize("seed", [7, 8])
def test_regrid_matches_oracle(seed):
    """Estimator, new tree and moved fields against the oracle: the tree bit for bit."""
    from paper_2004_03275_gb300 import inputs
    nb, B, L = 4, 8, 2.0
    lev, crd3 = random_balanced_tree(2, [nb, nb, 1], 3, np.random.default_rng(seed), 6)
    crd = crd3[:, :2]
    X, Y = inputs.leaf_cell_centres(lev, crd, nb, B, L)
    u, v = inputs.gray_scott_gaussians(X, Y, centres=((0.6, 1.3), (1.5, 0.4)))
    s = amrvac.TreeRdSolver(lev, crd, nb, B, L, Du=2e-5, Dv=1e-5, F=0.046, k=0.063, dt=0.5)
    s.set_state(u.ravel(), v.ravel())
    err = s.regrid(refine_tol=0.05, coarsen_frac=0.5, max_level=3)
    nl, nc, nu, nv, eo = O.amg_regrid(lev, crd, u, v, nb, B, L, refine_tol=0.05, coarsen_frac=0.5, max_level=3)
    assert np.array_equal(err, eo)
    gl, gc = s.leaves()
    assert np.array_equal(gl, nl) and np.array_equal(gc, nc)
    ug, vg = s.read_state()
    assert np.max(np.abs(ug - nu.ravel())) <= 1e-15 and np.max(np.abs(vg - nv.ravel())) <= 1e-15


def test_gray_scott_with_regrids_matches_oracle():
    """Steps and regrids alternate on the paper's mesh (4^2 base blocks): leaves and fields
    against the oracle after two rounds."""
    from paper_2004_03275_gb300 import inputs
    nb, B, L = 4, 8, 2.0
    p = dict(Du=2e-5, Dv=1e-5, F=0.046, k=0.063, dt=0.5)
    lev, crd = inputs.gray_scott_tree(nb=nb, L=L, radii=(0.5, 0.25))
    X, Y = inputs.leaf_cell_centres(lev, crd, nb, B, L)
    u, v = inputs.gray_scott_gaussians(X, Y)
    s = amrvac.TreeRdSolver(lev, crd, nb, B, L, **p)
    s.set_state(u.ravel(), v.ravel())
    uo, vo, lo, co = u.ravel(), v.ravel(), lev, crd
    for _ in range(2):
        s.step(3)
        for _ in range(3):
            uo, vo, _ = O.amg_rd_step(lo, co, uo, vo, nb, B, L, **p)
        s.regrid(refine_tol=0.02)
        lo, co, uo, vo, _ = O.amg_regrid(lo, co, uo.reshape(len(lo), -1), vo.reshape(len(lo), -1), nb, B, L,
                                         refine_tol=0.02)
        uo, vo = uo.ravel(), vo.ravel()
    gl, gc = s.leaves()
    assert np.array_equal(gl, lo) and np.array_equal(gc, co)
    ug, vg = s.read_state()
    assert np.max(np.abs(ug - uo)) <= 1e-12 * np.max(np.abs(uo)) and np.max(np.abs(vg - vo)) <= 1e-12 * np.max(np.abs(vo))
