"""Pins of the oracle's block-tree operations: ghost filling between levels,
refluxing, Lohner estimator, regrid with 2:1 balance (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import inputs
from treeutil import random_balanced_tree, is_balanced, covers_domain, touching

GAM = 1.4


def grid_on_tree(ndim, bnx, base, max_level, lev, crd, **kw):
    g = O.Grid(ndim=ndim, block_nx=bnx, base=base, max_level=max_level, gamma=kw.pop("gamma", GAM),
               cfl=kw.pop("cfl", 0.5), flux=kw.pop("flux", "hllc"), limiter=kw.pop("limiter", "koren"),
               rk=kw.pop("rk", 3), **kw)
    g.set_leaves(lev, crd)
    return g


def centres(g, base):
    lev, crd = g.leaves()
    c = g.cfg
    return inputs.cell_centres(lev, crd, g.ndim, c.block_nx, list(base) + [1] * (3 - len(base)),
                               list(c.xmin), list(c.xmax))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_random_trees_are_valid(ndim):
    rng = np.random.default_rng(10 + ndim)
    base = [2, 2, 2][:ndim] + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 4)
    leaves = list(zip(lev.tolist(), [tuple(c) for c in crd.tolist()]))
    assert covers_domain(leaves, ndim, base, 3)
    assert is_balanced(leaves, ndim, base, 3, (True, True, True))
    g = grid_on_tree(ndim, 4, base, 3, lev, crd)
    l2, c2 = g.leaves()
    assert sorted(zip(l2.tolist(), map(tuple, c2.tolist()))) == sorted(leaves)


@pytest.mark.parametrize("ndim", [2, 3])
def test_constant_state_exact_on_tree(ndim):
    rng = np.random.default_rng(20 + ndim)
    base = [2] * ndim + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 3)
    g = grid_on_tree(ndim, 4, base, 3, lev, crd)
    V = np.zeros((g.nleaves, ndim + 2, g.ncell))
    V[:, 0] = 1.7
    V[:, 1] = 0.3
    V[:, ndim + 1] = 0.9
    g.set_prim(V)
    U0 = g.get_cons()
    for _ in range(2):
        g.step()
    assert np.allclose(g.get_cons(), U0, rtol=1e-14, atol=1e-15)


def test_linear_data_ghosts_exact_1d():
    """In 1D every ghost (copy, restriction, prolongation) of linear data is exact."""
    # four level-1 blocks; block 1 split into a level-2 and two level-3 blocks
    leaves = [(1, 0), (2, 2), (3, 6), (3, 7), (2, 4), (2, 5), (1, 3)]
    lev = np.array([l for l, _ in leaves], dtype=np.int32)
    crd = np.array([[c, 0, 0] for _, c in leaves], dtype=np.int32)
    g = grid_on_tree(1, 4, [4, 1, 1], 3, lev, crd, bc="periodic")
    x, _ = centres(g, [4])
    V = np.zeros((g.nleaves, 3, g.ncell))
    V[:, 0] = 2.0 + 0.5 * x[:, 0]   # linear, positive, no wrap jump inside the test leaves
    V[:, 2] = 1.0
    g.set_prim(V)
    U = g.get_cons()
    l2, c2 = g.leaves()
    for b in range(g.nleaves):
        lv, cx = l2[b], c2[b, 0]
        if cx == 0 and lv == 1 or (lv == 1 and cx == 3):
            continue  # blocks at the periodic seam see the wrap jump
        gh = g.face_ghosts(b)  # [var][face][layer][1]
        h = 1.0 / (4 * 4 * 2 ** (lv - 1))
        x0 = cx * 4 * h
        want_lo = [2.0 + 0.5 * (x0 - h / 2), 2.0 + 0.5 * (x0 - 3 * h / 2)]
        want_hi = [2.0 + 0.5 * (x0 + 4 * h + h / 2), 2.0 + 0.5 * (x0 + 4 * h + 3 * h / 2)]
        assert np.allclose(gh[0, 0, :, 0], want_lo, rtol=1e-14), (lv, cx)
        assert np.allclose(gh[0, 1, :, 0], want_hi, rtol=1e-14), (lv, cx)


def test_ghosts_exact_for_normal_linear_2d():
    """Data linear in x only: ghosts across x-faces are exact at every level jump
    (the tangential slope is zero), and likewise for y."""
    rng = np.random.default_rng(31)
    base = [3, 3]
    lev, crd = random_balanced_tree(2, base + [1], 3, rng, 4, periodic=(False, False, False))
    g = grid_on_tree(2, 4, base + [1], 3, lev, crd, bc="outflow")
    x, _ = centres(g, base)
    l2, c2 = g.leaves()
    for dim in (0, 1):
        V = np.zeros((g.nleaves, 4, g.ncell))
        V[:, 0] = 2.0 + 0.7 * x[:, dim]
        V[:, 3] = 1.0
        g.set_prim(V)
        for b in range(g.nleaves):
            gh = g.face_ghosts(b)
            lv = l2[b]
            h = 1.0 / (3 * 4 * 2 ** (lv - 1))
            lo = c2[b, dim] * 4 * h
            for side in (0, 1):
                at_edge = (side == 0 and c2[b, dim] == 0) or (side == 1 and (c2[b, dim] + 1) * 4 * h > 1 - 1e-12)
                if at_edge:
                    continue
                for m in (0, 1):
                    xg = lo - (m + 0.5) * h if side == 0 else lo + 4 * h + (m + 0.5) * h
                    assert np.allclose(gh[0, 2 * dim + side, m], 2.0 + 0.7 * xg, rtol=1e-13), (b, dim, side, m)


@pytest.mark.parametrize("ndim", [2, 3])
def test_conservation_on_periodic_tree(ndim):
    """Refluxing keeps sum U dV constant to round-off across level jumps."""
    rng = np.random.default_rng(40 + ndim)
    base = [2] * ndim + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, base, 3, rng, 3)
    g = grid_on_tree(ndim, 4, base, 3, lev, crd, flux="hllc", limiter="koren")
    x, _ = centres(g, base)
    V = np.zeros((g.nleaves, ndim + 2, g.ncell))
    V[:, 0] = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    V[:, 1] = 0.5 * np.cos(2 * np.pi * x[:, 1])
    V[:, ndim + 1] = 1.0 + 0.2 * np.sin(2 * np.pi * (x[:, 0] + x[:, 1]))
    g.set_prim(V)
    t0 = g.totals()
    for _ in range(4):
        g.step()
    t1 = g.totals()
    assert np.all(np.abs(t1 - t0) <= 4e-14 * np.maximum(np.abs(t0), 1.0)), (t0, t1)


def test_reflux_is_needed():
    """Without the fine-flux mean on the coarse side, mass would not be conserved:
    check that the coarse face flux actually changes at a level jump."""
    lev = np.array([1, 2, 2, 2, 2], dtype=np.int32)
    crd = np.array([[0, 0, 0], [2, 0, 0], [3, 0, 0], [2, 1, 0], [3, 1, 0]], dtype=np.int32)
    g = grid_on_tree(2, 4, [2, 1, 1], 2, lev, crd, bc="periodic")
    x, _ = centres(g, [2, 1])
    V = np.zeros((g.nleaves, 4, g.ncell))
    V[:, 0] = 1.0 + 0.5 * np.sin(2 * np.pi * x[:, 1]) + 0.2 * x[:, 0]
    V[:, 1] = 0.7
    V[:, 3] = 1.0
    g.set_prim(V)
    t0 = g.totals()
    g.step()
    assert abs(g.totals()[0] - t0[0]) < 1e-14 * abs(t0[0])


def test_lohner_closed_form_sine():
    """q = 1 + A sin(2 pi x), filter 0: E = 2 sin(pi h)|sin 2pi x| /
    (|cos 2pi(x+h/2)| + |cos 2pi(x-h/2)|) per cell (trig identities), max per block."""
    n, bnx = 64, 8
    g = O.Grid(ndim=1, block_nx=bnx, base=[n // bnx], gamma=GAM, bc="periodic", wavefilter=0.0, var_mask=1)
    x, _ = centres(g, [n // bnx])
    V = np.zeros((g.nleaves, 3, bnx))
    V[:, 0] = 1.0 + 0.4 * np.sin(2 * np.pi * x[:, 0])
    V[:, 2] = 1.0
    g.set_prim(V)
    h = 1.0 / n
    xc = x[:, 0]
    E = 2 * np.sin(np.pi * h) * np.abs(np.sin(2 * np.pi * xc)) / (
        np.abs(np.cos(2 * np.pi * (xc + h / 2))) + np.abs(np.cos(2 * np.pi * (xc - h / 2))))
    assert np.allclose(g.lohner(), E.max(axis=1), rtol=1e-9)


def test_lohner_step_and_filter():
    """A jump gives E close to 1; the filter eps lowers it; linear data gives ~0."""
    n, bnx = 64, 8
    g = O.Grid(ndim=1, block_nx=bnx, base=[n // bnx], gamma=GAM, bc="periodic", wavefilter=0.01, var_mask=1)
    x, _ = centres(g, [n // bnx])
    V = np.zeros((g.nleaves, 3, bnx))
    V[:, 0] = np.where(x[:, 0] < 0.5, 2.0, 1.0)
    V[:, 2] = 1.0
    g.set_prim(V)
    e = g.lohner()
    # at the jump: |d2| = 1, d1 = 1 + 0.01 (|2| + 2|2| + |1|) or (2 + 2 + 2*1... ) -> E = 1/(1+eps*s)
    jump = 1.0 / (1.0 + 0.01 * 7.0)   # cell with q- = q0 = 2, q+ = 1: 2 + 4 + 1 = 7
    assert e.max() == pytest.approx(max(jump, 1.0 / (1.0 + 0.01 * 5.0)), rel=1e-14)
    assert np.sum(e > 0.5) == 4  # the two blocks at x = 0.5 and the two at the periodic seam


@pytest.mark.parametrize("ndim", [2, 3])
def test_regrid_refine_then_coarsen_roundtrip(ndim):
    base = [2] * ndim + [1] * (3 - ndim)
    g = O.Grid(ndim=ndim, block_nx=4, base=base, max_level=2, gamma=GAM, refine_tol=-1.0, coarsen_frac=0.5)
    x, _ = centres(g, base)
    V = np.zeros((g.nleaves, ndim + 2, g.ncell))
    V[:, 0] = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0])
    V[:, ndim + 1] = 1.0 + 0.1 * x[:, 1]
    g.set_prim(V)
    U0, t0 = g.get_cons(), g.totals()
    n1 = g.regrid()
    assert n1 == g.nleaves == (2 ** ndim) * int(np.prod(base[:ndim]))
    assert np.allclose(g.totals(), t0, rtol=1e-14, atol=1e-15)
    g2 = O.Grid(ndim=ndim, block_nx=4, base=base, max_level=2, gamma=GAM, refine_tol=1e30, coarsen_frac=0.5)
    l2, c2 = g.leaves()
    g2.set_leaves(l2, c2)
    g2.set_cons(g.get_cons())
    g2.regrid()
    assert g2.nleaves == int(np.prod(base[:ndim]))
    assert np.allclose(g2.get_cons(), U0, rtol=1e-14, atol=1e-15)


def test_regrid_balance_and_levels():
    """Regrid around a sharp 2D feature: 2:1 balanced, levels within [1, max_level],
    domain covered, leaves at the feature reach max_level."""
    base = [4, 4]
    g = O.Grid(ndim=2, block_nx=8, base=base + [1], max_level=4, gamma=5 / 3, refine_tol=0.2,
               coarsen_frac=0.5, var_mask=1 | 8)
    for _ in range(3):
        x, _ = centres(g, base)
        r2 = (x[:, 0] - 0.3) ** 2 + (x[:, 1] - 0.6) ** 2
        V = np.zeros((g.nleaves, 4, g.ncell))
        V[:, 0] = 1.0
        V[:, 3] = np.where(r2 < 0.01, 1000.0, 1.0)
        g.set_prim(V)
        g.regrid()
    lev, crd = g.leaves()
    leaves = list(zip(lev.tolist(), [tuple(c) for c in crd.tolist()]))
    assert lev.max() == 4 and lev.min() >= 1
    assert covers_domain(leaves, 2, base + [1], 4)
    assert is_balanced(leaves, 2, base + [1], 4, (True, True, True))


def test_regrid_coarsens_smooth_regions():
    base = [2, 2]
    lev, crd = random_balanced_tree(2, base + [1], 3, np.random.default_rng(5), 3)
    g = grid_on_tree(2, 8, base + [1], 3, lev, crd, refine_tol=0.2, coarsen_frac=0.5)
    V = np.zeros((g.nleaves, 4, g.ncell))
    V[:, 0] = 1.0
    V[:, 3] = 1.0
    g.set_prim(V)
    n0 = g.nleaves
    for _ in range(3):
        g.regrid()
    assert g.nleaves == 4 and g.nleaves < n0


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_cfl_dt_closed_form_on_a_tree(ndim):
    """Sec. 1.2's Courant condition on a uniform state: every cell has the same signal speeds,
    so the bound is set by the finest level present, dt = cfl / sum_d (|v_d| + c) / dx_d(finest)
    with c = sqrt(gamma p / rho) in closed form; the last step is clipped to t_end."""
    rng = np.random.default_rng(50 + ndim)
    base = [2, 3, 2][:ndim]
    lev, crd = random_balanced_tree(ndim, base + [1] * (3 - ndim), 3, rng, 2)
    xmin, xmax = (0.0, -1.0, 0.5)[:ndim], (1.0, 2.0, 1.25)[:ndim]
    cfl, bnx = 0.7, 4
    g = grid_on_tree(ndim, bnx, base, 3, lev, crd, cfl=cfl, xmin=xmin, xmax=xmax)
    rho, p = 1.3, 0.9
    vel = np.array([0.4, -0.75, 0.2][:ndim])
    V = np.zeros((g.nleaves, ndim + 2, bnx ** ndim))
    V[:, 0], V[:, ndim + 1] = rho, p
    for d in range(ndim):
        V[:, 1 + d] = vel[d]
    g.set_prim(V)
    c = np.sqrt(GAM * p / rho)
    fine = int(lev.max())
    dx = [(xmax[d] - xmin[d]) / (base[d] * bnx * 2 ** (fine - 1)) for d in range(ndim)]
    want = cfl / sum((abs(vel[d]) + c) / dx[d] for d in range(ndim))
    assert g.dt() == pytest.approx(want, rel=1e-13)
    g.t = 0.25
    assert g.dt(t_end=0.25 + 0.1 * want) == pytest.approx(0.1 * want, rel=1e-9)
    assert g.dt(t_end=1.0) == pytest.approx(want, rel=1e-13)


def _linear(x, coef):
    """a + sum_d g_d x_d for cell centres x [leaf][cell][3]."""
    a, g = coef
    return a + sum(g[d] * x[:, d] for d in range(len(g)))


@pytest.mark.parametrize("ndim", [2, 3])
def test_regrid_children_exact_for_linear_data(ndim):
    """Sec. 1.3's refinement fills each new child by limited linear prolongation of its parent:
    for conserved data linear in every direction the minmod slopes are the exact gradient, so each
    child cell must hold the linear function at its own centre.  The children themselves are
    checked (a restriction round trip would hide a wrong sign or factor of the slopes).  At an
    outflow domain boundary the parent's ghost is a zero-gradient copy, so the slope normal to that
    boundary is zero there: those children hold the value at the parent's position along it."""
    base = [3, 3, 2][:ndim]
    bnx = 4
    g = O.Grid(ndim=ndim, block_nx=bnx, base=base, max_level=2, gamma=GAM, bc="outflow",
               refine_tol=-1.0, coarsen_frac=0.5)
    x, _ = centres(g, base)
    grads = [(1.7, [0.6, -0.4, 0.25][:ndim]), (0.3, [0.2, 0.1, -0.3][:ndim]), (-0.2, [0.05, 0.3, 0.1][:ndim]),
             (0.1, [-0.1, 0.2, 0.15][:ndim]), (4.0, [0.9, 0.5, -0.7][:ndim])][:ndim + 2]
    grads[-1] = (4.0, [0.9, 0.5, -0.7][:ndim])  # energy, comfortably positive
    U = np.stack([_linear(x, c) for c in grads], axis=1)
    g.set_cons(U)
    n1 = g.regrid()
    assert n1 == (2 ** ndim) * int(np.prod(base))
    lev, crd = g.leaves()
    assert np.all(lev == 2)
    xf, _ = centres(g, base)
    Uf = g.get_cons()
    hc = [1.0 / (base[d] * bnx) for d in range(ndim)]
    # parent cell centre and whether it touches the domain boundary, per direction
    want = np.zeros_like(Uf)
    for v, (a0, gv) in enumerate(grads):
        acc = np.full(xf[:, 0].shape, a0)
        for d in range(ndim):
            ip = np.floor(xf[:, d] / hc[d]).astype(int)
            xc = (ip + 0.5) * hc[d]
            edge = (ip == 0) | (ip == base[d] * bnx - 1)
            acc = acc + gv[d] * np.where(edge, xc, xf[:, d])
        want[:, v] = acc
    err = np.max(np.abs(Uf - want))
    assert err <= 1e-13, err
    # the children of interior parent cells carry the full gradient (the case above is not vacuous)
    inner = np.ones(xf[:, 0].shape, dtype=bool)
    for d in range(ndim):
        ip = np.floor(xf[:, d] / hc[d]).astype(int)
        inner &= (ip > 0) & (ip < base[d] * bnx - 1)
    assert inner.sum() > 0.3 * inner.size


def test_regrid_children_exact_across_a_level_jump():
    """Refining a level-2 leaf that borders a level-1 leaf: the parent's ghosts on that face come
    from the coarse neighbour's prolongation.  For data linear along the jump's normal (x) the
    ghosts are exact, so every child of a level-2 parent is exact except at the outflow domain
    boundary in x."""
    lev = np.array([1, 2, 2, 2, 2, 1, 1], dtype=np.int32)
    crd = np.array([[0, 0, 0], [2, 0, 0], [3, 0, 0], [2, 1, 0], [3, 1, 0], [0, 1, 0], [1, 1, 0]],
                   dtype=np.int32)
    base, bnx = [2, 2], 4
    g = O.Grid(ndim=2, block_nx=bnx, base=base + [1], max_level=3, gamma=GAM, bc="outflow",
               refine_tol=1e30, coarsen_frac=0.0)
    g.set_leaves(lev, crd)
    x, _ = centres(g, base)
    U = np.zeros((g.nleaves, 4, g.ncell))
    U[:, 0] = 2.0 + 0.8 * x[:, 0]
    U[:, 1] = 0.3 - 0.5 * x[:, 0]
    U[:, 3] = 5.0 + 1.1 * x[:, 0]
    g.set_cons(U)
    # force refinement of the level-2 leaves only: a grid whose tolerance is below their estimate
    # would also refine the level-1 leaves, so refine by hand through set_leaves + the tree check
    g2 = O.Grid(ndim=2, block_nx=bnx, base=base + [1], max_level=3, gamma=GAM, bc="outflow",
                refine_tol=-1.0, coarsen_frac=0.0)
    l1 = np.array([1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2], dtype=np.int32)
    c1 = np.array([[0, 0, 0], [2, 0, 0], [3, 0, 0], [2, 1, 0], [3, 1, 0], [0, 2, 0], [1, 2, 0], [0, 3, 0],
                   [1, 3, 0], [2, 2, 0], [3, 2, 0], [2, 3, 0], [3, 3, 0]], dtype=np.int32)
    g2.set_leaves(l1, c1)
    x2, _ = centres(g2, base)
    U2 = np.zeros((g2.nleaves, 4, g2.ncell))
    U2[:, 0] = 2.0 + 0.8 * x2[:, 0]
    U2[:, 1] = 0.3 - 0.5 * x2[:, 0]
    U2[:, 3] = 5.0 + 1.1 * x2[:, 0]
    g2.set_cons(U2)
    g2.regrid()  # every leaf refines: level 1 -> 2, level 2 -> 3 (balanced)
    lv, cc = g2.leaves()
    assert lv.max() == 3 and lv.min() == 2
    xf, _ = centres(g2, base)
    Uf = g2.get_cons()
    ncx = base[0] * bnx
    for b in range(g2.nleaves):
        hcx = 1.0 / (ncx * 2 ** (lv[b] - 2))  # the parent's cell width
        ip = np.floor(xf[b, 0] / hcx).astype(int)
        edge = (ip == 0) | (ip == ncx * 2 ** (lv[b] - 2) - 1)
        xe = np.where(edge, (ip + 0.5) * hcx, xf[b, 0])
        for v, (a0, gx) in ((0, (2.0, 0.8)), (1, (0.3, -0.5)), (3, (5.0, 1.1))):
            assert np.allclose(Uf[b, v], a0 + gx * xe, rtol=0, atol=1e-13), (b, lv[b], v)
    assert np.allclose(Uf[:, 2], 0.0)
    assert g.nleaves == 7  # the first grid is untouched (its tolerance refines nothing)


@pytest.mark.parametrize("ndim", [2, 3])
def test_coarse_to_fine_ghosts_for_data_linear_in_every_direction(ndim):
    """Coarse -> fine ghosts (limited linear prolongation, q_c + 1/4 sum_e sigma_e s_e) of data
    linear in every direction, tangential directions and 3D included.  Where both coarse neighbours
    of the sampled coarse cell along a direction e lie inside the coarse leaf (and always along the
    face normal, whose inner neighbour is the restriction of the requesting leaf), the minmod slope
    is the exact gradient; a tangential neighbour outside the coarse leaf gives a zero slope (the
    reading for cells at a coarse leaf's tangential edge).  So each ghost must equal the linear
    function at the point whose coordinate along e is the ghost centre's if e carries a slope and
    the coarse cell centre's otherwise.  Same-level copies and finer-neighbour restrictions of
    linear data are exact.  Data: rho linear, v = 0, p linear, so conserved rho and E are linear."""
    rng = np.random.default_rng(70 + ndim)
    base = [3, 3, 2][:ndim]
    bnx = 4
    b3 = base + [1] * (3 - ndim)
    lev, crd = random_balanced_tree(ndim, b3, 3, rng, 4, periodic=(False, False, False))
    g = grid_on_tree(ndim, bnx, b3, 3, lev, crd, bc="outflow")
    x, _ = centres(g, base)
    grad = [0.7, -0.45, 0.3][:ndim]
    V = np.zeros((g.nleaves, ndim + 2, g.ncell))
    V[:, 0] = 2.0 + sum(grad[d] * x[:, d] for d in range(ndim))
    V[:, ndim + 1] = 3.0 + sum(0.5 * grad[d] * x[:, d] for d in range(ndim))
    g.set_prim(V)
    l2, c2 = g.leaves()
    L = 3
    leafset = {(int(l2[i]), tuple(int(v) for v in c2[i, :3])): i for i in range(g.nleaves)}
    ncell0 = [base[d] * bnx for d in range(ndim)]

    def covering(level, gi):
        """(leaf level, leaf coords) of the leaf covering global cell gi of `level`."""
        for lv in range(1, L + 1):
            sh = lv - level
            c = tuple(((gi[d] << sh) if sh >= 0 else (gi[d] >> -sh)) // bnx if d < ndim else 0 for d in range(3))
            if (lv, c) in leafset:
                return lv, c
        raise AssertionError("uncovered cell")

    checked = {"coarse": 0, "coarse_tang_zero": 0}
    for b in range(g.nleaves):
        lv = int(l2[b])
        h = [1.0 / (ncell0[d] * 2 ** (lv - 1)) for d in range(ndim)]
        gh = g.face_ghosts(b)  # [var][face][layer][tangential]
        tdims = None
        for fd in range(ndim):
            tdims = [e for e in range(ndim) if e != fd]
            for side in (0, 1):
                for m in (0, 1):
                    for t in range(bnx ** (ndim - 1)):
                        loc = [0, 0, 0]
                        if tdims:
                            loc[tdims[0]] = t % bnx
                        if len(tdims) > 1:
                            loc[tdims[1]] = t // bnx
                        loc[fd] = -1 - m if side == 0 else bnx + m
                        gi = [int(c2[b, d]) * bnx + loc[d] for d in range(ndim)]
                        nfine = ncell0[fd] * 2 ** (lv - 1)
                        if gi[fd] < 0 or gi[fd] >= nfine:
                            continue  # outflow: zero-gradient copy
                        xg = [(gi[d] + 0.5) * h[d] for d in range(ndim)]
                        clv, cc = covering(lv, gi)
                        if clv >= lv:
                            pt = xg
                        else:
                            gc = [gi[d] >> 1 for d in range(ndim)]
                            hc = [2 * h[d] for d in range(ndim)]
                            pt = []
                            zero = False
                            for e in range(ndim):
                                xc = (gc[e] + 0.5) * hc[e]
                                if e == fd:
                                    pt.append(xg[e])
                                    continue
                                lo_leaf = cc[e] * bnx
                                inside = lo_leaf <= gc[e] - 1 and gc[e] + 1 <= lo_leaf + bnx - 1
                                pt.append(xg[e] if inside else xc)
                                zero |= not inside
                            checked["coarse"] += 1
                            checked["coarse_tang_zero"] += int(zero)
                        want_r = 2.0 + sum(grad[d] * pt[d] for d in range(ndim))
                        want_e = (3.0 + sum(0.5 * grad[d] * pt[d] for d in range(ndim))) / (GAM - 1)
                        assert gh[0, 2 * fd + side, m, t] == pytest.approx(want_r, rel=1e-14, abs=1e-14), \
                            (b, fd, side, m, t, clv, lv)
                        assert gh[ndim + 1, 2 * fd + side, m, t] == pytest.approx(want_e, rel=1e-14, abs=1e-14)
    assert checked["coarse"] > 0 and 0 < checked["coarse_tang_zero"] < checked["coarse"], checked


@pytest.mark.parametrize("ndim", [2, 3])
def test_lohner_matches_an_independent_uniform_grid_evaluation(ndim):
    """The oracle's estimator (the per-direction reading of Sec. 1.3's weighted second derivatives,
    filter eps (|q+| + 2|q0| + |q-|), max over rho and p and over the block) against a numpy
    evaluation on the whole uniform periodic grid with array shifts, which shares no code with the
    oracle's block and ghost machinery."""
    rng = np.random.default_rng(90 + ndim)
    bnx, nb = 4, 3
    base = [nb] * ndim
    g = O.Grid(ndim=ndim, block_nx=bnx, base=base + [1] * (3 - ndim), gamma=GAM, bc="periodic",
               wavefilter=0.01, var_mask=1 | (1 << (ndim + 1)))
    lev, crd = g.leaves()
    N = nb * bnx
    shape = (N,) * ndim  # axis d of the array is dimension ndim - 1 - d ([z][y][x])
    rho = 1.0 + 0.5 * rng.random(shape)
    p = 0.5 + rng.random(shape)
    vel = [0.3 * rng.standard_normal(shape) for _ in range(ndim)]
    V = np.zeros((g.nleaves, ndim + 2, g.ncell))
    for b in range(g.nleaves):
        sl = tuple(slice(crd[b, d] * bnx, (crd[b, d] + 1) * bnx) for d in reversed(range(ndim)))
        V[b, 0] = rho[sl].ravel()
        for d in range(ndim):
            V[b, 1 + d] = vel[d][sl].ravel()
        V[b, ndim + 1] = p[sl].ravel()
    g.set_prim(V)
    # the oracle converts the conserved state back to primitives: do the same here
    U = g.get_cons()
    grid = np.zeros((ndim + 2,) + shape)
    for b in range(g.nleaves):
        sl = tuple(slice(crd[b, d] * bnx, (crd[b, d] + 1) * bnx) for d in reversed(range(ndim)))
        grid[(slice(None),) + sl] = U[b].reshape((ndim + 2,) + (bnx,) * ndim)
    r = grid[0]
    kin = sum(grid[1 + d] ** 2 for d in range(ndim)) * 0.5 / r
    pr = (GAM - 1) * (grid[ndim + 1] - kin)

    def est(q):
        num = np.zeros_like(q)
        den = np.zeros_like(q)
        for d in range(ndim):
            ax = ndim - 1 - d
            qp, qm = np.roll(q, -1, axis=ax), np.roll(q, 1, axis=ax)
            num += (qp - 2 * q + qm) ** 2
            den += (np.abs(qp - q) + np.abs(q - qm) + 0.01 * (np.abs(qp) + 2 * np.abs(q) + np.abs(qm))) ** 2
        return np.sqrt(num / den)

    E = np.maximum(est(r), est(pr))
    want = np.array([E[tuple(slice(crd[b, d] * bnx, (crd[b, d] + 1) * bnx) for d in reversed(range(ndim)))].max()
                     for b in range(g.nleaves)])
    assert np.allclose(g.lohner(), want, rtol=1e-12, atol=0)
