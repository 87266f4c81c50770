"""Pins of the oracle's multigrid on a 2D block quadtree (Sec. 1.4, Sec. 2.5.2).

Fixed by: the uniform periodic multigrid (a tree refined everywhere poses the same discrete
problem at the finer resolution), exactness of every ghost rule on linear data,
conservation of the composite operator (sum of cell area x Laplacian = 0 for any data),
constants, second-order convergence to a manufactured smooth solution on refined trees,
and resolution-independent V-cycle counts."""
import numpy as np
import pytest

import oracle as O
from treeutil import is_balanced, random_balanced_tree


def patch_tree(nb, centre=(0.5, 0.5)):
    """Level 2 where a level-1 block's centre is within 0.25 of `centre` (max norm), level 3
    where a level-2 block's centre is within 0.125: a refined patch of fixed geometry."""
    leaves = []
    cx0, cy0 = centre
    for by in range(nb):
        for bx in range(nb):
            cx, cy = (bx + 0.5) / nb, (by + 0.5) / nb
            if abs(cx - cx0) < 0.25 and abs(cy - cy0) < 0.25:
                for q in range(4):
                    x2, y2 = 2 * bx + (q & 1), 2 * by + (q >> 1)
                    c2x, c2y = (x2 + 0.5) / (2 * nb), (y2 + 0.5) / (2 * nb)
                    if abs(c2x - cx0) < 0.125 and abs(c2y - cy0) < 0.125:
                        leaves += [(3, (2 * x2 + (r & 1), 2 * y2 + (r >> 1))) for r in range(4)]
                    else:
                        leaves.append((2, (x2, y2)))
            else:
                leaves.append((1, (bx, by)))
    assert is_balanced([(l, c + (0,)) for l, c in leaves], 2, [nb, nb, 1], 3, (True, True, True))
    return np.array([l for l, _ in leaves], np.int32), np.array([c for _, c in leaves], np.int32)


def centres(lev, crd, nb, B, L=1.0):
    h = L / (nb * B) / 2.0 ** (lev - 1)
    i = np.arange(B)
    X = (crd[:, :1] * B + i[None, :] + 0.5) * h[:, None]
    Y = (crd[:, 1:2] * B + i[None, :] + 0.5) * h[:, None]
    return np.tile(X, (1, B)), np.repeat(Y, B, axis=1), h


def test_tree_refined_everywhere_is_the_uniform_problem():
    nb, B, L, lam = 4, 8, 1.3, 7.0
    lev = np.full(4 * nb * nb, 2, np.int32)
    crd = np.array([(x, y) for y in range(2 * nb) for x in range(2 * nb)], np.int32)
    rng = np.random.default_rng(1)
    n = 2 * nb * B
    bu = rng.standard_normal((n, n))
    # leaf k = (bx, by) holds the uniform cells [by*B:(by+1)*B, bx*B:(bx+1)*B]
    bl = np.stack([bu[y * B:(y + 1) * B, x * B:(x + 1) * B].ravel() for x, y in crd])
    x, cyc, rr = O.amg_solve(lev, crd, bl, np.zeros_like(bl), nb, B, L, lam, rtol=1e-12)
    xu, _, _ = O.mg_solve(bu, np.zeros_like(bu), L, lam, rtol=1e-13)
    xl = np.stack([xu[y * B:(y + 1) * B, x * B:(x + 1) * B].ravel() for x, y in crd])
    assert rr <= 1e-12
    assert np.max(np.abs(x - xl)) <= 1e-10 * np.max(np.abs(xl))
    # the composite operator is the periodic 5-point operator there
    assert np.allclose(O.amg_apply(lev, crd, xl, nb, B, L, lam),
                       np.stack([O.mg_apply(xu, L, lam)[y * B:(y + 1) * B, x * B:(x + 1) * B].ravel()
                                 for x, y in crd]), rtol=0, atol=1e-9 * np.max(np.abs(bu)))


@pytest.mark.parametrize("B", [8, 16])
def test_ghosts_reproduce_linear_data(B):
    nb, L = 4, 1.0
    lev, crd = patch_tree(nb)
    X, Y, h = centres(lev, crd, nb, B, L)
    f = lambda x, y: 0.3 + 1.7 * x - 2.9 * y
    g = O.amg_face_ghosts(lev, crd, f(X, Y), nb, B, L)
    t = np.arange(B)
    checked = 0
    for k in range(len(lev)):
        x0, y0 = crd[k, 0] * B * h[k], crd[k, 1] * B * h[k]
        pos = [(x0 - 0.5 * h[k], y0 + (t + 0.5) * h[k]), (x0 + (B + 0.5) * h[k], y0 + (t + 0.5) * h[k]),
               (x0 + (t + 0.5) * h[k], y0 - 0.5 * h[k]), (x0 + (t + 0.5) * h[k], y0 + (B + 0.5) * h[k])]
        for face, (px, py) in enumerate(pos):
            # away from the periodic wrap, where linear data is not periodic
            if np.min(px) < 0.2 or np.max(px) > 0.8 or np.min(py) < 0.2 or np.max(py) > 0.8:
                continue
            assert np.allclose(g[k, face], f(px, py), rtol=0, atol=1e-13), (k, face, lev[k])
            checked += 1
    assert checked > 40


@pytest.mark.parametrize("seed", [None, 2])
def test_composite_operator_conserves_and_keeps_constants(seed):
    nb, B, L = 4, 8, 1.0
    if seed is None:
        lev, crd = patch_tree(nb)
    else:
        lev, crd3 = random_balanced_tree(2, [nb, nb, 1], 3, np.random.default_rng(seed), 8)
        lev, crd = lev, crd3[:, :2]
    rng = np.random.default_rng(2)
    x = rng.standard_normal((len(lev), B * B))
    _, _, h = centres(lev, crd, nb, B, L)
    lap = -O.amg_apply(lev, crd, x, nb, B, L, 0.0)  # lambda = 0: A x = -lap x
    area = (h ** 2)[:, None]
    assert abs(np.sum(area * lap)) <= 1e-12 * np.sum(np.abs(area * lap))
    c = np.full_like(x, 2.25)
    assert np.allclose(O.amg_apply(lev, crd, c, nb, B, L, 3.0), 3.0 * 2.25, rtol=1e-14, atol=0)


def test_second_order_convergence_on_a_refined_patch():
    """x* = sin(2 pi x) sin(2 pi y): b = (lambda + 8 pi^2) x*; the error falls at second order
    in max and L1 norms as the base grid is refined with the patch geometry kept."""
    B, lam = 8, 10.0
    errs = []
    for nb in (4, 8, 16):
        lev, crd = patch_tree(nb)
        X, Y, h = centres(lev, crd, nb, B)
        xs = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
        x, cyc, rr = O.amg_solve(lev, crd, (lam + 8 * np.pi ** 2) * xs, np.zeros_like(xs), nb, B, 1.0, lam, rtol=1e-11)
        assert cyc <= 10, cyc
        e = np.abs(x - xs)
        errs.append((e.max(), np.sum(e * (h ** 2)[:, None])))
    e = np.array(errs)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order > 1.9), (e, order)


@pytest.mark.parametrize("seed", [3, 4])
def test_random_trees_converge_and_report_their_residual(seed):
    rng = np.random.default_rng(seed)
    nb, B, L, lam = 4, 8, 2.0, 4.0
    lev, crd3 = random_balanced_tree(2, [nb, nb, 1], 3, rng, 6)
    crd = crd3[:, :2]
    assert len(np.unique(lev)) >= 2
    b = rng.standard_normal((len(lev), B * B))
    x, cyc, rr = O.amg_solve(lev, crd, b, np.zeros_like(b), nb, B, L, lam, rtol=1e-10)
    assert 0 < cyc <= 12 and rr <= 1e-10
    r = b - O.amg_apply(lev, crd, x, nb, B, L, lam)
    assert np.max(np.abs(r)) <= 1e-10 * np.max(np.abs(b)) * 1.0001


def test_invalid_trees_are_rejected():
    nb, B = 2, 8
    lev = np.array([1, 1, 1], np.int32)  # a base block missing
    crd = np.array([(0, 0), (1, 0), (0, 1)], np.int32)
    with pytest.raises(ValueError):
        O.amg_solve(lev, crd, np.zeros((3, B * B)), np.zeros((3, B * B)), nb, B, 1.0, 1.0)


# ------------------------------------------------------------ Gray-Scott on the tree --
GS = dict(Du=2e-5, Dv=1e-5, F=0.046, k=0.063)


def test_rd_step_on_a_tree_refined_everywhere_is_the_uniform_step():
    nb, B, L, dt = 2, 8, 0.25, 0.5
    lev = np.full(4 * nb * nb, 2, np.int32)
    crd = np.array([(x, y) for y in range(2 * nb) for x in range(2 * nb)], np.int32)
    n = 2 * nb * B
    rng = np.random.default_rng(4)
    uu, vu = 1.0 - 0.3 * rng.random((n, n)), 0.25 * rng.random((n, n))
    blk = lambda a: np.stack([a[y * B:(y + 1) * B, x * B:(x + 1) * B].ravel() for x, y in crd])
    u1, v1, cyc = O.amg_rd_step(lev, crd, blk(uu), blk(vu), nb, B, L, dt=dt, rtol=1e-12, **GS)
    uo, vo, _ = O.rd_step(uu, vu, L, dt=dt, rtol=1e-13, **GS)
    assert np.max(np.abs(u1 - blk(uo))) <= 1e-10 and np.max(np.abs(v1 - blk(vo))) <= 1e-10


def test_rd_step_on_a_tree_keeps_the_homogeneous_state_and_conserves():
    nb, B, L, dt = 4, 8, 2.0, 0.5
    lev, crd = patch_tree(nb)
    n = len(lev) * B * B
    u1, v1, cyc = O.amg_rd_step(lev, crd, np.ones(n), np.zeros(n), nb, B, L, dt=dt, **GS)
    assert np.array_equal(u1, np.ones(n)) and np.array_equal(v1, np.zeros(n)) and np.all(cyc == 0)
    # F = k = 0: the reactions exchange u and v, and the composite diffusion is conservative,
    # so the area-weighted total of u + v is kept
    X, Y, h = centres(lev, crd, nb, B, L)
    u = (1.0 - 0.5 * np.exp(-25 * ((X - 1.0) ** 2 + (Y - 1.0) ** 2))).ravel()
    v = (0.5 * np.exp(-25 * ((X - 1.0) ** 2 + (Y - 1.1) ** 2))).ravel()
    area = np.repeat(h ** 2, B * B)
    u1, v1, _ = O.amg_rd_step(lev, crd, u, v, nb, B, L, dt=dt, Du=2e-3, Dv=1e-3, F=0.0, k=0.0, rtol=1e-13)
    t0, t1 = np.sum(area * (u + v)), np.sum(area * (u1 + v1))
    assert abs(t1 - t0) <= 1e-12 * t0, (t0, t1)
    assert np.max(np.abs(u1 - u)) > 1e-4  # the step did something


def test_paper_gray_scott_tree_is_a_balanced_three_level_cover():
    from paper_2004_03275_gb300 import inputs
    from treeutil import covers_domain
    lev, crd = inputs.gray_scott_tree()
    assert set(np.unique(lev)) == {1, 2, 3}
    leaves = [(int(l), (int(c[0]), int(c[1]), 0)) for l, c in zip(lev, crd)]
    assert covers_domain(leaves, 2, [16, 16, 1], 3)
    assert is_balanced(leaves, 2, [16, 16, 1], 3, (True, True, True))


# ------------------------------------------------------------ regrid of the RD tree --
def _leaves(lev, crd):
    return [(int(l), (int(c[0]), int(c[1]), 0)) for l, c in zip(lev, crd)]


@pytest.mark.parametrize("seed", [7, 8])
def test_regrid_keeps_a_balanced_cover_and_conserves(seed):
    from treeutil import covers_domain
    from paper_2004_03275_gb300 import inputs
    nb, B, L = 4, 8, 2.0
    lev, crd3 = random_balanced_tree(2, [nb, nb, 1], 3, np.random.default_rng(seed), 6)
    crd = crd3[:, :2]
    X, Y, h = centres(lev, crd, nb, B, L)
    u, v = inputs.gray_scott_gaussians(X, Y, centres=((0.6, 1.3), (1.5, 0.4)))
    nl, nc, nu, nv, err = O.amg_regrid(lev, crd, u, v, nb, B, L, refine_tol=0.05, coarsen_frac=0.5, max_level=3)
    assert covers_domain(_leaves(nl, nc), 2, [nb, nb, 1], 3)
    assert is_balanced(_leaves(nl, nc), 2, [nb, nb, 1], 3, (True, True, True))
    assert np.max(nl) <= 3 and len(err) == len(lev)
    assert not np.array_equal(np.sort(nl), np.sort(lev))  # the tree changed
    _, _, h2 = centres(nl, nc, nb, B, L)
    for a, b in ((u, nu), (v, nv)):
        t0 = np.sum(a * (h ** 2)[:, None])
        t1 = np.sum(b * (h2 ** 2)[:, None])
        assert abs(t1 - t0) <= 1e-13 * abs(t0)


def test_regrid_flags_follow_the_estimator():
    """A constant field has estimator 0: every sibling group coarsens (one level per regrid) and
    the values stay exact.  A linear field also has estimator 0 (no second differences)."""
    nb, B, L = 4, 8, 1.0
    lev, crd = patch_tree(nb)
    n = len(lev)
    u, v = np.full((n, B * B), 0.7), np.full((n, B * B), 0.2)
    nl, nc, nu, nv, err = O.amg_regrid(lev, crd, u, v, nb, B, L, refine_tol=0.1)
    assert np.all(err == 0.0)
    assert np.max(nl) == 2 and np.all(nu == 0.7) and np.all(nv == 0.2)
    X, Y, _ = centres(lev, crd, nb, B, L)
    lin = 0.3 + 0.2 * X - 0.1 * Y
    _, _, _, _, err = O.amg_regrid(lev, crd, lin, lin, nb, B, L, refine_tol=0.1)
    interior = [k for k in range(n) if 0.3 < crd[k, 0] / (nb * 2 ** (lev[k] - 1)) < 0.7
                and 0.3 < crd[k, 1] / (nb * 2 ** (lev[k] - 1)) < 0.7]
    assert np.max(err[interior]) <= 1e-12


def test_regrid_prolongation_is_exact_for_linear_data():
    """Refining a leaf of linear data: its children's cells get the linear function at their
    centres (minmod slopes of linear data are the exact one-sided differences)."""
    nb, B, L = 4, 8, 1.0
    lev = np.ones(nb * nb, np.int32)
    crd = np.array([(x, y) for y in range(nb) for x in range(nb)], np.int32)
    X, Y, _ = centres(lev, crd, nb, B, L)
    f = lambda x, y: 0.5 + 0.3 * x + 0.2 * y
    u = f(X, Y)
    bump = np.exp(-400 * ((X - 0.6) ** 2 + (Y - 0.6) ** 2))  # refines the blocks around (0.6, 0.6)
    nl, nc, nu, nv, err = O.amg_regrid(lev, crd, u, u + bump, nb, B, L, refine_tol=0.2)
    assert np.any(nl == 2)
    X2, Y2, _ = centres(nl, nc, nb, B, L)
    for k in np.where(nl == 2)[0]:
        xk, yk = X2[k], Y2[k]
        if xk.min() > 0.3 and xk.max() < 0.9 and yk.min() > 0.3 and yk.max() < 0.9:
            assert np.allclose(nu[k], f(xk, yk), rtol=0, atol=1e-14)
