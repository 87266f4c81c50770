"""Seeded synthetic inputs for the finite-volume and reaction-diffusion workloads.

This module only samples initial conditions (primitive variables at cell
centres, species concentrations); it contains none of the method's arithmetic,
so the CUDA path and the CPU oracle can both take their inputs from it.

Random numbers come from a counter-based generator: splitmix64 (Steele, Lea,
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied
to ``seed + (counter + 1) * 0x9E3779B97F4A7C15``; the top 53 bits give a double
in [0, 1).  Every value is a pure function of (seed, counter), so any subset of
cells can be regenerated independently.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def uniform(seed: int, counter) -> np.ndarray:
    """splitmix64 output for each counter, mapped to [0, 1)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ------------------------------------------------------------ block geometry --
def cell_centres(level, coords, ndim, block_nx, base, xmin, xmax):
    """Cell-centre coordinates of every leaf cell.

    Returns (x, gidx): x has shape [nleaf, 3, ncell] (unused dims 0), gidx the
    global cell index on the leaf's own level, shape [nleaf, 3, ncell].  Cells
    are ordered i fastest, then j, then k.
    """
    level = np.asarray(level)
    coords = np.asarray(coords).reshape(-1, 3)
    n = block_nx
    ncell = n ** ndim
    loc = np.zeros((3, ncell), dtype=np.int64)
    ar = np.arange(ncell)
    loc[0] = ar % n
    if ndim > 1:
        loc[1] = (ar // n) % n
    if ndim > 2:
        loc[2] = ar // (n * n)
    nl = len(level)
    x = np.zeros((nl, 3, ncell))
    g = np.zeros((nl, 3, ncell), dtype=np.int64)
    for d in range(ndim):
        N = base[d] * n * (2 ** (level.astype(np.int64) - 1))  # cells on each leaf's level
        dx = (xmax[d] - xmin[d]) / N
        g[:, d, :] = coords[:, d, None].astype(np.int64) * n + loc[d][None, :]
        x[:, d, :] = xmin[d] + (g[:, d, :] + 0.5) * dx[:, None]
    return x, g


def _prim(nl, ndim, ncell):
    return np.zeros((nl, ndim + 2, ncell))


def sod(x, ndim=1, x0=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Sod shock tube: (rho, v, p) = left for x < x0, right otherwise."""
    nl, _, ncell = x.shape
    V = _prim(nl, ndim, ncell)
    L = x[:, 0, :] < x0
    V[:, 0] = np.where(L, left[0], right[0])
    V[:, 1] = np.where(L, left[1], right[1])
    V[:, ndim + 1] = np.where(L, left[2], right[2])
    return V


def kelvin_helmholtz(x, gidx, base_cells, seed=2004, amp=0.01):
    """2D shear layer: rho=2, vx=+0.5 for |y-0.5|<0.25, else rho=1, vx=-0.5; p=2.5;
    vy = amp*(2U-1) with U drawn per cell from the global cell index j*Nx + i."""
    nl, _, ncell = x.shape
    V = _prim(nl, 2, ncell)
    inner = np.abs(x[:, 1, :] - 0.5) < 0.25
    V[:, 0] = np.where(inner, 2.0, 1.0)
    V[:, 1] = np.where(inner, 0.5, -0.5)
    cidx = gidx[:, 1, :] * base_cells + gidx[:, 0, :]
    V[:, 2] = amp * (2.0 * uniform(seed, cidx) - 1.0)
    V[:, 3] = 2.5
    return V


def blast(x, seed=7, radius=0.1, p_in=1000.0, p_out=1.0, jitter=0.02, ndim=3):
    """Sphere of radius `radius` around (0.5,0.5,0.5) + uniform jitter in
    [-jitter, jitter] per axis (counters 0..2 of `seed`), p_in inside, p_out
    outside, rho = 1, v = 0."""
    nl, _, ncell = x.shape
    V = _prim(nl, ndim, ncell)
    c = 0.5 + jitter * (2.0 * uniform(seed, np.arange(3)) - 1.0)
    r2 = np.zeros((nl, ncell))
    for d in range(ndim):
        r2 += (x[:, d, :] - c[d]) ** 2
    V[:, 0] = 1.0
    V[:, ndim + 1] = np.where(r2 < radius * radius, p_in, p_out)
    return V


def blast_centre(seed=7, jitter=0.02):
    return 0.5 + jitter * (2.0 * uniform(seed, np.arange(3)) - 1.0)


def smooth_wave(x, ndim, t=0.0, amp=0.2, vel=None):
    """rho = 1 + amp*sin(2 pi (sum_d x_d - t*sum_d v_d)), v = vel (default 1 along
    every axis), p = 1 (advected density wave, exact solution = translation)."""
    nl, _, ncell = x.shape
    vel = [1.0] * ndim if vel is None else list(vel)
    V = _prim(nl, ndim, ncell)
    phase = np.zeros((nl, ncell))
    for d in range(ndim):
        phase += x[:, d, :] - vel[d] * t
    V[:, 0] = 1.0 + amp * np.sin(2.0 * np.pi * phase)
    for d in range(ndim):
        V[:, 1 + d] = vel[d]
    V[:, ndim + 1] = 1.0
    return V


# ---------------------------------------------------------- reaction-diffusion --
def gray_scott_patches(n, ndim=2, L=2.5, seed=4000, npatch=20, side_frac=1.0 / 20.0,
                       u_patch=0.5, v_patch=0.25, noise=0.01):
    """u = 1, v = 0 plus `npatch` axis-aligned square (cube) patches of side
    L*side_frac at uniform-random centres (periodic), where u = u_patch and
    v = v_patch, each multiplied per cell by (1 + noise*(2U - 1)).

    Counters: patch centres use 0 .. npatch*ndim-1; cell noise uses
    2^32 + cell (u) and 2^33 + cell (v), cell = flat index of the n^ndim grid."""
    shape = (n,) * ndim
    u = np.ones(shape)
    v = np.zeros(shape)
    h = L / n
    centres = uniform(seed, np.arange(npatch * ndim)).reshape(npatch, ndim) * L
    axes = [(np.arange(n) + 0.5) * h for _ in range(ndim)]
    mesh = np.meshgrid(*axes, indexing="ij")  # mesh[d][i0, i1, ...] with axis 0 = dim 0
    half = 0.5 * L * side_frac
    mask = np.zeros(shape, dtype=bool)
    for p in range(npatch):
        inside = np.ones(shape, dtype=bool)
        for d in range(ndim):
            dd = np.abs(mesh[d] - centres[p, d])
            dd = np.minimum(dd, L - dd)
            inside &= dd < half
        mask |= inside
    # storage order: x fastest -> transpose so that the flat index is i + n*(j + n*k)
    mask = mask.transpose(tuple(range(ndim))[::-1])
    flat = np.arange(n ** ndim, dtype=np.uint64).reshape((n,) * ndim)
    nu = 1.0 + noise * (2.0 * uniform(seed, flat + np.uint64(1 << 32)) - 1.0)
    nv = 1.0 + noise * (2.0 * uniform(seed, flat + np.uint64(1 << 33)) - 1.0)
    u = np.where(mask, u_patch * nu, 1.0)
    v = np.where(mask, v_patch * nv, 0.0)
    return u, v


def gray_scott_batch_sizes(count=16):
    """Instance sides of the batched workload: 128*(i+2) for i = 0..14 plus a
    second 2048 (16 instances, 256^2 .. 2048^2)."""
    sizes = [128 * (i + 2) for i in range(15)]
    return (sizes + [2048])[:count]


def gresho_chan(x, mach=3.0 ** 0.5 / 5.0, gamma=5.0 / 3.0):
    """Gresho-Chan vortex (Sec. 2.2, Eqs. (gcp), (gcv)) on [-0.5, 0.5]^2: rho = 1, rotation
    v_phi = 5r (r < 0.2), 2 - 5r (0.2 <= r < 0.4), 0 beyond; the pressure balances the
    centrifugal force: p0 + 12.5 r^2 inside 0.2, p0 + 12.5 r^2 + 4(1 - 5r - ln 0.2 + ln r) up to
    0.4, p0 - 2 + 4 ln 2 beyond, with p0 = 1/(gamma M^2).  A stationary solution of the Euler
    equations.  gamma = 5/3 is the value the paper fixes for its hydrodynamic tests (Sec. 2.2).
    x: cell centres [leaf][dim][cell]; returns primitive (rho, v_x, v_y, p)."""
    nl, _, nc = x.shape
    X, Y = x[:, 0], x[:, 1]
    r = np.sqrt(X * X + Y * Y)
    p0 = 1.0 / (gamma * mach * mach)
    rs = np.maximum(r, 1e-300)
    vphi = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    p = np.where(r < 0.2, p0 + 12.5 * r * r,
                 np.where(r < 0.4, p0 + 12.5 * r * r + 4.0 * (1.0 - 5.0 * r - np.log(0.2) + np.log(rs)),
                          p0 - 2.0 + 4.0 * np.log(2.0)))
    V = np.zeros((nl, 4, nc))
    V[:, 0] = 1.0
    V[:, 1] = np.where(r > 0, -vphi * Y / rs, 0.0)
    V[:, 2] = np.where(r > 0, vphi * X / rs, 0.0)
    V[:, 3] = p
    return V


SCHNAKENBERG = dict(Du=0.05, Dv=1.0, kappa=100.0, a=0.1305, b=0.7695)  # Sec. 2.5, Eq. (schnakenberg)


def schnakenberg_initial(n, ndim=2, L=1.0, a=0.1305, b=0.7695):
    """Initial state of the Schnakenberg runs (Sec. 2.5.2) on an n^ndim cell-centred grid of
    [0, L]^ndim: v = b / (a + b)^2 and u = a + b + exp(-100 |r - r0|^2), with r0 = (1/3, 1/2)
    in 2D and (1/3, 1/2, 1/2) in 3D.  Arrays of shape (n,)*ndim, x fastest (last axis)."""
    r0 = [1.0 / 3.0, 0.5, 0.5][:ndim]
    axes = [(np.arange(n) + 0.5) * (L / n) for _ in range(ndim)]
    mesh = np.meshgrid(*axes, indexing="ij")  # mesh[d] varies along axis d
    r2 = sum((mesh[d] - r0[d]) ** 2 for d in range(ndim))
    u = (a + b) + np.exp(-100.0 * r2)
    v = np.full(u.shape, b / (a + b) ** 2)
    # storage order: x fastest, so the flat index is i + n*(j + n*k)
    return np.ascontiguousarray(u.transpose(tuple(range(ndim))[::-1])), v


def quadtree_from_levels(want):
    """Leaves (level, (bx, by)) of a periodic 2D block quadtree with three levels from a wanted
    level per finest-level block position, want[by, bx] in {1, 2, 3} (shape (4 nb, 4 nb)).
    The wish is raised until the tree exists and is 2:1 balanced across faces and corners:
    every neighbour of a level-L position reaches L - 1, and a refined block refines all its
    children.  Returns (level int32 [n], coords int32 [n, 2])."""
    lv = np.array(want, dtype=np.int32)
    ny, nx = lv.shape
    while True:
        old = lv.copy()
        nbmax = lv.copy()
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nbmax = np.maximum(nbmax, np.roll(np.roll(lv, dy, 0), dx, 1))
        lv = np.maximum(lv, nbmax - 1)
        g2 = lv.reshape(ny // 2, 2, nx // 2, 2).max(axis=(1, 3))  # level-2 blocks with a level-3 position
        lv = np.where(np.repeat(np.repeat(g2 == 3, 2, 0), 2, 1), 3, lv)
        g1 = lv.reshape(ny // 4, 4, nx // 4, 4).max(axis=(1, 3))  # level-1 blocks with a refined position
        lv = np.where(np.repeat(np.repeat(g1 >= 2, 4, 0), 4, 1), np.maximum(lv, 2), lv)
        if np.array_equal(lv, old):
            break
    leaves = []
    for by in range(ny // 4):
        for bx in range(nx // 4):
            if lv[4 * by, 4 * bx] == 1:
                leaves.append((1, bx, by))
                continue
            for q in range(4):
                x2, y2 = 2 * bx + (q & 1), 2 * by + (q >> 1)
                if lv[2 * y2, 2 * x2] == 2:
                    leaves.append((2, x2, y2))
                else:
                    leaves += [(3, 2 * x2 + (r & 1), 2 * y2 + (r >> 1)) for r in range(4)]
    arr = np.array(leaves, dtype=np.int32)
    return arr[:, 0].copy(), arr[:, 1:].copy()


GRAY_SCOTT_PAPER = dict(Du=2e-5, Dv=1e-5, F=0.046, k=0.063, dt=0.5, L=2.0)  # Sec. 2.5.2


def gray_scott_tree(nb=16, L=2.0, centres=((0.5, 0.5), (0.55, 0.6)), radii=(0.5, 0.3)):
    """The three-level mesh of Sec. 2.5.2's Gray-Scott run on [0, L]^2 (nb^2 base blocks):
    level 3 within radii[1] of a perturbation centre, level 2 within radii[0], then
    balanced.  (The paper adapts the mesh as the pattern grows; this mesh is fixed.)"""
    n = 4 * nb
    h = L / n
    c = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    d = np.min([np.hypot(X - cx, Y - cy) for cx, cy in centres], axis=0)
    want = np.where(d < radii[1], 3, np.where(d < radii[0], 2, 1))
    return quadtree_from_levels(want)


def gray_scott_gaussians(X, Y, centres=((0.5, 0.5), (0.55, 0.6))):
    """Sec. 2.5.2: u = 1, v = 0 with two perturbations (1/2) exp(-25 |r - r_i|^2) subtracted
    from u and added to v."""
    p = sum(0.5 * np.exp(-25.0 * ((X - cx) ** 2 + (Y - cy) ** 2)) for cx, cy in centres)
    return 1.0 - p, p


def leaf_cell_centres(level, coords, nb, B, L):
    """Cell centres (X, Y), each [leaf][B*B] x fastest, of quadtree leaves on [0, L]^2."""
    level = np.asarray(level)
    coords = np.asarray(coords)
    h = L / (nb * B) / 2.0 ** (level - 1)
    i = np.arange(B)
    X = (coords[:, :1] * B + i[None, :] + 0.5) * h[:, None]
    Y = (coords[:, 1:2] * B + i[None, :] + 0.5) * h[:, None]
    return np.tile(X, (1, B)), np.repeat(Y, B, axis=1)
