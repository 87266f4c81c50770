"""Pins of the oracle's Helmholtz multigrid and Gray-Scott IMEX step (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import inputs
from conftest import golden


def grid_coords(n, ndim, L):
    h = L / n
    ax = (np.arange(n) + 0.5) * h
    mesh = np.meshgrid(*([ax] * ndim), indexing="ij")
    # storage: x fastest -> array axes (z, y, x)
    return [m.transpose(tuple(range(ndim))[::-1]) for m in mesh]


@pytest.mark.parametrize("ndim,n", [(2, 64), (2, 96), (3, 32)])
def test_discrete_eigenfunction(ndim, n):
    """For g = prod_d sin(2 pi x_d / L) the periodic discrete problem
    (lambda - lap_h) x = lambda g has the exact solution
    x = lambda g / (lambda + (4/h^2) sum_d sin^2(pi h / L))."""
    L, lam = 2.5, 3.0
    X = grid_coords(n, ndim, L)
    g = np.ones_like(X[0])
    for d in range(ndim):
        g = g * np.sin(2 * np.pi * X[d] / L)
    h = L / n
    mu = (4 / h ** 2) * ndim * np.sin(np.pi * h / L) ** 2
    exact = lam * g / (lam + mu)
    x, cyc, rr = O.mg_solve(lam * g, np.zeros_like(g), L, lam, rtol=1e-12)
    assert cyc > 0 and rr <= 1e-12
    assert np.max(np.abs(x - exact)) <= 1e-11


@pytest.mark.parametrize("ndim,n", [(2, 8), (2, 16), (2, 12), (3, 8)])
def test_matches_dense_direct(ndim, n):
    rng = np.random.default_rng(n + ndim)
    L, lam = 1.0, 0.7
    b = rng.normal(size=(n,) * ndim)
    xd = O.dense_solve(b, L, lam)
    # the residual of the dense solution is at round-off
    assert np.max(np.abs(O.mg_apply(xd, L, lam) - b)) < 1e-10 * np.max(np.abs(b)) * n * n
    x, cyc, rr = O.mg_solve(b, np.zeros_like(b), L, lam, rtol=1e-14, coarse_max=4, max_cycles=100)
    assert cyc >= 0
    assert np.max(np.abs(x - xd)) <= 1e-12 * np.max(np.abs(xd))


def test_operator_row_sums():
    """Constant vectors: (lambda - lap) c = lambda c exactly (periodic stencil rows sum to 0)."""
    for ndim in (1, 2, 3):
        x = np.full((8,) * ndim, 1.25)
        assert np.array_equal(O.mg_apply(x, 2.0, 3.5), np.full_like(x, 3.5 * 1.25))


def test_manufactured_second_order():
    """Continuous solution x = sin(2pi x/L) sin(2pi y/L) with b = (lambda + 8 pi^2/L^2) x:
    the discrete solution converges with order 2 in h."""
    L, lam = 1.0, 2.0
    errs = []
    for n in (32, 64, 128):
        X = grid_coords(n, 2, L)
        xe = np.sin(2 * np.pi * X[0] / L) * np.sin(2 * np.pi * X[1] / L)
        b = (lam + 8 * np.pi ** 2 / L ** 2) * xe
        x, cyc, rr = O.mg_solve(b, np.zeros_like(b), L, lam)
        errs.append(np.max(np.abs(x - xe)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.05), (errs, orders)


def test_vcycles_flat_in_n():
    """Linear cost: the number of V-cycles to 1e-10 does not grow with N (Sec. 2.5.1)."""
    L, lam = 1.0, 1.0
    counts = []
    for n in (32, 64, 128, 256):
        rng = np.random.default_rng(n)
        b = rng.normal(size=(n, n))
        x, cyc, rr = O.mg_solve(b, np.zeros_like(b), L, lam)
        assert rr <= 1e-10
        counts.append(cyc)
    assert max(counts) - min(counts) <= 1 and max(counts) <= 12, counts


def test_vcycle_contracts():
    rng = np.random.default_rng(9)
    L, lam = 1.0, 1.0
    b = rng.normal(size=(64, 64))
    e = O.mg_vcycle(b, L, lam)
    r1 = b - O.mg_apply(e, L, lam)
    assert np.max(np.abs(r1)) < 0.15 * np.max(np.abs(b))


# -------------------------------------------------------------- Gray-Scott ---
GS = dict(Du=2e-5, Dv=1e-5, F=0.04, k=0.06)


def test_homogeneous_fixed_point():
    u = np.ones((32, 32))
    v = np.zeros((32, 32))
    u1, v1, cyc = O.rd_step(u, v, 2.5, dt=0.5, **GS)
    assert np.array_equal(u1, u) and np.array_equal(v1, v)
    assert list(cyc) == [0, 0]


def test_uniform_state_reduces_to_heun():
    """With spatially uniform data the Laplacian vanishes and Eq. (imex) is the
    explicit trapezoidal (Heun) method on the reaction ODE."""
    u = np.full((16, 16), 0.6)
    v = np.full((16, 16), 0.3)
    dt = 0.5
    u1, v1, _ = O.rd_step(u, v, 2.5, dt=dt, **GS)

    def f(a, b):
        return -a * b * b + GS["F"] * (1 - a), a * b * b - (GS["F"] + GS["k"]) * b
    fu, fv = f(0.6, 0.3)
    us, vs = 0.6 + dt * fu, 0.3 + dt * fv
    fus, fvs = f(us, vs)
    assert np.allclose(u1, 0.6 + dt / 2 * (fu + fus), rtol=1e-9)
    assert np.allclose(v1, 0.3 + dt / 2 * (fv + fvs), rtol=1e-9)


def test_pure_diffusion_is_crank_nicolson_mode():
    """With F = k = 0 and v = 0, u obeys du/dt = Du lap u; a discrete Fourier mode
    is multiplied per step by the trapezoidal factor (1 - z/2)/(1 + z/2),
    z = dt Du mu (mu the discrete eigenvalue), for every dt: A-stable."""
    n, L = 32, 1.0
    X = grid_coords(n, 2, L)
    mode = np.cos(2 * np.pi * 3 * X[0] / L)
    u = 1.0 + 0.1 * mode
    v = np.zeros_like(u)
    h = L / n
    mu = (4 / h ** 2) * np.sin(np.pi * 3 * h / L) ** 2
    Du, dt = 1e-2, 5.0  # far beyond the explicit limit h^2/(4 Du) = 0.024
    z = dt * Du * mu
    u1, v1, _ = O.rd_step(u, v, L, Du=Du, Dv=Du, F=0.0, k=0.0, dt=dt, rtol=1e-13)
    want = 1.0 + 0.1 * mode * (1 - z / 2) / (1 + z / 2)
    assert np.max(np.abs(u1 - want)) < 1e-11
    assert np.array_equal(v1, v)


def test_imex_second_order_in_time():
    n, L = 32, 1.0
    X = grid_coords(n, 2, L)
    u0 = 1.0 - 0.5 * np.exp(-40 * ((X[0] - 0.5) ** 2 + (X[1] - 0.5) ** 2))
    v0 = 0.25 * np.exp(-40 * ((X[0] - 0.5) ** 2 + (X[1] - 0.5) ** 2))
    p = dict(Du=2e-3, Dv=1e-3, F=0.04, k=0.06)

    def run(dt, T=8.0):
        u, v = u0.copy(), v0.copy()
        for _ in range(int(round(T / dt))):
            u, v, _ = O.rd_step(u, v, L, dt=dt, rtol=1e-13, **p)
        return u, v
    ref = run(1.0 / 32)
    errs = []
    for dt in (1.0, 0.5, 0.25):
        u, v = run(dt)
        errs.append(np.max(np.abs(u - ref[0])) + np.max(np.abs(v - ref[1])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8) and np.all(orders < 2.3), (errs, orders)


def test_explicit_limit_table_from_paper():
    """The paper's table of explicit diffusion limits dt < h^2/(2 N_dim D_max) (2D)."""
    rows = [l.split() for l in open(golden("explicit_dt_table.txt")) if l.strip() and not l.startswith("#")]
    for name, D, *vals in rows:
        for h, want in zip((1 / 128, 1 / 256, 1 / 512), map(float, vals)):
            assert (h * h) / (2 * 2 * float(D)) == pytest.approx(want, rel=0.03), (name, h)


def test_gray_scott_patch_input_shape():
    u, v = inputs.gray_scott_patches(256, seed=4000)
    assert u.shape == (256, 256) and v.shape == (256, 256)
    assert 0.49 < u.min() < 0.51 and u.max() == 1.0
    assert v.min() == 0.0 and 0.24 < v.max() < 0.26
    frac = np.mean(v > 0)
    assert 0.01 < frac < 0.06  # 20 patches of (L/20)^2 cover at most 5% of the domain


def test_gray_scott_reaction_steady_states_and_jacobian():
    """Eq. (gray-scott)'s reaction terms vanish at its homogeneous steady states: (1, 0), and
    where F^2 >= 4 F (F + k)^2 the two roots v = (F -+ sqrt(F^2 - 4 F (F + k)^2)) / (2 (F + k)),
    u = (F + k) / v of v (F + k) = F (1 - u), u v = F + k.  At the configuration's F = 0.04,
    k = 0.06 the discriminant is exactly zero: one double root (u, v) = (0.5, 0.2).  The
    Jacobian at (1, 0), by central differences, is diag(-F, -(F + k)) (the autocatalytic
    term is quadratic in v), and the autocatalytic terms cancel in the sum."""
    def roots(F, k):
        disc = F * F - 4 * F * (F + k) ** 2
        if abs(disc) <= 1e-15:
            disc = 0.0  # the configuration's double root (zero up to rounding)
        out = [(1.0, 0.0)]
        if disc >= 0:
            for sgn in (-1, 1):
                v = (F + sgn * np.sqrt(disc)) / (2 * (F + k))
                out.append(((F + k) / v, v))
        return out

    for F, k in ((0.04, 0.06), (0.03, 0.05), (0.02, 0.03), (0.05, 0.04)):
        for us, vs in roots(F, k):
            fu, fv = O.rd_reaction(F, k, np.array([us]), np.array([vs]))
            assert abs(fu[0]) <= 1e-15 and abs(fv[0]) <= 1e-15, (F, k, us, vs, fu, fv)
    F, k = GS["F"], GS["k"]
    assert roots(F, k)[1] == pytest.approx((0.5, 0.2), rel=1e-12)
    eps = 1e-6
    J = np.zeros((2, 2))
    for j, (du, dv) in enumerate([(eps, 0.0), (0.0, eps)]):
        p = O.rd_reaction(F, k, np.array([1.0 + du]), np.array([dv]))
        m = O.rd_reaction(F, k, np.array([1.0 - du]), np.array([-dv]))
        J[:, j] = [(p[0][0] - m[0][0]) / (2 * eps), (p[1][0] - m[1][0]) / (2 * eps)]
    assert np.allclose(J, [[-F, 0.0], [0.0, -(F + k)]], rtol=1e-8, atol=1e-10)
    rng = np.random.default_rng(8)
    u, v = rng.uniform(0, 1, 64), rng.uniform(0, 1, 64)
    fu, fv = O.rd_reaction(F, k, u, v)
    assert np.allclose(fu + fv, F * (1 - u) - (F + k) * v, rtol=1e-13, atol=1e-15)
