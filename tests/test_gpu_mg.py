"""GPU parity of the batched Helmholtz multigrid and the Gray-Scott IMEX step.

FP64 path: same algorithm and stopping rule as the oracle -> solutions within
1e-12 relative.  FP32 path (float V-cycles on the float64 defect): both sides
satisfy max|b - A x| <= rtol max|b|, and for the periodic operator
||A^-1||_inf = 1/lambda (row sums lambda, M-matrix), so each solution is within
rtol max|b| / lambda of the exact discrete one: |x_gpu - x_oracle| <=
2 rtol max|b| / lambda.
"""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs

pytestmark = pytest.mark.gpu

SIZES_2D = [16, 24, 32, 40, 12, 64, 48]  # coarsest sides 8, 6, 8, 5, 6, 8, 6


def pack(arrs):
    return np.concatenate([a.ravel() for a in arrs])


def unpack(x, sizes, ndim):
    out, o = [], 0
    for n in sizes:
        m = n ** ndim
        out.append(x[o:o + m].reshape((n,) * ndim))
        o += m
    return out


def batch(sizes, ndim, seed, lam_scale=1.0):
    rng = np.random.default_rng(seed)
    lam = lam_scale * rng.uniform(0.5, 3.0, len(sizes))
    bs = [rng.normal(size=(n,) * ndim) for n in sizes]
    return lam, bs


@pytest.mark.parametrize("ndim,sizes", [(2, SIZES_2D), (3, [16, 12, 24])])
def test_fp64_matches_oracle(ndim, sizes):
    L = 1.7
    lam, bs = batch(sizes, ndim, 3)
    s = amrvac.MgSolver(ndim, sizes, lam, L, precision="fp64")
    x = np.zeros(s.n)
    cyc, rr = s.solve(pack(bs), x)
    xs = unpack(x, sizes, ndim)
    for i, n in enumerate(sizes):
        xo, co, ro = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i])
        assert rr[i] <= 1e-10
        assert abs(int(cyc[i]) - co) <= 1, (i, cyc[i], co)
        assert np.max(np.abs(xs[i] - xo)) <= 1e-12 * np.max(np.abs(xo)), i


@pytest.mark.parametrize("nu1,nu2", [(2, 2), (1, 3), (0, 1)])
def test_fp64_tiled_sweeps_ragged_tiles(nu1, nu2):
    """2D sides above one 64 x 16 sweep tile and not multiples of it (96, 80, 144:
    coarsest 6, 5, 9), with even and odd sweep counts (an odd count ends in the
    second iterate array and is copied back)."""
    sizes, L = [96, 80, 144], 2.1
    lam, bs = batch(sizes, 2, 11)
    s = amrvac.MgSolver(2, sizes, lam, L, nu1=nu1, nu2=nu2, precision="fp64")
    x = np.zeros(s.n)
    cyc, rr = s.solve(pack(bs), x)
    xs = unpack(x, sizes, 2)
    for i, n in enumerate(sizes):
        xo, co, ro = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i], nu1=nu1, nu2=nu2)
        assert rr[i] <= 1e-10
        assert abs(int(cyc[i]) - co) <= 1, (i, cyc[i], co)
        assert np.max(np.abs(xs[i] - xo)) <= 1e-12 * np.max(np.abs(xo)), i


def test_instance_size_limit():
    with pytest.raises(amrvac.AmrError) as ei:
        amrvac.MgSolver(3, [2048], [1.0], 1.0)
    assert ei.value.code == -1


@pytest.mark.parametrize("ndim,sizes", [(2, SIZES_2D), (2, [18, 30, 10, 22]), (3, [16, 12, 24])])
def test_fp32_defect_correction_within_bound(ndim, sizes):
    """(2D sides not divisible by 4 take the defect update's strided form, the others its
    four-consecutive-cell form.)"""
    L, rtol = 2.5, 1e-10
    lam, bs = batch(sizes, ndim, 4, lam_scale=10.0)
    s = amrvac.MgSolver(ndim, sizes, lam, L, precision="fp32", rtol=rtol)
    x = np.zeros(s.n)
    cyc, rr = s.solve(pack(bs), x)
    xs = unpack(x, sizes, ndim)
    for i, n in enumerate(sizes):
        assert rr[i] <= rtol
        xo, co, ro = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i], rtol=rtol)
        bound = 2.0 * rtol * np.max(np.abs(bs[i])) / lam[i]
        assert np.max(np.abs(xs[i] - xo)) <= bound * 1.05, i
        assert cyc[i] <= co + 3
        # the solver's own claim, checked with the oracle's operator
        r = bs[i] - O.mg_apply(xs[i], L, lam[i])
        assert np.max(np.abs(r)) <= rtol * np.max(np.abs(bs[i])) * 1.0001


def test_discrete_eigenfunction_gpu():
    n, L, lam = 256, 2.5, 3.0
    h = L / n
    ax = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(ax, ax, indexing="xy")  # [j, i]
    g = np.sin(2 * np.pi * X / L) * np.sin(2 * np.pi * Y / L)
    mu = (4 / h ** 2) * 2 * np.sin(np.pi * h / L) ** 2
    exact = lam * g / (lam + mu)
    for prec in ("fp64", "fp32"):
        s = amrvac.MgSolver(2, [n], [lam], L, precision=prec, rtol=1e-12)
        x = np.zeros(n * n)
        cyc, rr = s.solve((lam * g).ravel(), x)
        assert rr[0] <= 1e-12
        assert np.max(np.abs(x.reshape(n, n) - exact)) <= 1e-11


def test_zero_cycles_when_guess_is_solution():
    n, L, lam = 32, 1.0, 2.0
    rng = np.random.default_rng(5)
    xk = rng.normal(size=(n, n))
    b = O.mg_apply(xk, L, lam)
    s = amrvac.MgSolver(2, [n], [lam], L, precision="fp32")
    x = xk.ravel().copy()
    cyc, rr = s.solve(b.ravel(), x)
    assert cyc[0] == 0 and np.array_equal(x, xk.ravel())


def test_not_converged_is_reported():
    n = 64
    s = amrvac.MgSolver(2, [n], [1.0], 1.0, precision="fp32", max_cycles=1, rtol=1e-15)
    b = np.random.default_rng(1).normal(size=n * n)
    with pytest.raises(amrvac.AmrError) as ei:
        s.solve(b, np.zeros(n * n))
    assert ei.value.code == -6


def test_device_pointers():
    torch = pytest.importorskip("torch")
    sizes, L = [32, 16], 1.0
    lam, bs = batch(sizes, 2, 8)
    s = amrvac.MgSolver(2, sizes, lam, L, precision="fp32")
    b = torch.from_numpy(pack(bs)).cuda()
    x = torch.zeros_like(b)
    cyc, rr = s.solve(b, x)
    xh = np.zeros(s.n)
    s2 = amrvac.MgSolver(2, sizes, lam, L, precision="fp32")
    s2.solve(pack(bs), xh)
    assert np.array_equal(x.cpu().numpy(), xh)


def test_gray_scott_batch_full_size_one_solve():
    """The 16-instance batch (256^2 .. 2048^2, 28.7 M unknowns) with the implicit
    diffusion constant of u (lambda = 2/(dt Du)): every instance reaches 1e-10,
    checked with the oracle's operator."""
    sizes = inputs.gray_scott_batch_sizes()
    L, dt, Du = 2.5, 0.5, 2e-5
    lam = 2.0 / (dt * Du)
    bs = []
    for i, n in enumerate(sizes):
        u, v = inputs.gray_scott_patches(n, seed=4000 + i)
        bs.append(lam * u)
    s = amrvac.MgSolver(2, sizes, lam, L, precision="fp32")
    x = pack([b / lam for b in bs])  # previous-step guess w_n
    cyc, rr = s.solve(pack(bs), x)
    assert np.all(rr <= 1e-10)
    xs = unpack(x, sizes, 2)
    for i in (0, 7, 15):
        r = bs[i] - O.mg_apply(xs[i], L, lam)
        assert np.max(np.abs(r)) <= 1e-10 * np.max(np.abs(bs[i])) * 1.0001


# ------------------------------------------------------------- Gray-Scott --
GS = dict(Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=0.5)


def gs_inputs(sizes, L):
    us, vs = [], []
    for i, n in enumerate(sizes):
        u, v = inputs.gray_scott_patches(n, L=L, seed=4000 + i)
        us.append(u)
        vs.append(v)
    return us, vs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rd_steps_match_oracle(precision):
    sizes, L = [64, 48, 96], 0.4  # small domain: diffusion is stiff (Du dt / h^2 ~ 0.26 .. 0.6)
    us, vs = gs_inputs(sizes, L)
    s = amrvac.RdSolver(2, sizes, L, precision=precision, **GS)
    s.set_state(pack(us), pack(vs))
    cyc = s.step(3)
    u, v = s.read_state()
    ug, vg = unpack(u, sizes, 2), unpack(v, sizes, 2)
    for i in range(len(sizes)):
        uo, vo = us[i], vs[i]
        co = []
        for _ in range(3):
            uo, vo, c = O.rd_step(uo, vo, L, **GS)
            co.append(c)
        tol = 1e-12 if precision == "fp64" else 2e-9
        assert np.max(np.abs(ug[i] - uo)) <= tol, (i, np.max(np.abs(ug[i] - uo)))
        assert np.max(np.abs(vg[i] - vo)) <= tol
        if precision == "fp64":
            assert np.all(np.abs(cyc[:, 0, i] - np.array(co)[:, 0]) <= 1)


def test_rd_homogeneous_fixed_point():
    sizes = [32, 16]
    s = amrvac.RdSolver(2, sizes, 2.5, precision="fp32", **GS)
    u = np.ones(32 * 32 + 16 * 16)
    v = np.zeros_like(u)
    s.set_state(u, v)
    cyc = s.step(2)
    u1, v1 = s.read_state()
    assert np.array_equal(u1, u) and np.array_equal(v1, v)
    assert np.all(cyc == 0)


def test_rd_uniform_state_is_heun():
    s = amrvac.RdSolver(2, [16], 2.5, precision="fp64", **GS)
    s.set_state(np.full(256, 0.6), np.full(256, 0.3))
    s.step(1)
    u1, v1 = s.read_state()
    F, k, dt = GS["F"], GS["k"], GS["dt"]

    def f(a, b):
        return -a * b * b + F * (1 - a), a * b * b - (F + k) * b
    fu, fv = f(0.6, 0.3)
    fus, fvs = f(0.6 + dt * fu, 0.3 + dt * fv)
    assert np.allclose(u1, 0.6 + dt / 2 * (fu + fus), rtol=1e-9)
    assert np.allclose(v1, 0.3 + dt / 2 * (fv + fvs), rtol=1e-9)


def test_autotuned_strip_heights():
    """mg_create times every candidate strip height of the 2D sweep per level side and keeps
    the fastest; the heights are candidates, a side that is not swept has none, and the
    solve reaches the oracle's solution whatever was chosen (every height gives the same
    iterate)."""
    sizes, L = [256, 160, 288], 2.1
    lam, bs = batch(sizes, 2, 13)
    s = amrvac.MgSolver(2, sizes, lam, L, precision="fp64")
    # strip sweeps run above the shared-memory coarse cycle (float64: from the first side <= 64)
    for n in (256, 128, 160, 80, 288, 144, 72):
        assert s.strip_height(n) in (4, 8, 16, 32, 64), n
    for n in (64, 40, 36, 5):  # depths of the shared-memory cycle, and a coarsest side
        with pytest.raises(amrvac.AmrError):
            s.strip_height(n)
    x = np.zeros(s.n)
    s.solve(pack(bs), x)
    xs = unpack(x, sizes, 2)
    for i in range(len(sizes)):
        xo, _, _ = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i])
        assert np.max(np.abs(xs[i] - xo)) <= 1e-12 * np.max(np.abs(xo))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_profile_vcycle_is_one_more_cycle(precision):
    """mg_profile_vcycle runs one V-cycle kernel by kernel: before any solve it is refused; after
    a solve it reports every kernel of the cycle (the sweeps, residual-restriction and
    prolongation of the depths above the shared-memory ones, the shared-memory coarse cycle,
    and the level-0 update of the precision), each with a positive time, and the handle stays
    usable."""
    sizes, L = [64, 48, 32], 1.3
    lam, bs = batch(sizes, 2, 21)
    s = amrvac.MgSolver(2, sizes, lam, L, rtol=1e-4, precision=precision)
    with pytest.raises(amrvac.AmrError):
        s.profile_vcycle()
    b = pack(bs)
    x = np.zeros(s.n)
    s.solve(b, x)
    prof = s.profile_vcycle()
    kinds = [k for k, _ in prof]
    # depth 0 by per-depth kernels (2 + 2 sweeps, one restriction, one prolongation); the coarse
    # depths (sides <= 128 in float32, <= 64 in float64) of every instance in shared memory
    assert kinds.count("sweep") == 4 and kinds.count("resrestrict") == 1 and kinds.count("prolong") == 1
    assert kinds.count("coarse_cycle") == 1 and kinds.count("coarse") == 0
    # float32 cycles end with the defect update (in 2D the next cycle's first pre-sweep starts
    # from a zero correction without reading it, so no zeroing kernel follows)
    tail = ["sweep", "update"] if precision == "fp32" else ["correct64", "residual64"]
    assert kinds[-2:] == tail and "zero" not in kinds
    assert all(us > 0.0 for _, us in prof)
    # a second solve from the first one's result is converged at once
    cyc, rr = s.solve(b, x)
    assert np.all(cyc == 0) and np.all(rr <= 1e-4)
    s.close()
