"""GPU parity of the zero-flux (Neumann) multigrid and of the reaction-diffusion schemes
(Sec. 2.5.1-2.5.2: Schnakenberg with Neumann boundaries; IMEX, split and explicit steps)
against the FP64 oracle.

Multigrid tolerances as for the periodic solver: FP64 within 1e-12 of the oracle's
solution; FP32 (float V-cycles on the float64 defect) within 2 rtol max|b| / lambda of it,
because the Neumann operator is also an M-matrix with row sums lambda, so
||A^-1||_inf <= 1/lambda.  Reaction-diffusion steps: FP64 within 1e-12 (explicit) or
1e-11 (after multigrid solves); FP32 within 1e-8 after three implicit steps (each solve
lands within 2 rtol max|w| of the exact discrete solution, rtol 1e-10, |w| < 2)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from test_gpu_mg import SIZES_2D, batch, pack, unpack

pytestmark = pytest.mark.gpu

SCH = dict(Du=inputs.SCHNAKENBERG["Du"], Dv=inputs.SCHNAKENBERG["Dv"], kappa=inputs.SCHNAKENBERG["kappa"],
           a=inputs.SCHNAKENBERG["a"], b=inputs.SCHNAKENBERG["b"], model="schnakenberg", bc="neumann")


@pytest.mark.parametrize("ndim,sizes", [(2, SIZES_2D), (3, [16, 12, 24])])
def test_neumann_fp64_matches_oracle(ndim, sizes):
    L = 1.3
    lam, bs = batch(sizes, ndim, 21)
    s = amrvac.MgSolver(ndim, sizes, lam, L, precision="fp64", bc="neumann")
    x = np.zeros(s.n)
    cyc, rr = s.solve(pack(bs), x)
    xs = unpack(x, sizes, ndim)
    for i in range(len(sizes)):
        xo, co, _ = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i], bc="neumann")
        assert rr[i] <= 1e-10
        assert abs(int(cyc[i]) - co) <= 1, (i, cyc[i], co)
        assert np.max(np.abs(xs[i] - xo)) <= 1e-12 * np.max(np.abs(xo)), i


@pytest.mark.parametrize("nu1,nu2", [(2, 2), (1, 3)])
def test_neumann_fp64_ragged_strips(nu1, nu2):
    """2D sides that leave ragged strips at the right and bottom domain edges (96, 80, 144),
    where the strip sweep's out-of-domain lanes and rows must read as zero."""
    sizes, L = [96, 80, 144], 0.9
    lam, bs = batch(sizes, 2, 23)
    s = amrvac.MgSolver(2, sizes, lam, L, nu1=nu1, nu2=nu2, precision="fp64", bc="neumann")
    x = np.zeros(s.n)
    cyc, rr = s.solve(pack(bs), x)
    xs = unpack(x, sizes, 2)
    for i in range(len(sizes)):
        xo, co, _ = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i], nu1=nu1, nu2=nu2, bc="neumann")
        assert abs(int(cyc[i]) - co) <= 1, (i, cyc[i], co)
        assert np.max(np.abs(xs[i] - xo)) <= 1e-12 * np.max(np.abs(xo)), i


@pytest.mark.parametrize("ndim,sizes", [(2, SIZES_2D), (3, [16, 12, 24])])
def test_neumann_fp32_defect_correction_within_bound(ndim, sizes):
    L, rtol = 1.0, 1e-10
    lam, bs = batch(sizes, ndim, 24, lam_scale=10.0)
    s = amrvac.MgSolver(ndim, sizes, lam, L, precision="fp32", rtol=rtol, bc="neumann")
    x = np.zeros(s.n)
    cyc, rr = s.solve(pack(bs), x)
    xs = unpack(x, sizes, ndim)
    for i in range(len(sizes)):
        assert rr[i] <= rtol
        xo, co, _ = O.mg_solve(bs[i], np.zeros_like(bs[i]), L, lam[i], rtol=rtol, bc="neumann")
        bound = 2.0 * rtol * np.max(np.abs(bs[i])) / lam[i]
        assert np.max(np.abs(xs[i] - xo)) <= bound * 1.05, i
        assert cyc[i] <= co + 3
        r = bs[i] - O.mg_apply(xs[i], L, lam[i], bc="neumann")
        assert np.max(np.abs(r)) <= rtol * np.max(np.abs(bs[i])) * 1.0001


def test_neumann_eigenmode_gpu():
    """cos(pi x / L) cos(2 pi y / L) is a discrete eigenfunction of the cell-centred Neumann
    Laplacian with eigenvalue -(4/h^2) (sin^2(pi h / 2L) + sin^2(pi h / L))."""
    n, L, lam = 256, 1.0, 3.0
    h = L / n
    ax = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(ax, ax, indexing="xy")  # [j, i]
    g = np.cos(np.pi * X / L) * np.cos(2 * np.pi * Y / L)
    mu = (4 / h ** 2) * (np.sin(np.pi * h / (2 * L)) ** 2 + np.sin(np.pi * h / L) ** 2)
    exact = lam * g / (lam + mu)
    # rtol 1e-11: at h = 1/256 the float64 residual itself is only good to ~2e-12 of max|b|.
    # Then |x - exact| <= ||A^-1||_inf rtol max|b| = rtol max|g|.
    for prec in ("fp64", "fp32"):
        s = amrvac.MgSolver(2, [n], [lam], L, precision=prec, rtol=1e-11, bc="neumann")
        x = np.zeros(n * n)
        cyc, rr = s.solve((lam * g).ravel(), x)
        assert rr[0] <= 1e-11
        assert np.max(np.abs(x.reshape(n, n) - exact)) <= 1.05e-11, prec


def sch_states(sizes, ndim):
    us, vs = [], []
    for n in sizes:
        u, v = inputs.schnakenberg_initial(n, ndim)
        us.append(u)
        vs.append(v)
    return us, vs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme,dt,steps", [("imex", 1e-3, 3), ("split", 1e-3, 3), ("explicit", 5e-5, 40)])
def test_schnakenberg_schemes_match_oracle(scheme, dt, steps, precision):
    sizes = [32, 48, 16]
    us, vs = sch_states(sizes, 2)
    rtol = 1e-12 if precision == "fp64" else 1e-10  # FP64: a one-cycle difference stays below 1e-11
    s = amrvac.RdSolver(2, sizes, 1.0, dt=dt, precision=precision, scheme=scheme, rtol=rtol, **SCH)
    s.set_state(pack(us), pack(vs))
    cyc = s.step(steps)
    ug, vg = (unpack(a, sizes, 2) for a in s.read_state())
    for i in range(len(sizes)):
        uo, vo = us[i], vs[i]
        co = []
        for _ in range(steps):
            uo, vo, c = O.rd_step(uo, vo, 1.0, dt=dt, scheme=scheme, rtol=rtol, **SCH)
            co.append(c)
        if scheme == "explicit":
            tol = 1e-12  # no solve: both sides take the same float64 steps
        else:
            tol = 1e-11 if precision == "fp64" else 1e-8
        assert np.max(np.abs(ug[i] - uo)) <= tol, (i, np.max(np.abs(ug[i] - uo)))
        assert np.max(np.abs(vg[i] - vo)) <= tol, (i, np.max(np.abs(vg[i] - vo)))
        if scheme == "explicit":
            assert np.all(cyc == 0)
        elif precision == "fp64":
            assert np.all(np.abs(cyc[:, :, i] - np.array(co)) <= 1), (cyc[:, :, i], co)


@pytest.mark.parametrize("scheme", ["imex", "split"])
def test_schnakenberg_3d_matches_oracle(scheme):
    sizes = [16, 12]
    us, vs = sch_states(sizes, 3)
    s = amrvac.RdSolver(3, sizes, 1.0, dt=1e-3, precision="fp64", scheme=scheme, rtol=1e-12, **SCH)
    s.set_state(pack(us), pack(vs))
    s.step(2)
    ug, vg = (unpack(a, sizes, 3) for a in s.read_state())
    for i in range(len(sizes)):
        uo, vo = us[i], vs[i]
        for _ in range(2):
            uo, vo, _ = O.rd_step(uo, vo, 1.0, dt=1e-3, scheme=scheme, rtol=1e-12, **SCH)
        assert np.max(np.abs(ug[i] - uo)) <= 1e-11
        assert np.max(np.abs(vg[i] - vo)) <= 1e-11


@pytest.mark.parametrize("scheme", ["split", "explicit"])
def test_gray_scott_periodic_other_schemes(scheme):
    """The Gray-Scott model on periodic grids through the split and explicit schemes."""
    sizes, L = [32, 48], 0.4
    dt = 0.5 if scheme == "split" else 0.02
    us, vs = [], []
    for i, n in enumerate(sizes):
        u, v = inputs.gray_scott_patches(n, L=L, seed=4000 + i)
        us.append(u)
        vs.append(v)
    gs = dict(Du=2e-5, Dv=1e-5, F=0.04, k=0.06)
    s = amrvac.RdSolver(2, sizes, L, dt=dt, precision="fp64", scheme=scheme, rtol=1e-12, **gs)
    s.set_state(pack(us), pack(vs))
    s.step(3)
    ug, vg = (unpack(a, sizes, 2) for a in s.read_state())
    for i in range(len(sizes)):
        uo, vo = us[i], vs[i]
        for _ in range(3):
            uo, vo, _ = O.rd_step(uo, vo, L, dt=dt, scheme=scheme, rtol=1e-12, **gs)
        assert np.max(np.abs(ug[i] - uo)) <= 1e-11
        assert np.max(np.abs(vg[i] - vo)) <= 1e-11


def test_explicit_graph_replay_matches_eager_steps():
    """Runs of at least 32 explicit steps replay a captured graph; 70 steps (two graph
    launches and 6 single steps) equal 70 oracle steps and 70 one-step calls."""
    sizes = [32]
    us, vs = sch_states(sizes, 2)
    dt = 5e-5
    a = amrvac.RdSolver(2, sizes, 1.0, dt=dt, precision="fp64", scheme="explicit", **SCH)
    b = amrvac.RdSolver(2, sizes, 1.0, dt=dt, precision="fp64", scheme="explicit", **SCH)
    a.set_state(pack(us), pack(vs))
    b.set_state(pack(us), pack(vs))
    a.step(70)
    for _ in range(70):
        b.step(1)
    ua, va = a.read_state()
    ub, vb = b.read_state()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    uo, vo = us[0], vs[0]
    for _ in range(70):
        uo, vo, _ = O.rd_step(uo, vo, 1.0, dt=dt, scheme="explicit", **SCH)
    assert np.max(np.abs(ua - uo.ravel())) <= 1e-12


def test_schnakenberg_imex_second_order_split_first_order_gpu():
    """Sec. 2.5.2's convergence study at 128^2 on a short interval: against an explicit run
    with dt = 1e-5 (below h^2 / (4 Dv) = 1.5e-5), IMEX errors fall at second order and
    split errors at first order."""
    n, T = 128, 0.02
    u0, v0 = inputs.schnakenberg_initial(n, 2)

    def run(scheme, nsteps):
        s = amrvac.RdSolver(2, [n], 1.0, dt=T / nsteps, precision="fp32", scheme=scheme, rtol=1e-12, **SCH)
        s.set_state(u0.ravel(), v0.ravel())
        s.step(nsteps)
        return s.read_state()

    ur, vr = run("explicit", 2000)
    err = {}
    for scheme in ("imex", "split"):
        err[scheme] = []
        for nsteps in (10, 20, 40):
            u, v = run(scheme, nsteps)
            err[scheme].append(np.sqrt(np.mean((u - ur) ** 2 + (v - vr) ** 2)))
    oi = np.log2(np.array(err["imex"][:-1]) / np.array(err["imex"][1:]))
    os_ = np.log2(np.array(err["split"][:-1]) / np.array(err["split"][1:]))
    assert np.all(oi > 1.8), (err, oi)
    assert np.all((os_ > 0.8) & (os_ < 1.25)), (err, os_)


def test_learned_guess_is_for_imex_only():
    s = amrvac.RdSolver(2, [32], 1.0, dt=1e-3, precision="fp32", scheme="split", **SCH)
    net = amrvac.CnnNet(ndim=2, seed=0)
    with pytest.raises(amrvac.AmrError) as ei:
        s.set_guess(net, 1.0)
    assert ei.value.code == -1
