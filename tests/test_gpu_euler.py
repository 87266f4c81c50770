"""GPU parity of the finite-volume Euler update on uniform block grids.

The CUDA path (through the C ABI) is compared cell by cell with the FP64 CPU
oracle on the same seeded inputs: FP64 within 1e-12 relative per cell, the
CFL step to round-off; the FP32 path by its normalised L1 error.
"""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from gpu_util import assert_parity, pair, centres_for, rel_err

pytestmark = pytest.mark.gpu


def kh_kw(nside, bnx=16, **over):
    nb = nside // bnx
    kw = dict(ndim=2, block_nx=bnx, base=[nb, nb], gamma=1.4, cfl=0.8, flux="hllc", limiter="vanleer", rk=3,
              bc="periodic")
    kw.update(over)
    return kw


def kh_state(s, kw, nside, seed=2004):
    lev, crd = s.leaves()
    x, gi = centres_for(lev, crd, kw)
    return inputs.kelvin_helmholtz(x, gi, nside, seed=seed)


def test_sod_config_parity_and_exact():
    """512 cells as 32 blocks of 16, HLL + minmod, SSPRK2, CFL 0.8, outflow, to t = 0.2."""
    kw = dict(ndim=1, block_nx=16, base=[32], gamma=1.4, cfl=0.8, flux="hll", limiter="minmod", rk=2,
              bc="outflow")
    s, g = pair(**kw)
    lev, crd = s.leaves()
    x, _ = centres_for(lev, crd, kw)
    V = inputs.sod(x)
    s.set_prim(V)
    g.set_prim(V)
    n = 0
    while g.t < 0.2:
        dto = g.step(0.2)
        dtg = s.step(0.2)
        assert abs(dtg - dto) <= 1e-14 * dto
        n += 1
        if n in (1, 10, 50):
            assert_parity(s.read_state(), g.get_cons(), what=f"Sod step {n}")
    assert s.t == 0.2 and g.t == 0.2
    U = s.read_state()
    assert_parity(U, g.get_cons(), what="Sod final")
    ex, _, _ = O.exact_riemann(1.4, [1, 0, 1], [0.125, 0, 0.1], (x[:, 0].ravel() - 0.5) / 0.2)
    assert np.mean(np.abs(U[:, 0].ravel() - ex[:, 0])) <= 1e-2
    assert s.step(0.2) == 0.0  # past t_end: no-op


@pytest.mark.parametrize("flux", ["tvdlf", "hll", "hllc"])
@pytest.mark.parametrize("limiter", ["minmod", "vanleer", "koren", "none", "mc", "cada"])
def test_2d_schemes_fp64_parity(flux, limiter):
    """Every flux x limiter pair, 15 leaves of 8^2 (ragged last CTA), 6 steps."""
    kw = dict(ndim=2, block_nx=8, base=[3, 5], gamma=1.4, cfl=0.8, flux=flux, limiter=limiter, rk=3,
              bc="periodic", xmax=(1.0, 5.0 / 3.0, 1.0))
    s, g = pair(**kw)
    lev, crd = s.leaves()
    x, gi = centres_for(lev, crd, kw)
    V = inputs.kelvin_helmholtz(x, gi, 24, seed=7)
    s.set_prim(V)
    g.set_prim(V)
    for k in range(6):
        assert abs(s.step() - g.step()) <= 1e-14 * g.dt() * 10
    assert_parity(s.read_state(), g.get_cons(), what=f"{flux}/{limiter}")


@pytest.mark.parametrize("bnx", [8, 16])
@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("limiter", ["koren", "cada"])
def test_1d_parity(bnx, rk, limiter):
    kw = dict(ndim=1, block_nx=bnx, base=[9], gamma=1.4, cfl=0.6, flux="hllc", limiter=limiter, rk=rk,
              bc="periodic")
    s, g = pair(**kw)
    lev, crd = s.leaves()
    x, _ = centres_for(lev, crd, kw)
    V = inputs.smooth_wave(x, 1)
    V[:, 2] += 0.5 * (x[:, 0] > 0.5)
    s.set_prim(V)
    g.set_prim(V)
    for _ in range(20):
        s.step()
        g.step()
    assert_parity(s.read_state(), g.get_cons(), what="1D")


@pytest.mark.parametrize("bnx,base", [(8, [2, 2, 3]), (16, [2, 1, 1])])
@pytest.mark.parametrize("flux,limiter", [("hll", "koren"), ("hllc", "koren"), ("hllc", "cada")])
def test_3d_parity(bnx, base, flux, limiter):
    kw = dict(ndim=3, block_nx=bnx, base=base, gamma=5.0 / 3.0, cfl=0.8, flux=flux, limiter=limiter, rk=3,
              bc="periodic", xmax=(base[0] / max(base), base[1] / max(base), base[2] / max(base)))
    s, g = pair(**kw)
    lev, crd = s.leaves()
    x, _ = centres_for(lev, crd, kw)
    c = np.array([0.3, 0.25, 0.35]) * np.array(kw["xmax"])
    r2 = sum((x[:, d] - c[d]) ** 2 for d in range(3))
    V = np.zeros((len(lev), 5, bnx ** 3))
    V[:, 0] = 1.0 + 0.2 * np.sin(2 * np.pi * x[:, 2])
    V[:, 1] = 0.1
    V[:, 3] = -0.05
    V[:, 4] = np.where(r2 < 0.02, 10.0, 1.0)
    s.set_prim(V)
    g.set_prim(V)
    for _ in range(4):
        s.step()
        g.step()
    assert_parity(s.read_state(), g.get_cons(), what="3D")


def test_kh_64_fp64_long_parity():
    """KH amplifies round-off: parity checked at steps 1, 10 and 60."""
    kw = kh_kw(64)
    s, g = pair(**kw)
    V = kh_state(s, kw, 64)
    s.set_prim(V)
    g.set_prim(V)
    for n in range(1, 61):
        s.step()
        g.step()
        if n in (1, 10, 60):
            assert_parity(s.read_state(), g.get_cons(), what=f"KH64 step {n}")
    assert_parity(s.totals(), g.totals(), what="totals")


def test_kh_conservation_gpu():
    kw = kh_kw(128)
    s = amrvac.AmrSolver(precision="fp64", **kw)
    s.set_prim(kh_state(s, kw, 128))
    t0 = s.totals()
    s.run(20)
    s.sync()
    t1 = s.totals()
    assert np.all(np.abs(t1 - t0) <= 20 * 1e-13 * np.maximum(np.abs(t0), 1.0)), (t0, t1)


def test_fp32_l1_vs_fp64_oracle():
    """FP32 path: normalised L1 of rho against the FP64 oracle after 20 steps."""
    kw = kh_kw(128)
    s, g = pair(precision="fp32", **kw)
    V = kh_state(s, kw, 128)
    s.set_prim(V)
    g.set_prim(V)
    for _ in range(20):
        s.step()
        g.step()
    a, b = s.read_state()[:, 0], g.get_cons()[:, 0]
    l1 = np.sum(np.abs(a - b)) / np.sum(np.abs(b))
    assert l1 <= 1e-4, l1
    assert s.t == pytest.approx(g.t, rel=1e-5)


def test_run_matches_step_and_graph_replay():
    """amr_run (graph launches) gives bit-identical results to repeated amr_step."""
    kw = kh_kw(64)
    a = amrvac.AmrSolver(precision="fp64", **kw)
    b = amrvac.AmrSolver(precision="fp64", **kw)
    V = kh_state(a, kw, 64)
    a.set_prim(V)
    b.set_prim(V)
    for _ in range(7):
        a.step()
    b.run(7)
    b.sync()
    assert np.array_equal(a.read_state(), b.read_state())


def test_t_end_clip_lands_exactly():
    kw = kh_kw(32)
    s, g = pair(**kw)
    V = kh_state(s, kw, 32)
    s.set_prim(V)
    g.set_prim(V)
    dt0 = g.dt()
    t_end = 2.5 * dt0
    while g.t < t_end:
        g.step(t_end)
    s.run(10, t_end)  # the extra launches after t_end are device no-ops
    t, _ = s.sync()
    assert t == t_end == g.t
    assert_parity(s.read_state(), g.get_cons(), what="t_end")


def test_nonphysical_state_reported():
    kw = kh_kw(32)
    s = amrvac.AmrSolver(precision="fp64", **kw)
    V = kh_state(s, kw, 32)
    V[3, 3, 5] = -1.0  # negative pressure in one cell
    with pytest.raises(amrvac.AmrError) as ei:
        s.set_prim(V)
    assert ei.value.code == -4


def test_invalid_config_rejected():
    with pytest.raises(amrvac.AmrError):
        amrvac.AmrSolver(ndim=2, block_nx=12, base=[2, 2])
    with pytest.raises(amrvac.AmrError):
        amrvac.AmrSolver(ndim=2, block_nx=16, base=[2, 2], max_blocks=3)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_kh_one_step(precision):
    """2048^2 as 128x128 blocks of 16^2 (the benchmark launch configuration):
    one SSPRK3 step against the oracle, FP64 to 1e-12 per cell, FP32 by L1."""
    kw = kh_kw(2048)
    s, g = pair(precision=precision, **kw)
    V = kh_state(s, kw, 2048)
    s.set_prim(V)
    g.set_prim(V)
    s.step()
    g.step()
    a, b = s.read_state(), g.get_cons()
    if precision == "fp64":
        assert_parity(a, b, what="KH 2048 FP64")
    else:
        l1 = np.sum(np.abs(a[:, 0] - b[:, 0])) / np.sum(np.abs(b[:, 0]))
        assert l1 <= 1e-6, l1


@pytest.mark.parametrize("flux", ["tvdlf", "hll", "hllc"])
@pytest.mark.parametrize("limiter", ["minmod", "vanleer", "koren", "none", "mc", "cada"])
@pytest.mark.parametrize("bnx,base", [(8, [3, 5]), (16, [3, 2])])
def test_2d_fp32_schemes(flux, limiter, bnx, base):
    """FP32 batched kernel: every flux x limiter, ragged last CTA for 8^2 leaves.
    One step: per-cell difference <= 1e-5 of each variable's max norm (float32
    rounding of O(1) flux terms makes a per-cell relative bound meaningless for
    near-zero momenta); 10 steps: normalised L1(rho) <= 1e-5."""
    n = [b * bnx for b in base]
    kw = dict(ndim=2, block_nx=bnx, base=base, gamma=1.4, cfl=0.8, flux=flux, limiter=limiter, rk=3,
              bc="periodic", xmax=(1.0, n[1] / n[0], 1.0))
    s, g = pair(precision="fp32", **kw)
    lev, crd = s.leaves()
    x, gi = centres_for(lev, crd, kw)
    V = inputs.kelvin_helmholtz(x, gi, n[0], seed=11)
    s.set_prim(V)
    g.set_cons(s.read_state())  # same (float-rounded) initial state on both sides
    s.step()
    g.step()
    a1, b1 = s.read_state(), g.get_cons()
    e1 = np.max(np.abs(a1 - b1) / np.max(np.abs(b1), axis=(0, 2), keepdims=True))
    assert e1 <= 1e-5, e1
    for _ in range(9):
        s.step()
        g.step()
    a, b = s.read_state()[:, 0], g.get_cons()[:, 0]
    assert np.sum(np.abs(a - b)) / np.sum(np.abs(b)) <= 1e-5


def test_fp32_totals_and_dt():
    """Last-stage reductions of the FP32 path: float-float totals equal the float64
    sum of the float32 state; the CFL step matches the oracle on the same state."""
    kw = kh_kw(256)
    s, g = pair(precision="fp32", **kw)
    s.set_prim(kh_state(s, kw, 256))
    s.run(5)
    s.sync()
    U = s.read_state()
    dV = (1.0 / 256) ** 2
    want = U.sum(axis=(0, 2)) * dV
    got = s.totals()
    assert np.all(np.abs(got - want) <= 1e-11 * np.maximum(np.abs(want), 1.0)), (got, want)
    g.set_cons(U)
    g.t = s.t
    dt_next = s.step()
    assert dt_next == pytest.approx(g.dt(), rel=1e-5)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_state_io_through_every_buffer_kind(precision):
    """Pageable host arrays (staged), pinned host arrays (read and written in place by the
    conversion kernels), device arrays, and arrays that are not 16-byte aligned (staged) give
    the same state."""
    torch = pytest.importorskip("torch")
    nb = 4
    kw = dict(ndim=2, block_nx=16, base=[nb, nb], gamma=1.4, cfl=0.8, flux="hllc", limiter="vanleer", rk=3,
              bc="periodic")
    s = amrvac.AmrSolver(precision=precision, **kw)
    lev, crd = s.leaves()
    x, gidx = inputs.cell_centres(lev, crd, 2, 16, [nb, nb, 1], [0, 0, 0], [1, 1, 1])
    s.set_prim(inputs.kelvin_helmholtz(x, gidx, nb * 16))
    s.run(2)
    s.sync()
    ref = s.read_state()
    n = ref.size
    host = torch.from_numpy(ref.ravel().copy())
    pinned = host.pin_memory()
    pinned_off = torch.empty(n + 1, dtype=torch.float64).pin_memory()
    pinned_off[1:] = host
    dev = host.cuda()
    dev_off = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    dev_off[1:] = dev
    for src in (host.numpy(), pinned, pinned_off[1:], dev, dev_off[1:]):
        s.set_state(src, primitive=False)
        assert np.array_equal(s.read_state(), ref)
    for out in (torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(n + 1, dtype=torch.float64).pin_memory()[1:],
                torch.empty(n, dtype=torch.float64, device="cuda"),
                torch.empty(n + 1, dtype=torch.float64, device="cuda")[1:]):
        s.read_state(out.view(ref.shape))
        assert np.array_equal(out.cpu().numpy(), ref.ravel())
