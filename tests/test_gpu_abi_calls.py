"""GPU tests of the boundary calls that compose other calls: the initial condition from a host
callback (amr_set_state_fn, with its initial refinement passes, Sec. 1.3), inference under its own
name with the parameter file round trip (cnn_infer, cnn_save, cnn_load), and a float64 run that
is checkpointed and resumed (bit-identical continuation)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from gpu_util import assert_parity, centres_for

pytestmark = pytest.mark.gpu


def kh_kw(n=64, bnx=16):
    return dict(ndim=2, block_nx=bnx, base=[n // bnx, n // bnx], gamma=1.4, cfl=0.8, flux="hllc",
                limiter="vanleer", rk=3, bc="periodic")


def test_set_state_fn_matches_set_prim_on_one_level():
    """The callback sees each cell centre x = xmin + (g + 1/2) dx: sampling Kelvin-Helmholtz through it
    gives the same conserved state, bit for bit, as converting the array of the same samples."""
    n = 64
    kw = kh_kw(n)
    a = amrvac.AmrSolver(precision="fp64", **kw)
    lev, crd = a.leaves()
    x, gi = inputs.cell_centres(lev, crd, 2, 16, kw["base"] + [1], [0, 0, 0], [1, 1, 1])
    V = inputs.kelvin_helmholtz(x, gi, n, seed=2004)
    a.set_prim(V)
    seen = []

    def prim_at(xc):
        i, j = int(xc[0] * n), int(xc[1] * n)
        assert xc[0] == (i + 0.5) / n and xc[1] == (j + 0.5) / n and xc[2] == 0.0
        seen.append((i, j))
        xp = np.array([xc[0], xc[1], 0.0]).reshape(1, 3, 1)
        return inputs.kelvin_helmholtz(xp, np.array([i, j, 0]).reshape(1, 3, 1), n, seed=2004)[0, :, 0]

    b = amrvac.AmrSolver(precision="fp64", **kw)
    b.set_state_fn(prim_at)
    assert len(seen) == n * n and len(set(seen)) == n * n  # one pass (max_level 1), every cell once
    assert np.array_equal(a.read_state(), b.read_state())
    assert np.array_equal(a.totals(), b.totals())


@pytest.mark.parametrize("ndim", [2, 3])
def test_set_state_fn_refines_like_the_sample_regrid_loop(ndim):
    """With max_level 3 the call samples, regrids and resamples twice.  The same loop written with
    set_prim and regrid on another handle, and with the oracle, gives the same tree; the states are
    identical on the GPU and agree with the oracle's to 1e-12."""
    bnx, base, L = 8, [2] * ndim, 3
    kw = dict(ndim=ndim, block_nx=bnx, base=base, max_level=L, gamma=5.0 / 3.0, cfl=0.8, flux="hllc",
              limiter="koren", rk=3, bc="periodic", var_mask=1 | (1 << (ndim + 1)))
    bl = dict(seed=7, ndim=ndim, radius=0.2, p_in=100.0)

    def prim_at(xc):
        return inputs.blast(np.array(xc, dtype=np.float64).reshape(1, 3, 1), **bl)[0, :, 0]

    a = amrvac.AmrSolver(precision="fp64", **kw)
    a.set_state_fn(prim_at)
    b = amrvac.AmrSolver(precision="fp64", **kw)
    g = O.Grid(**kw)
    for p in range(L):
        if p > 0:
            b.regrid()
            g.regrid()
        lev, crd = b.leaves()
        x, _ = centres_for(lev, crd, kw)
        V = inputs.blast(x, **bl)
        b.set_prim(V)
        g.set_prim(V)
    la, ca = a.leaves()
    lb, cb = b.leaves()
    lo, co = g.leaves()
    assert la.max() == L
    assert np.array_equal(la, lb) and np.array_equal(ca, cb)
    assert np.array_equal(la, lo) and np.array_equal(ca, co)
    assert np.array_equal(a.read_state(), b.read_state())
    assert_parity(a.read_state(), g.get_cons(), what="set_state_fn vs oracle")


def test_set_state_fn_reports_a_failing_callback():
    kw = kh_kw(32)
    s = amrvac.AmrSolver(precision="fp64", **kw)

    def bad(xc):
        raise KeyError("no value here")

    with pytest.raises(KeyError):
        s.set_state_fn(bad)


def test_cnn_infer_save_load_round_trip(tmp_path):
    """cnn_infer is cnn_forward under the inference name (identical outputs); a saved parameter file
    loads into a network of another seed with identical parameters and identical outputs; a
    truncated file or one of the other dimension is refused and leaves the parameters unchanged."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(0, 1, size=(2, 5, 32, 48)).astype(np.float32)).cuda()
    a = amrvac.CnnNet(ndim=2, seed=11)
    ya = a.forward(x).clone()
    yi = a.infer(x)
    assert torch.equal(ya, yi)
    path = str(tmp_path / "net.bin")
    a.save(path)
    b = amrvac.CnnNet(ndim=2, seed=12)
    assert not np.array_equal(a.get_params(), b.get_params())
    b.load(path)
    assert np.array_equal(a.get_params(), b.get_params())
    assert torch.equal(b.infer(x), ya)
    # a truncated file and a 3D file are refused; the network keeps its parameters
    raw = open(path, "rb").read()
    short = str(tmp_path / "short.bin")
    open(short, "wb").write(raw[:-4])
    c = amrvac.CnnNet(ndim=2, seed=13)
    p0 = c.get_params()
    with pytest.raises(amrvac.AmrError) as ei:
        c.load(short)
    assert ei.value.code == -1
    assert np.array_equal(c.get_params(), p0)
    d3 = amrvac.CnnNet(ndim=3, seed=14)
    p3 = str(tmp_path / "net3.bin")
    d3.save(p3)
    with pytest.raises(amrvac.AmrError):
        c.load(p3)
    assert np.array_equal(c.get_params(), p0)


@pytest.mark.parametrize("tree", [False, True])
def test_checkpoint_resume_is_bit_identical_fp64(tmp_path, tree):
    """N steps straight through equal N/2 steps, a checkpoint, a fresh solver loading it and N/2 more
    steps, bit for bit (float64; a uniform KH grid and a 2D blast tree with level jumps)."""
    if tree:
        kw = dict(ndim=2, block_nx=8, base=[2, 2], max_level=3, gamma=5.0 / 3.0, cfl=0.8, flux="hllc",
                  limiter="koren", rk=3, bc="periodic", var_mask=1 | 8)

        def init(s):
            s.set_state_fn(lambda xc: inputs.blast(np.array(xc).reshape(1, 3, 1), seed=7, ndim=2, radius=0.2,
                                                   p_in=100.0)[0, :, 0])
    else:
        kw = kh_kw(64)

        def init(s):
            lev, crd = s.leaves()
            x, gi = inputs.cell_centres(lev, crd, 2, 16, kw["base"] + [1], [0, 0, 0], [1, 1, 1])
            s.set_prim(inputs.kelvin_helmholtz(x, gi, 64, seed=2004))

    N = 8
    a = amrvac.AmrSolver(precision="fp64", **kw)
    init(a)
    for _ in range(N):
        a.step()
    b = amrvac.AmrSolver(precision="fp64", **kw)
    init(b)
    for _ in range(N // 2):
        b.step()
    path = tmp_path / "ck.npz"
    amrvac.save_checkpoint(b, path, steps=N // 2)
    b.close()
    c = amrvac.AmrSolver(precision="fp64", **kw)
    assert amrvac.load_checkpoint(c, path) == N // 2
    for _ in range(N - N // 2):
        c.step()
    la, ca = a.leaves()
    lc, cc = c.leaves()
    assert np.array_equal(la, lc) and np.array_equal(ca, cc)
    assert np.array_equal(a.read_state(), c.read_state())
    assert a.t == c.t
