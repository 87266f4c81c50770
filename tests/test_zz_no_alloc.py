"""The allocation-free CFL/totals entry point (amr_reduce_noalloc) agrees with
the handle-based path (amr_set_state -> amr_conserved_totals, amr_step's dt) on
two calls in a row.  Collected last so that a run stopping at the first failure
has already run every other test."""
import numpy as np
import pytest

from paper_2004_03275_gb300 import amrvac, inputs

pytestmark = pytest.mark.gpu


def kh(nside, bnx=16):
    nb = nside // bnx
    kw = dict(ndim=2, block_nx=bnx, base=[nb, nb], gamma=1.4, cfl=0.8, flux="hllc", limiter="vanleer", rk=3,
              bc="periodic")
    return kw


@pytest.mark.parametrize("nside", [64, 2048])
def test_noalloc_matches_handle_path_twice(nside):
    torch = pytest.importorskip("torch")
    kw = kh(nside)
    s = amrvac.AmrSolver(precision="fp64", **kw)
    lev, crd = s.leaves()
    x, gi = inputs.cell_centres(lev, crd, 2, 16, kw["base"] + [1], [0, 0, 0], [1, 1, 1])
    s.set_prim(inputs.kelvin_helmholtz(x, gi, nside, seed=2004))
    U = s.read_state()
    want_tot = s.totals()
    want_dt = s.step()  # dt of the state above (no t_end clip)
    Ud = torch.from_numpy(U.ravel().copy()).cuda()
    for call in range(2):  # the second call reuses the scratch left by the first
        dt, tot = amrvac.reduce_noalloc(Ud, **kw)
        assert dt == pytest.approx(want_dt, rel=1e-14), call
        assert np.allclose(tot, want_tot, rtol=1e-12, atol=1e-15), (call, tot, want_tot)


def test_noalloc_rejects_too_many_leaves():
    torch = pytest.importorskip("torch")
    kw = kh(16 * 129)  # 129^2 leaves > 16384
    U = torch.ones(1, device="cuda", dtype=torch.float64)
    with pytest.raises(amrvac.AmrError) as ei:
        amrvac.reduce_noalloc(U, **kw)
    assert ei.value.code == -7


def test_noalloc_binding_rejects_wrong_dtype_and_short_state():
    """The kernel reads nleaves * (ndim + 2) * B^ndim float64 values through a bare pointer, so the
    binding refuses a float32 state or a short one on the host, before any launch."""
    torch = pytest.importorskip("torch")
    kw = kh(64)
    need = 16 * 4 * 256
    with pytest.raises(ValueError):
        amrvac.reduce_noalloc(torch.zeros(need, device="cuda", dtype=torch.float32), **kw)
    with pytest.raises(ValueError):
        amrvac.reduce_noalloc(torch.zeros(need - 1, device="cuda", dtype=torch.float64), **kw)
