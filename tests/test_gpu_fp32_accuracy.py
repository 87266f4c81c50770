"""Accuracy of the float32 path against the FP64 oracle, as the normalised L1 of the
density, sum |rho32 - rho_oracle| / sum |rho_oracle|:

* 3D blast, base 2^3 blocks of 16^3, 3 levels (effective 128^3), HLLC + Koren, SSPRK3,
  100 steps with a regrid after every 10.  The float32 run may flag a block differently
  from the oracle, so both states are projected onto the uniform 128^3 grid and both
  runs regrid at the oracle's regrid times.  Stated accuracy: <= 1e-3.
* Kelvin-Helmholtz 256^2 (HLLC + van Leer), 100 steps, at the oracle's time.  Stated
  accuracy: <= 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac, inputs
from paper_2004_03275_gb300.analysis import l1_relative, project_uniform

pytestmark = pytest.mark.gpu

BASE = [2, 2, 2]
KW = dict(ndim=3, block_nx=16, base=BASE, max_level=3, gamma=5.0 / 3.0, cfl=0.8, flux="hllc", limiter="koren",
          rk=3, bc="periodic", refine_tol=0.2, coarsen_frac=0.5, var_mask=1 | 16)


def refine_initial(g):
    for it in range(3):
        lev, crd = g.leaves()
        x, _ = inputs.cell_centres(lev, crd, 3, 16, BASE, [0, 0, 0], [1, 1, 1])
        g.set_prim(inputs.blast(x, seed=7))
        if it < 2:
            g.regrid()


def catch_up(s, t, nsteps):
    for _ in range(4):  # float32 dt may differ from the oracle's in the last digits
        if s.t >= t:
            break
        s.run(nsteps, t_end=t)
        s.sync()
    assert s.t == pytest.approx(t, rel=1e-12, abs=0)


def test_blast_128_fp32_l1_with_regrids():
    g = O.Grid(**KW)
    s = amrvac.AmrSolver(**KW, precision="fp32")
    refine_initial(g)
    refine_initial(s)
    assert np.array_equal(np.sort(g.leaves()[0]), np.sort(s.leaves()[0]))
    for blk in range(10):
        g.run(10)
        catch_up(s, g.t, 10)
        if blk < 9:
            g.regrid()
            s.regrid()
    lo, co = g.leaves()
    ls, cs = s.leaves()
    r64 = project_uniform(lo, co, g.get_cons()[:, 0], 3, 16, BASE, 3)
    r32 = project_uniform(ls, cs, s.read_state()[:, 0], 3, 16, BASE, 3)
    err = l1_relative(r32, r64)
    print(f"blast 128^3 float32 L1(rho) after 100 steps with regrids: {err:.3e} ({len(ls)} / {len(lo)} leaves)")
    assert err <= 1e-3
    s.close()


def test_kh_256_fp32_l1():
    nb = 16
    kw = dict(ndim=2, block_nx=16, base=[nb, nb], gamma=1.4, cfl=0.8, flux="hllc", limiter="vanleer", rk=3,
              bc="periodic")
    g = O.Grid(**kw)
    s = amrvac.AmrSolver(**kw, precision="fp32")
    lev, crd = g.leaves()
    x, gi = inputs.cell_centres(lev, crd, 2, 16, [nb, nb, 1], [0, 0, 0], [1, 1, 1])
    V = inputs.kelvin_helmholtz(x, gi, 256, seed=2004)
    g.set_prim(V)
    s.set_prim(V)
    g.run(100)
    catch_up(s, g.t, 100)
    err = l1_relative(s.read_state()[:, 0], g.get_cons()[:, 0])
    print(f"KH 256^2 float32 L1(rho) after 100 steps: {err:.3e}")
    assert err <= 1e-4
    s.close()
