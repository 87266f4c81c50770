"""Checkpoint files of the block-tree solver (host logic, no GPU): a round trip through a
stand-in object with the solver's calls restores tree, state and time exactly, and a file
of another geometry is refused."""
import numpy as np
import pytest

from paper_2004_03275_gb300 import amrvac


class FakeSolver:
    """Holds what the checkpoint reads and writes, with the AmrSolver call signatures."""

    def __init__(self, ndim=2, block_nx=8, base=(2, 3, 1), max_level=3):
        self.cfg = amrvac.AmrConfig()
        self.cfg.ndim, self.cfg.block_nx, self.cfg.max_level = ndim, block_nx, max_level
        for d in range(3):
            self.cfg.base_nblocks[d] = base[d]
        self.lev = np.ones(base[0] * base[1], dtype=np.int32)
        self.crd = np.array([[i % base[0], i // base[0], 0] for i in range(len(self.lev))], dtype=np.int32)
        self.U = np.zeros((len(self.lev), ndim + 2, block_nx ** ndim))
        self.t = 0.0

    def leaves(self):
        return self.lev.copy(), self.crd.copy()

    def read_state(self):
        return self.U.copy()

    def set_leaves(self, level, coords):
        self.lev = np.asarray(level, dtype=np.int32).copy()
        self.crd = np.asarray(coords, dtype=np.int32).reshape(-1, 3).copy()
        self.U = np.zeros((len(self.lev),) + self.U.shape[1:])

    def set_state(self, W, primitive=True):
        assert primitive is False
        self.U = np.asarray(W, dtype=np.float64).reshape(self.U.shape).copy()

    def set_time(self, t):
        self.t = t


def test_round_trip_restores_tree_state_and_time(tmp_path):
    rng = np.random.default_rng(1)
    a = FakeSolver()
    # a refined tree: the first base block split into four level-2 blocks
    lev = np.array([2, 2, 2, 2, 1, 1, 1, 1, 1], dtype=np.int32)
    crd = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 2, 0],
                    [1, 2, 0]], dtype=np.int32)
    a.set_leaves(lev, crd)
    a.U = rng.normal(size=a.U.shape)
    a.t = 0.123456789012345
    path = tmp_path / "ck.npz"
    amrvac.save_checkpoint(a, path)
    b = FakeSolver()
    amrvac.load_checkpoint(b, path)
    assert np.array_equal(b.lev, lev) and np.array_equal(b.crd, crd)
    assert np.array_equal(b.U, a.U) and b.t == a.t


@pytest.mark.parametrize("other", [dict(ndim=3, base=(2, 3, 1)), dict(block_nx=16), dict(base=(3, 3, 1)),
                                   dict(max_level=4)])
def test_other_geometry_is_refused(tmp_path, other):
    a = FakeSolver()
    path = tmp_path / "ck.npz"
    amrvac.save_checkpoint(a, path)
    with pytest.raises(ValueError):
        amrvac.load_checkpoint(FakeSolver(**other), path)


@pytest.mark.parametrize("field,value", [("gamma", 5 / 3), ("cfl", 0.5), ("flux", 1), ("limiter", 2), ("rk", 2),
                                         ("precision", 1), ("refine_tol", 0.1), ("coarsen_frac", 0.25),
                                         ("wavefilter", 0.02), ("refine_var_mask", 3)])
def test_other_physics_or_scheme_is_refused(tmp_path, field, value):
    """A file written under one scheme, physics or refinement setting does not load into a solver
    with another: the continuation would not repeat the saved run."""
    a = FakeSolver()
    path = tmp_path / "ck.npz"
    amrvac.save_checkpoint(a, path, steps=7)
    b = FakeSolver()
    assert amrvac.load_checkpoint(b, path) == 7
    c = FakeSolver()
    setattr(c.cfg, field, value)
    with pytest.raises(ValueError, match=field):
        amrvac.load_checkpoint(c, path)


def test_other_domain_or_boundaries_are_refused(tmp_path):
    a = FakeSolver()
    path = tmp_path / "ck.npz"
    amrvac.save_checkpoint(a, path)
    b = FakeSolver()
    b.cfg.xmax[0] = 2.0
    with pytest.raises(ValueError, match="xmax"):
        amrvac.load_checkpoint(b, path)
    c = FakeSolver()
    c.cfg.bc[1][0] = 1
    with pytest.raises(ValueError, match="bc"):
        amrvac.load_checkpoint(c, path)
    np.savez(tmp_path / "x.npz", kind="something else")
    with pytest.raises(ValueError):
        amrvac.load_checkpoint(FakeSolver(), tmp_path / "x.npz")
