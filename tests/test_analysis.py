"""Projection of a block-tree field onto a uniform grid (used for float32 accuracy
figures on trees that may differ between precisions): exact on trees whose leaves are
all on the target level, block means for finer leaves, replication for coarser ones,
and errors for trees that overlap or leave a hole."""
import numpy as np
import pytest

from paper_2004_03275_gb300.analysis import l1_relative, project_uniform


def uniform_leaves(base, level, ndim):
    n = [b * 2 ** (level - 1) for b in base[:ndim]]
    crd = np.array([c[::-1] for c in np.ndindex(*n[::-1])]).reshape(-1, ndim)
    return np.full(len(crd), level), crd


def test_uniform_tree_reassembles_exactly_2d():
    B, base = 4, [2, 3]
    lev, crd = uniform_leaves(base, 2, 2)
    big = np.random.default_rng(0).standard_normal((3 * B * 2, 2 * B * 2))  # (y, x)
    field = np.stack([big[c[1] * B:(c[1] + 1) * B, c[0] * B:(c[0] + 1) * B].ravel() for c in crd])
    out = project_uniform(lev, crd, field, 2, B, base, 2)
    assert np.array_equal(out, big)
    # one level down: means of 2 x 2 cells
    coarse = project_uniform(lev, crd, field, 2, B, base, 1)
    assert np.allclose(coarse, big.reshape(3 * B, 2, 2 * B, 2).mean(axis=(1, 3)), rtol=0, atol=1e-15)


def test_coarse_leaf_is_replicated_3d():
    # two level-1 blocks along x: the first stays a leaf, the second is split into 8 level-2 leaves
    B, base = 2, [2, 1, 1]
    lev = [1] + [2] * 8
    crd = [[0, 0, 0]] + [[2 + i, j, k] for k in range(2) for j in range(2) for i in range(2)]
    rng = np.random.default_rng(1)
    field = rng.standard_normal((9, B ** 3))
    out = project_uniform(lev, crd, field, 3, B, base, 2)
    assert out.shape == (4, 4, 8)
    coarse = field[0].reshape(B, B, B)
    for z in range(4):
        for y in range(4):
            for x in range(4):
                assert out[z, y, x] == coarse[z // 2, y // 2, x // 2]
    # a fine leaf lands where its coordinates say
    k = 1 + 1 + 2 * 0 + 4 * 1  # the leaf at (3, 0, 1)
    assert np.array_equal(out[2:4, 0:2, 6:8], field[k].reshape(B, B, B))


def test_rejects_overlap_and_holes():
    B, base = 2, [2, 1]
    with pytest.raises(ValueError):
        project_uniform([1, 1], [[0, 0], [0, 0]], np.zeros((2, 4)), 2, B, base, 1)
    with pytest.raises(ValueError):
        project_uniform([1], [[0, 0]], np.zeros((1, 4)), 2, B, base, 1)


def test_l1_relative():
    assert l1_relative([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert l1_relative([1.5, 2.0], [1.0, 3.0]) == pytest.approx(1.5 / 4.0)
