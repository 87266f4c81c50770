"""Pins of the seeded input generator (no GPU): splitmix64 against its reference outputs, and
the sampling properties the workloads rely on."""
import numpy as np
import pytest

from paper_2004_03275_gb300 import inputs

# The first three outputs of splitmix64 from state 0 (Steele, Lea and Flood, OOPSLA 2014; the
# widely used reference values of the generator).
SPLITMIX64_FROM_ZERO = (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F)


def test_uniform_is_splitmix64_top_53_bits():
    u = inputs.uniform(0, np.arange(3))
    want = [(z >> 11) / 2.0 ** 53 for z in SPLITMIX64_FROM_ZERO]
    assert list(u) == want


def test_uniform_is_counter_based_and_in_range():
    c = np.arange(100000)
    u = inputs.uniform(2004, c)
    assert np.all((u >= 0.0) & (u < 1.0))
    # any subset regenerates independently, and seeds differ
    idx = np.array([99999, 5, 31337])
    assert np.array_equal(inputs.uniform(2004, idx), u[idx])
    assert not np.array_equal(inputs.uniform(2005, c[:100]), u[:100])
    # first two moments of U(0, 1) within 5 standard errors
    n = len(u)
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)


def test_gray_scott_batch_sizes_are_the_configuration():
    sizes = inputs.gray_scott_batch_sizes()
    assert sizes == [128 * (i + 2) for i in range(15)] + [2048]
    assert sum(n * n for n in sizes) == 28688384  # 28.7 M unknowns per species


@pytest.mark.parametrize("seed", [4000, 4007])
def test_gray_scott_patches_values(seed):
    n = 256
    u, v = inputs.gray_scott_patches(n, L=2.5, seed=seed)
    inside = v > 0
    assert inside.any() and (~inside).any()
    assert np.all(u[~inside] == 1.0) and np.all(v[~inside] == 0.0)
    # patch cells: (0.5, 0.25) times a per-cell factor in [0.99, 1.01]
    assert np.all(np.abs(u[inside] / 0.5 - 1) <= 0.01 + 1e-15)
    assert np.all(np.abs(v[inside] / 0.25 - 1) <= 0.01 + 1e-15)
