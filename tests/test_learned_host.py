"""Host-side logic of the learned-guess training (no GPU): the learning-rate schedule and
the operator's kappa per species."""
import numpy as np
import pytest

from paper_2004_03275_gb300 import learned_guess as LG


@pytest.mark.parametrize("iters", [1, 2, 3, 10, 1500, 5000])
def test_lr_schedule_is_constant_then_decays_to_the_final_fraction(iters):
    lrs = np.array([LG.lr_at(i, iters, 1e-3) for i in range(iters)])
    assert lrs[0] == 1e-3
    assert np.all(np.diff(lrs) <= 1e-18)
    assert np.all(lrs[: iters // 2] == 1e-3)
    if iters >= 3:
        assert lrs[-1] == pytest.approx(5e-5, rel=1e-12)


def test_operator_kappa_matches_the_stiffness_ratio():
    # kappa = lambda h^2 / (2 ndim) with lambda = 2 / (dt D): kappa = h^2 / (ndim dt D) = 1 / (ndim * (D dt / h^2))
    ku, kv = LG.operator_kappa(2048, 2.5, ndim=2)
    h = 2.5 / 2048
    stiff_u = LG.GS["Du"] * LG.GS["dt"] / h ** 2
    assert ku == pytest.approx(1.0 / (2 * stiff_u), rel=1e-12)
    assert kv == pytest.approx(2 * ku, rel=1e-12)
    # the stiffness-matched smaller domain keeps h, hence kappa
    assert LG.operator_kappa(256, LG.domain_for(256)) == pytest.approx((ku, kv), rel=1e-12)
