"""The learned multigrid guess against the previous-step guess (Gray-Scott IMEX at
the stiffness of the 2048^2 configuration, D dt / h^2 = 6.7 for u).

Trained on seeds disjoint from evaluation, the network must learn (its masked
MSE over the whole training set falls), the multigrid must reach the same 1e-10 tolerance from the learned
guess (fallback guarantee), the solution must agree with the plain run, and the
learned guess must never cost more V-cycles than the previous-step guess.  The
measured V-cycles, initial residuals and wall times are what the trained
network gains; the benchmark reports them at 2048^2."""
import numpy as np
import pytest

from paper_2004_03275_gb300 import amrvac, learned_guess as LG

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_learned_guess_against_previous_step_guess():
    n = 256
    L = LG.domain_for(n)
    X, Y, scale = LG.generate(torch, [n, n], [0, 1], L, steps=24, crops_per_step=48, crop=64, warm=40)
    assert X.shape[0] == 24 * 48 and np.isfinite(scale) and scale > 0
    net = amrvac.CnnNet(ndim=2, seed=3)
    before = LG.dataset_loss(torch, net, X, Y)
    losses, secs = LG.train(torch, net, X, Y, iters=1500, batch=64, lr=1e-3)
    after = LG.dataset_loss(torch, net, X, Y)
    assert after < 0.8 * before, (before, after)
    seeds = [10000]
    c_plain, t_plain, (u0, v0), r_plain = LG.evaluate(torch, [n], seeds, L, steps=8, warm=40)
    c_net, t_net, (u1, v1), r_net = LG.evaluate(torch, [n], seeds, L, steps=8, warm=40, net=net, scale=scale)
    assert np.mean(c_net) <= np.mean(c_plain), (c_net.ravel(), c_plain.ravel())
    assert np.all(np.isfinite(r_net)) and np.median(r_net) <= np.median(r_plain) * 1.01
    # both runs reach 1e-10 every step, so the states agree to that level
    assert np.max(np.abs(u1 - u0)) < 1e-8 and np.max(np.abs(v1 - v0)) < 1e-8


def test_learned_guess_3d_trains_and_keeps_the_tolerance():
    """3D (configuration 5's 256^3 case at small size): the 3D network trains on 3D
    crops of the plain solver's steps, and from its guess the multigrid still reaches
    1e-10 every step, so the state matches the plain run."""
    n = 32
    L = LG.domain_for(n, ref_n=256, ref_L=2.5)
    X, Y, scale = LG.generate(torch, [n], [0], L, steps=6, crops_per_step=8, crop=16, warm=10, ndim=3)
    assert tuple(X.shape) == (48, 5, 16, 16, 16) and tuple(Y.shape) == (48, 2, 16, 16, 16)
    assert np.isfinite(scale) and scale > 0
    net = amrvac.CnnNet(ndim=3, seed=3)
    before = LG.dataset_loss(torch, net, X, Y)
    LG.train(torch, net, X, Y, iters=300, batch=4, lr=1e-3)
    after = LG.dataset_loss(torch, net, X, Y)
    assert after < 0.8 * before, (before, after)
    c0, _, (u0, v0), _ = LG.evaluate(torch, [48], [10000], 2.5 * 48 / 256, steps=3, warm=10, ndim=3)
    c1, _, (u1, v1), r1 = LG.evaluate(torch, [48], [10000], 2.5 * 48 / 256, steps=3, warm=10, ndim=3, net=net,
                                      scale=scale)
    assert np.all(np.isfinite(r1)) and np.all(c1 >= 1)
    assert np.max(np.abs(u1 - u0)) < 1e-8 and np.max(np.abs(v1 - v0)) < 1e-8
