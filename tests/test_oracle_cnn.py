"""Pins of the oracle's CNN (the learned multigrid guess): gradients against
central finite differences, tap orientation from impulse responses, periodic
translation equivariance, GELU and Adam closed forms (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O


def rand_params(ndim, rng, scale=0.3):
    p = np.zeros(O.cnn_num_params(ndim))
    for ws, bs, ci, co in O.cnn_layer_slices(ndim):
        T = 27 if ndim == 3 else 9
        p[ws] = rng.normal(size=co * ci * T) * scale / math.sqrt(ci * T) * 3
        p[bs] = rng.normal(size=co) * 0.1
    return p


def test_gelu_closed_forms():
    assert O.gelu(0.0) == 0.0
    assert O.gelu_d(0.0) == 0.5
    for z in (0.3, 1.7, -2.2):
        assert O.gelu(z) - O.gelu(-z) == pytest.approx(z, rel=1e-14)  # Phi(z) + Phi(-z) = 1
        assert O.gelu(z) == pytest.approx(0.5 * z * math.erfc(-z / math.sqrt(2)), rel=1e-14)
        h = 1e-6
        assert O.gelu_d(z) == pytest.approx((O.gelu(z + h) - O.gelu(z - h)) / (2 * h), rel=1e-8)


@pytest.mark.parametrize("ndim,shape,margin", [(2, (2, 5, 8, 8), 1), (3, (1, 5, 4, 4, 4), 1)])
def test_gradient_matches_finite_differences(ndim, shape, margin):
    rng = np.random.default_rng(ndim)
    p = rand_params(ndim, rng)
    x = rng.uniform(0, 1, size=shape)
    tgt = rng.normal(size=(shape[0], 2) + shape[2:]) * 0.1
    loss, g = O.cnn_loss_grad(p, x, tgt, margin=margin, ndim=ndim)
    idx = rng.choice(len(p), size=120, replace=False)
    # include every bias and the last layer
    idx = np.unique(np.concatenate([idx, np.arange(len(p) - 2, len(p))]))
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.cnn_loss_grad(pp, x, tgt, margin, ndim)[0] - O.cnn_loss_grad(pm, x, tgt, margin, ndim)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), abs(g[i])) + 1e-11, (i, fd, g[i])


def test_zero_weights_give_last_bias():
    p = np.zeros(O.cnn_num_params(2))
    ws, bs, _, _ = O.cnn_layer_slices(2)[3]
    p[bs] = [0.25, -1.5]
    out = O.cnn_forward(p, np.random.default_rng(0).uniform(size=(1, 5, 6, 6)))
    assert np.all(out[0, 0] == 0.25) and np.all(out[0, 1] == -1.5)


def test_tap_orientation_impulse():
    """Layer 1 uses only the tap at offset (dx, dy) = (+1, 0); layers 2-4 only
    their centre tap.  z[p] = sum W x[p + off], so an impulse at p0 appears at
    p0 - off = (x0 - 1, y0) and nowhere else."""
    p = np.zeros(O.cnn_num_params(2))
    sl = O.cnn_layer_slices(2)
    for l, (ws, bs, ci, co) in enumerate(sl):
        W = np.zeros((co, ci, 9))
        tap = 5 if l == 0 else 4  # t = (dy+1)*3 + (dx+1): (0,+1) -> 5, centre -> 4
        W[0, 0, tap] = 1.0
        p[ws] = W.ravel()
    x = np.zeros((1, 5, 7, 9))
    y0, x0 = 3, 4
    x[0, 0, y0, x0] = 1.0
    out = O.cnn_forward(p, x)
    nz = np.argwhere(np.abs(out[0, 0]) > 0)
    assert nz.tolist() == [[y0, x0 - 1]]
    assert out[0, 0, y0, x0 - 1] == pytest.approx(O.gelu(O.gelu(O.gelu(1.0))), rel=1e-15)
    assert np.all(out[0, 1] == 0)


def test_periodic_translation_equivariance():
    rng = np.random.default_rng(3)
    p = rand_params(2, rng)
    x = rng.uniform(size=(1, 5, 8, 10))
    out = O.cnn_forward(p, x)
    xs = np.roll(x, shift=(3, -2), axis=(2, 3))
    outs = O.cnn_forward(p, xs)
    assert np.allclose(outs, np.roll(out, shift=(3, -2), axis=(2, 3)), rtol=1e-13, atol=1e-14)


def test_adam_first_step_closed_form():
    """t = 1: m_hat = g, v_hat = g^2, so each parameter moves by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    O.cnn_adam(p, g, m, v, 1, lr=1e-3)
    assert np.allclose(p, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_training_reduces_loss():
    """A few Adam steps on a fixed batch reduce the loss (the oracle's training loop works)."""
    rng = np.random.default_rng(5)
    p = rand_params(2, rng)
    x = rng.uniform(size=(2, 5, 8, 8))
    tgt = 0.1 * np.sin(x[:, :2] * 3)
    m, v = np.zeros_like(p), np.zeros_like(p)
    l0 = O.cnn_loss_grad(p, x, tgt)[0]
    for t in range(1, 31):
        loss, g = O.cnn_loss_grad(p, x, tgt)
        O.cnn_adam(p, g, m, v, t, lr=3e-3)
    assert O.cnn_loss_grad(p, x, tgt)[0] < 0.5 * l0
