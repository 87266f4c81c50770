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


# ---- operator-weighted loss: q = (1 + kappa) e - (1/(2 ndim)) sum_faces e, e = out - target ----

def test_operator_loss_of_a_fourier_mode_closed_form():
    """For e = cos(theta i + phi) along x, every counted pixel has q = (kappa + (1 - cos theta)/ndim) e:
    the symbol of the normalised 5/7-point operator."""
    rng = np.random.default_rng(21)
    for ndim, shape in ((2, (1, 2, 6, 20)), (3, (1, 2, 5, 4, 12))):
        W = shape[-1]
        m, phi = 3, 0.4
        theta = 2 * np.pi * m / W
        i = np.arange(W)
        e = np.broadcast_to(np.cos(theta * i + phi), shape).copy()
        tgt = rng.normal(size=shape)
        kappa = (0.25, 0.0625)
        margin = 1
        loss, _ = O.cnn_output_loss(tgt + e, tgt, margin=margin, ndim=ndim, loss="operator", kappa=kappa)
        sl = (slice(None),) + tuple(slice(margin, n - margin) for n in shape[2:])
        want = []
        for c in range(2):
            q = (kappa[c] + (1 - np.cos(theta)) / ndim) * e[:, c]
            want.append(q[sl] ** 2)
        want = np.mean(np.stack(want))
        assert loss == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("ndim,n", [(2, 16), (3, 8)])
def test_operator_loss_is_the_scaled_residual_of_the_guess(ndim, n):
    """With target = (w* - w_n)/s and the guess X = w_n + s out, the multigrid oracle's own
    operator gives lambda g - A X = A (w* - X) = s (2 ndim / h^2) q on every counted pixel, for
    kappa = lambda h^2 / (2 ndim) per species."""
    rng = np.random.default_rng(7 + ndim)
    L, s = 2.5, 0.01
    h = L / n
    lams = (2.0 / (0.5 * 2e-5), 2.0 / (0.5 * 1e-5))
    shape = (n,) * ndim
    wn = rng.uniform(0.2, 1.0, size=(2,) + shape)
    ws = wn + s * rng.normal(size=(2,) + shape)
    out = rng.normal(size=(2,) + shape)
    tgt = (ws - wn) / s
    kappa = [lam * h * h / (2 * ndim) for lam in lams]
    margin = 1
    loss, _ = O.cnn_output_loss(out[None], tgt[None], margin=margin, ndim=ndim, loss="operator", kappa=kappa)
    sl = tuple(slice(margin, n - margin) for _ in range(ndim))
    terms = []
    for c in range(2):
        X = wn[c] + s * out[c]
        r = O.mg_apply(ws[c], L, lams[c]) - O.mg_apply(X, L, lams[c])
        terms.append((r * h * h / (2 * ndim * s))[sl] ** 2)
    assert loss == pytest.approx(np.mean(np.stack(terms)), rel=1e-9)


def test_operator_loss_tends_to_mse_for_large_kappa():
    rng = np.random.default_rng(4)
    out, tgt = rng.normal(size=(2, 2, 9, 11)), rng.normal(size=(2, 2, 9, 11))
    k = 1e7
    lo, go = O.cnn_output_loss(out, tgt, margin=2, loss="operator", kappa=(k, k))
    lm, gm = O.cnn_output_loss(out, tgt, margin=2, loss="mse")
    assert lo / (1 + k) ** 2 == pytest.approx(lm, rel=1e-6)
    assert np.max(np.abs(go / (1 + k) ** 2 - gm)) <= 1e-6 * np.max(np.abs(gm))
    with pytest.raises(ValueError):
        O.cnn_output_loss(out, tgt, margin=0, loss="operator", kappa=(k, k))


@pytest.mark.parametrize("ndim", [2, 3])
def test_operator_loss_output_gradient_matches_finite_differences(ndim):
    rng = np.random.default_rng(30 + ndim)
    shape = (2, 2, 7, 9) if ndim == 2 else (1, 2, 5, 6, 7)
    out, tgt = rng.normal(size=shape), rng.normal(size=shape)
    kappa = (0.3, 0.07)
    _, g = O.cnn_output_loss(out, tgt, margin=1, ndim=ndim, loss="operator", kappa=kappa)
    flat = out.reshape(-1)
    h = 1e-2  # the loss is quadratic in the outputs: central differences are exact up to rounding
    for i in rng.choice(flat.size, size=60, replace=False).tolist() + [0, flat.size - 1]:
        op, om = flat.copy(), flat.copy()
        op[i] += h
        om[i] -= h
        fp = O.cnn_output_loss(op.reshape(shape), tgt, margin=1, ndim=ndim, loss="operator", kappa=kappa)[0]
        fm = O.cnn_output_loss(om.reshape(shape), tgt, margin=1, ndim=ndim, loss="operator", kappa=kappa)[0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g.reshape(-1)[i]) <= 1e-10, (i, fd, g.reshape(-1)[i])


@pytest.mark.parametrize("ndim,shape", [(2, (1, 5, 10, 10)), (3, (1, 5, 6, 6, 6))])
def test_operator_loss_parameter_gradient_matches_finite_differences(ndim, shape):
    rng = np.random.default_rng(40 + ndim)
    p = rand_params(ndim, rng)
    x = rng.uniform(0, 1, size=shape)
    tgt = rng.normal(size=(shape[0], 2) + shape[2:]) * 0.1
    kw = dict(margin=2, ndim=ndim, loss="operator", kappa=(0.15, 0.075))
    _, g = O.cnn_loss_grad(p, x, tgt, **kw)
    idx = np.unique(np.concatenate([rng.choice(len(p), size=60, replace=False), np.arange(len(p) - 2, len(p))]))
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.cnn_loss_grad(pp, x, tgt, **kw)[0] - O.cnn_loss_grad(pm, x, tgt, **kw)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), abs(g[i])) + 1e-11, (i, fd, g[i])


@pytest.mark.parametrize("ndim", [2, 3])
def test_receptive_field_is_four_cells(ndim):
    """Four layers of 3^ndim taps: an output depends on the inputs within Chebyshev distance 4
    and on no input farther away; a crop with that margin reproduces the full image's output."""
    rng = np.random.default_rng(70 + ndim)
    p = rand_params(ndim, rng)
    shape = (1, 5, 24, 24) if ndim == 2 else (1, 5, 12, 12, 12)
    x = rng.uniform(0, 1, size=shape)
    out = O.cnn_forward(p, x, ndim=ndim)
    c = tuple(s // 2 for s in shape[2:])
    for dist, changes in ((4, True), (5, False)):
        xp = x.copy()
        idx = (0, 1) + tuple(ci + (dist if d == 0 else 0) for d, ci in enumerate(c))
        xp[idx] += 0.5
        o2 = O.cnn_forward(p, xp, ndim=ndim)
        diff = np.max(np.abs(o2[(0, slice(None)) + c] - out[(0, slice(None)) + c]))
        assert (diff > 1e-9) == changes, (dist, diff)
    # a crop of side 9 (radius 4) around a pixel gives the same output at its centre
    sl = (slice(None), slice(None)) + tuple(slice(ci - 4, ci + 5) for ci in c)
    oc = O.cnn_forward(p, x[sl], ndim=ndim)
    centre = (0, slice(None)) + (4,) * ndim
    assert np.max(np.abs(oc[centre] - out[(0, slice(None)) + c])) <= 1e-12
