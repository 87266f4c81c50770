"""GPU kernels of the learned multigrid guess against the FP64 oracle CNN.

The GPU network runs bf16 weights and activations with fp32 accumulation; both
sides get the same bf16-representable weights and inputs.  Tolerances follow
from bf16 activation rounding (2^-9 relative per value, four layers):
forward outputs within 3e-2 of their max norm, gradients per layer within 5e-2
relative L2 with cosine similarity >= 0.998."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2004_03275_gb300 import amrvac

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf16_round(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def rand_params(ndim, rng):
    p = np.zeros(O.cnn_num_params(ndim))
    T = 27 if ndim == 3 else 9
    for ws, bs, ci, co in O.cnn_layer_slices(ndim):
        p[ws] = rng.normal(size=co * ci * T) * math.sqrt(2.0 / (ci * T))
        p[bs] = rng.normal(size=co) * 0.1
    return bf16_round(p).astype(np.float64)


@pytest.mark.parametrize("ndim,shape", [(2, (2, 5, 32, 48)), (3, (1, 5, 8, 16, 8))])
def test_forward_matches_oracle(ndim, shape):
    rng = np.random.default_rng(10 + ndim)
    p = rand_params(ndim, rng)
    x = bf16_round(rng.uniform(0, 1, size=shape)).astype(np.float64)
    net = amrvac.CnnNet(ndim=ndim)
    net.set_params(p)
    assert np.array_equal(net.get_params().astype(np.float64), p)
    out = net.forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    ref = O.cnn_forward(p, x, ndim=ndim)
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    assert err <= 3e-2, err


@pytest.mark.parametrize("ndim,shape,margin", [(2, (2, 5, 32, 32), 2), (3, (1, 5, 8, 8, 8), 1)])
def test_gradient_matches_oracle(ndim, shape, margin):
    rng = np.random.default_rng(20 + ndim)
    p = rand_params(ndim, rng)
    x = bf16_round(rng.uniform(0, 1, size=shape)).astype(np.float64)
    tgt = 0.05 * rng.normal(size=(shape[0], 2) + shape[2:])
    net = amrvac.CnnNet(ndim=ndim)
    net.set_params(p)
    loss, g = net.gradient(torch.from_numpy(x.astype(np.float32)).cuda(),
                           torch.from_numpy(tgt.astype(np.float32)).cuda(), margin=margin)
    lo, go = O.cnn_loss_grad(p, x, tgt, margin=margin, ndim=ndim)
    assert loss == pytest.approx(lo, rel=3e-2)
    for ws, bs, ci, co in O.cnn_layer_slices(ndim):
        for sl in (ws, bs):
            a, b = g[sl].astype(np.float64), go[sl]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            assert rel <= 5e-2 and cos >= 0.998, (sl, rel, cos)


@pytest.mark.parametrize("ndim,shape,margin", [(2, (2, 5, 32, 32), 2), (3, (1, 5, 8, 8, 8), 1)])
def test_operator_loss_gradient_matches_oracle(ndim, shape, margin):
    """Operator-weighted loss (kappa of the 2048^2 Gray-Scott species): the loss of the GPU's
    own outputs matches the oracle's loss of those outputs to float32 rounding; the parameter
    gradient matches the oracle's within the bf16 tolerance of the MSE test."""
    rng = np.random.default_rng(60 + ndim)
    p = rand_params(ndim, rng)
    x = bf16_round(rng.uniform(0, 1, size=shape)).astype(np.float64)
    tgt = (0.05 * rng.normal(size=(shape[0], 2) + shape[2:])).astype(np.float32)
    kappa = (0.0745, 0.149)
    net = amrvac.CnnNet(ndim=ndim)
    net.set_params(p)
    net.set_loss("operator", kappa)
    xt, tt = torch.from_numpy(x.astype(np.float32)).cuda(), torch.from_numpy(tgt).cuda()
    loss, g = net.gradient(xt, tt, margin=margin)
    out = net.forward(xt).double().cpu().numpy()
    lo_own, _ = O.cnn_output_loss(out, tgt, margin=margin, ndim=ndim, loss="operator", kappa=kappa)
    assert loss == pytest.approx(lo_own, rel=1e-4)
    lo, go = O.cnn_loss_grad(p, x, tgt, margin=margin, ndim=ndim, loss="operator", kappa=kappa)
    assert loss == pytest.approx(lo, rel=3e-2)
    for ws, bs, ci, co in O.cnn_layer_slices(ndim):
        for sl in (ws, bs):
            a, b = g[sl].astype(np.float64), go[sl]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            assert rel <= 5e-2 and cos >= 0.998, (sl, rel, cos)
    # margin 0 has no neighbours at the edge; the loss kinds are validated
    with pytest.raises(amrvac.AmrError):
        net.gradient(xt, tt, margin=0)
    with pytest.raises(amrvac.AmrError):
        net.set_loss("operator", (-1.0, 0.0))
    net.set_loss("mse")
    l_mse, _ = net.gradient(xt, tt, margin=margin)
    assert l_mse == pytest.approx(O.cnn_output_loss(out, tgt, margin=margin, ndim=ndim)[0], rel=1e-4)


def test_training_reduces_loss_and_adam_moves_by_lr():
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(0, 1, size=(8, 5, 32, 32)).astype(np.float32)).cuda()
    tgt = 0.1 * torch.sin(3 * x[:, :2]) + 0.05 * torch.roll(x[:, 1:3], 1, dims=2)
    net = amrvac.CnnNet(ndim=2, seed=7)
    p0 = net.get_params()
    l0 = net.train_step(x, tgt, lr=1e-3)
    p1 = net.get_params()
    # first Adam step: every parameter with a non-negligible gradient moves by ~lr
    moved = np.abs(p1 - p0)
    assert np.median(moved) == pytest.approx(1e-3, rel=0.05)
    for _ in range(200):
        loss = net.train_step(x, tgt, lr=2e-3, want_loss=False)
    lN = net.train_step(x, tgt, lr=2e-3)
    assert lN < 0.2 * l0, (l0, lN)


def test_shape_validation():
    net = amrvac.CnnNet(ndim=2)
    x = torch.zeros((1, 5, 20, 32), device="cuda")
    with pytest.raises(amrvac.AmrError):
        net.forward(x)


@pytest.mark.parametrize("shape", [(2, 5, 48, 64), (1, 5, 256, 256)])
def test_fused_inference_matches_oracle_and_layer_path(shape):
    """cnn_infer on 2D images whose sides tile by 32 x 16 runs the fused four-layer kernel with the
    tanh-form GELU (within 4.7e-4 of the erf form, plus the hardware tanh's error): against the FP64
    oracle network within the forward test's 3e-2 of the max norm, against the layer-by-layer bf16
    network (exact GELU) within 2e-2, periodic wrap included (the tiles' halos cross the image edge);
    repeated calls are identical."""
    rng = np.random.default_rng(31)
    p = rand_params(2, rng)
    x = bf16_round(rng.uniform(0, 1, size=shape)).astype(np.float64)
    net = amrvac.CnnNet(ndim=2)
    net.set_params(p)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    fused = net.infer(xd).cpu().numpy()
    layer = net.forward(xd).cpu().numpy()
    ref = O.cnn_forward(p, x, ndim=2)
    m = np.max(np.abs(ref))
    assert np.max(np.abs(fused - ref)) / m <= 3e-2
    assert np.max(np.abs(fused - layer)) / np.max(np.abs(layer)) <= 2e-2
    assert np.array_equal(net.infer(xd).cpu().numpy(), fused)
