"""Training and evaluation of the learned multigrid initial guess.

Orchestration only: the solver steps, the crop extraction, the network's
forward/backward passes and the Adam updates all run in the CUDA library.

Recipe (the project's own reading; the paper has no learned component):
* training data: Gray-Scott IMEX runs of the plain solver (previous-step guess)
  on training seeds, crops of side `crop` at seeded random positions after every
  step, inputs (u_n, v_n, u*_prev, v*_prev, dt), or (u_n, v_n, rho_u, rho_v, dt)
  with rho the normalised residual of the previous-step guess (inputs="residual":
  the increment is then the local inverse of the normalised operator applied to
  rho), target (w* - w_n) / scale (the
  increment over the previous-step guess; a network that outputs zero gives
  back that guess), where scale is the RMS of w* - w_n over the first
  collected step;
* loss: masked MSE (margin 4 = the network's receptive radius, so that the
  periodic padding inside a crop never reaches a counted pixel), or the
  operator-weighted loss: the mean square of the guess's residual under the
  diagonal-normalised Helmholtz operator of Eq. (diff-helmholtz), kappa =
  lambda h^2 / (2 ndim) per species (`operator_kappa`), margin 5 (the
  operator's stencil adds one cell to the receptive radius);
* Adam, lr 1e-3 over the first half of the steps, then a cosine decay to 5e-5
  (`lr_at`), batches of `batch` crops drawn uniformly with replacement;
* evaluation on disjoint seeds: V-cycles per step and wall time per step with
  the learned guess against the previous-step guess, both to the same rtol.
"""
from __future__ import annotations

import time

import numpy as np

from . import amrvac, inputs

GS = dict(Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=0.5)


def domain_for(n, ref_n=2048, ref_L=2.5):
    """Domain side giving the same stiffness D dt / h^2 as the reference grid."""
    return ref_L * n / ref_n


def operator_kappa(n, L, ndim=2, dt=GS["dt"], Du=GS["Du"], Dv=GS["Dv"]):
    """kappa_c = lambda_c h^2 / (2 ndim), lambda_c = 2 / (dt D_c) (IMEX, Eq. (imex)), h = L / n."""
    h = L / n
    return tuple(2.0 / (dt * D) * h * h / (2 * ndim) for D in (Du, Dv))


MARGIN = {"mse": 4, "operator": 5}


def start_state(sizes, L, seeds, ndim=2):
    us, vs = [], []
    for n, sd in zip(sizes, seeds):
        u, v = inputs.gray_scott_patches(n, ndim=ndim, L=L, seed=sd)
        us.append(u.ravel())
        vs.append(v.ravel())
    return np.concatenate(us), np.concatenate(vs)


def generate(torch, sizes, seeds, L, steps, crops_per_step, crop=64, warm=0, scale=None, seed=0, stream=None,
             ndim=2, inputs="prev"):
    """Returns (inputs [M][5][c]^ndim, targets [M][2][c]^ndim, scale) as CUDA float tensors;
    `inputs` selects channels 2, 3 (RdSolver.set_guess_inputs)."""
    rd = amrvac.RdSolver(ndim, sizes, L, precision="fp32", stream=stream, **GS)
    rd.set_guess_inputs(inputs)
    rd.set_state(*start_state(sizes, L, seeds, ndim))
    box = (crop,) * ndim
    if warm:
        rd.step(warm)
    rng = np.random.default_rng(seed)
    X, Y = [], []
    for s in range(steps):
        rd.step(1)
        inst = rng.integers(0, len(sizes), crops_per_step)
        corners = np.zeros((crops_per_step, 3), dtype=np.int32)
        for k in range(crops_per_step):
            n = sizes[inst[k]]
            corners[k, :ndim] = rng.integers(0, n, ndim)
        if scale is None:  # RMS of w* - w_n over the first step's crops
            xi = torch.empty((crops_per_step, 5) + box, device="cuda")
            yi = torch.empty((crops_per_step, 2) + box, device="cuda")
            rd.extract_crops(inst, corners, crop, 1.0, xi, yi)
            scale = float(torch.sqrt(torch.mean(yi.double() ** 2)).item())
        xi = torch.empty((crops_per_step, 5) + box, device="cuda")
        yi = torch.empty((crops_per_step, 2) + box, device="cuda")
        torch.cuda.synchronize()  # the buffers are free on every stream before the solver writes them
        rd.extract_crops(inst, corners, crop, scale, xi, yi)
        X.append(xi)
        Y.append(yi)
    rd.close()
    return torch.cat(X), torch.cat(Y), scale


def lr_at(it, iters, lr, final_frac=0.05):
    """Learning rate of Adam step `it` (0-based): constant over the first half, then a cosine
    decay to final_frac * lr at the last step, so that training ends on a settled iterate
    rather than on one of the fluctuating constant-rate iterates."""
    half = iters // 2
    if it < half or iters - half <= 1:
        return lr
    f = (it - half) / (iters - half - 1)
    return lr * (final_frac + (1.0 - final_frac) * 0.5 * (1.0 + np.cos(np.pi * f)))


def train(torch, net, X, Y, iters, batch=32, lr=1e-3, margin=4, seed=1):
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    for it in range(iters):
        # the network's kernels run on its own stream: the device-wide synchronisation orders the
        # previous step's reads of the last batch before torch may reuse that memory, and the
        # gather of this batch (on torch's stream) before the step reads it
        torch.cuda.synchronize()
        idx = torch.from_numpy(rng.integers(0, X.shape[0], batch)).cuda()
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        torch.cuda.synchronize()
        want = it == 0 or it == iters - 1 or (it + 1) % 100 == 0
        loss = net.train_step(xb, yb, lr=lr_at(it, iters, lr), margin=margin, want_loss=want)
        if want:
            losses.append((it + 1, loss))
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def dataset_loss(torch, net, X, Y, margin=4, chunk=16):
    """Masked MSE of the network over the whole data set (chunks in order, weighted by size)."""
    tot = 0.0
    torch.cuda.synchronize()  # X, Y complete before the network's stream reads them
    for i in range(0, X.shape[0], chunk):
        xb, yb = X[i:i + chunk].contiguous(), Y[i:i + chunk].contiguous()
        loss, _ = net.gradient(xb, yb, margin=margin)
        tot += loss * xb.shape[0]
    return tot / X.shape[0]


def evaluate(torch, sizes, seeds, L, steps, net=None, scale=1.0, warm=0, stream=None, ndim=2, inputs="prev"):
    """V-cycles per step (per species and instance) and wall time per step."""
    rd = amrvac.RdSolver(ndim, sizes, L, precision="fp32", stream=stream, **GS)
    rd.set_guess_inputs(inputs)
    rd.set_state(*start_state(sizes, L, seeds, ndim))
    if warm:
        rd.step(warm)
    if net is not None:
        rd.set_guess(net, scale)
    rd.step(1)  # the guess needs one previous solution; not timed
    torch.cuda.synchronize()
    cyc, init = [], []
    el = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        cyc.append(rd.step(1)[0])
        torch.cuda.synchronize()
        el += time.perf_counter() - t0
        init.append(rd.last_residuals()[0])
    u, v = rd.read_state()
    rd.close()
    return np.array(cyc), el / steps, (u, v), np.array(init)
