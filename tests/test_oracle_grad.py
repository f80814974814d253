"""Pins of the oracle's gradient (adjoint of the forward pass, FP64):
PyTorch float64 autograd of an independent PyTorch composition of the
network, and central finite differences of the oracle's own loss."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2307_09063_gb300 import inputs as I
from torch_ref import torch_forward


def test_adjoint_equals_torch_autograd(weights):
    params, buffers = weights
    rng = np.random.default_rng(21)
    x = rng.uniform(0, 1, (3, 16, 24)).astype(np.float32)
    gout = rng.standard_normal((16, 24))
    gp, gx = O.adjoint(params, buffers, x, gout)
    xt = torch.tensor(x.astype(np.float64), requires_grad=True)
    z, _, P = torch_forward(params, buffers, xt, requires_grad=True)
    (z * torch.tensor(gout)).sum().backward()
    ref = np.concatenate([P[name].grad.numpy() for name, _, _, _ in I.param_table()])
    assert ref.shape == gp.shape
    scale = np.abs(ref).max()
    assert np.max(np.abs(gp - ref)) <= 1e-11 * scale
    assert np.max(np.abs(gx - xt.grad.numpy())) <= 1e-11 * np.abs(xt.grad.numpy()).max()
    # every parameter tensor receives a gradient
    for name, (o, n) in I.param_offsets().items():
        assert np.any(gp[o:o + n] != 0.0), name


def test_mse_gradient_equals_central_differences(weights):
    """3 x 32 x 32 window: dL/dtheta_i against (L(theta + h) - L(theta - h)) / 2h
    for two parameters of every tensor. The loss is piecewise smooth (ReLU);
    h = 2^-16 keeps the perturbation from crossing activation kinks, and the
    FP64 loss keeps the difference quotient's rounding near 1e-12."""
    params, buffers = weights
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (1, 3, 32, 32)).astype(np.float32)
    t = rng.uniform(0, 1, (1, 32, 32)).astype(np.float32)
    loss, g = O.loss_grad(params, buffers, x, t)
    r2 = np.random.default_rng(7)
    h = np.float32(2.0 ** -16)
    for name, (o, n) in I.param_offsets().items():
        for _ in range(2):
            i = o + int(r2.integers(n))
            pp, pm = params.copy(), params.copy()
            pp[i] += h
            pm[i] -= h
            lp, _ = O.loss_grad(pp, buffers, x, t)
            lm, _ = O.loss_grad(pm, buffers, x, t)
            fd = (lp - lm) / (float(pp[i]) - float(pm[i]))
            assert abs(fd - g[i]) <= 1e-7 + 1e-4 * abs(g[i]), (name, i, fd, g[i])


def test_loss_grad_batch_is_sum_of_windows(weights):
    params, buffers = weights
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 1, (3, 3, 16, 16)).astype(np.float32)
    t = rng.uniform(0, 1, (3, 16, 16)).astype(np.float32)
    loss, g = O.loss_grad(params, buffers, x, t, nthreads=2)
    parts = [O.loss_grad(params, buffers, x[b:b + 1], t[b:b + 1]) for b in range(3)]
    assert abs(loss - sum(p[0] for p in parts) / 3) <= 1e-15
    assert np.max(np.abs(g - sum(p[1] for p in parts) / 3)) <= 1e-15 * np.abs(g).max() * 10
