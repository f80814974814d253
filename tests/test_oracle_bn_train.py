"""Pins of the oracle's training step with BatchNorm in training mode (batch
statistics over every window and pixel of a channel): against PyTorch
float64 autograd through F.batch_norm(training=True), against the
per-window oracle when the running statistics are used (mode 0), and the
defining property of batch normalisation."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2307_09063_gb300 import inputs as I
from torch_ref import torch_forward


def batch(seed, B, H, W):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (B, 3, H, W)).astype(np.float32)
    t = rng.uniform(0.2, 0.8, (B, H, W)).astype(np.float32)
    return x, t


def test_running_statistics_mode_equals_per_window_oracle(weights):
    x, t = batch(0, 3, 16, 24)
    loss0, g0, st = O.loss_grad_bn(*weights, x, t, mode=0)
    loss, g = O.loss_grad(*weights, x, t)
    assert abs(loss0 - loss) <= 1e-13 * loss
    assert np.max(np.abs(g0 - g)) <= 1e-12 * np.abs(g).max()
    np.testing.assert_array_equal(st, weights[1].astype(np.float64))  # the running statistics


@pytest.mark.parametrize("B,H,W", [(2, 16, 16), (3, 8, 24)])
def test_batch_statistics_match_torch_autograd(weights, B, H, W):
    params, bufs = weights
    x, t = batch(B * 7 + H, B, H, W)
    loss, g, st = O.loss_grad_bn(params, bufs, x, t, mode=1)
    stats = []
    z, _, P = torch_forward(params, bufs, torch.tensor(x.astype(np.float64)), requires_grad=True,
                            bn_training=True, stats=stats)
    L = ((z - torch.tensor(t.astype(np.float64))) ** 2).mean()
    L.backward()
    assert abs(loss - L.item()) <= 1e-12 * L.item()
    ref = np.concatenate([P[name].grad.numpy().ravel() for name, _, _, _ in I.param_table()])
    for name, (o, n) in I.param_offsets().items():
        assert np.max(np.abs(g[o:o + n] - ref[o:o + n])) <= 1e-9 * np.abs(ref[o:o + n]).max() + 1e-15, name
    # BN statistics in the buffer layout: (mean, biased var) per BN in bn_table order
    ref_st = np.concatenate([np.concatenate([m.detach().numpy(), v.detach().numpy()]) for m, v in stats])
    assert np.max(np.abs(st - ref_st)) <= 1e-12 * np.abs(ref_st).max()


def test_batch_statistics_differ_from_running_and_depend_on_the_batch(weights):
    x, t = batch(3, 4, 16, 16)
    l1, g1, s1 = O.loss_grad_bn(*weights, x, t, mode=1)
    l0, g0, _ = O.loss_grad_bn(*weights, x, t, mode=0)
    assert abs(l1 - l0) > 1e-6 * l0
    # the loss of window 0 changes when the other windows change (BN couples them)
    x2 = x.copy()
    x2[1:] = np.random.default_rng(9).uniform(0, 1, x2[1:].shape)
    _, _, s2 = O.loss_grad_bn(*weights, x2, t, mode=1)
    assert np.max(np.abs(s2 - s1)) > 1e-6
