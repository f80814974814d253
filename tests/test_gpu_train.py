"""Parity of the GPU training step (stda_backward: forward with a tape and
its adjoint, FP32) with the FP64 oracle's loss and gradient.

Tolerance: per parameter tensor, max |g_gpu - g_oracle| <= 2e-4 max |g_oracle|
(FP32 sums of up to ~10^5 terms per chunk, FP64 across chunks); loss to 1e-5
relative."""
import concurrent.futures as cf

import numpy as np
import pytest
import torch

import oracle as O
from paper_2307_09063_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GRAD_RTOL = 2e-4


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


def check_grad(got, ref):
    for name, (o, n) in I.param_offsets().items():
        g, r = got[o:o + n], ref[o:o + n]
        assert np.max(np.abs(g - r)) <= GRAD_RTOL * np.abs(r).max() + 1e-9, name


@pytest.mark.parametrize("B,H,W", [(2, 32, 32), (3, 24, 40), (1, 8, 8)])
def test_mse_backward_matches_oracle(stda, weights, B, H, W):
    rng = np.random.default_rng(B * 100 + H)
    x = rng.uniform(0, 1, (B, 3, H, W)).astype(np.float32)
    t = rng.uniform(0, 1, (B, H, W)).astype(np.float32)
    loss_ref, g_ref = O.loss_grad(*weights, x, t)
    ctx = stda.Context(H, W, B, "fp32", 0)
    loss, gp, _, z = ctx.backward(torch.from_numpy(x).cuda(), target=torch.from_numpy(t)[:, None].cuda().contiguous(),
                                  want_out=True)
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    check_grad(gp.cpu().numpy().astype(np.float64), g_ref)
    zr = O.forward_batch(*weights, x)
    assert np.max(np.abs(z[:, 0].cpu().numpy() - zr) / zr) <= 1e-4


def test_gout_backward_and_input_gradient(stda, weights):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (1, 3, 32, 48)).astype(np.float32)
    gout = rng.standard_normal((1, 32, 48)).astype(np.float32)
    g_ref, gin_ref = O.adjoint(*weights, x[0], gout[0])
    ctx = stda.Context(32, 48, 1, "fp32", 0)
    _, gp, gin, _ = ctx.backward(torch.from_numpy(x).cuda(), gout=torch.from_numpy(gout)[:, None].cuda().contiguous(),
                                 want_gin=True)
    check_grad(gp.cpu().numpy().astype(np.float64), g_ref)
    gi = gin[0].cpu().numpy()
    assert np.max(np.abs(gi - gin_ref)) <= GRAD_RTOL * np.abs(gin_ref).max()


def _gen(args):
    cid, w, g = args
    noisy, clean, _ = O.gen_window(0, cid, w, g)
    return noisy, clean


def test_training_batch_64_windows_256x128(stda, weights):
    """The 64-window training batch of 3 x 256 x 128 maps with their
    interference-free maps as targets, generated by the oracle."""
    w = I.WORKLOADS[3]
    g = w.gen
    with cf.ThreadPoolExecutor(16) as ex:
        wins = list(ex.map(_gen, [(w.cid, k, g) for k in range(w.batch)]))
    x = np.stack([a for a, _ in wins]).astype(np.float32)
    t = np.stack([b for _, b in wins]).astype(np.float32)
    loss_ref, g_ref = O.loss_grad(*weights, x, t)
    ctx = stda.Context(g.P, g.Q, w.batch, "fp32", 0)
    loss, gp, _, _ = ctx.backward(torch.from_numpy(x).cuda(), target=torch.from_numpy(t)[:, None].cuda().contiguous())
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    check_grad(gp.cpu().numpy().astype(np.float64), g_ref)


def test_bf16_context_backward_close_to_fp32(stda):
    rng = np.random.default_rng(8)
    x = torch.from_numpy(rng.uniform(0, 1, (2, 3, 32, 32)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0, 1, (2, 1, 32, 32)).astype(np.float32)).cuda()
    l32, g32, _, _ = stda.Context(32, 32, 2, "fp32", 0).backward(x.to(torch.bfloat16).float(), target=t)
    lbf, gbf, _, _ = stda.Context(32, 32, 2, "bf16", 0).backward(x.to(torch.bfloat16),
                                                                  target=t.to(torch.bfloat16))
    tb = t.to(torch.bfloat16).float()
    l32b, g32b, _, _ = stda.Context(32, 32, 2, "fp32", 0).backward(x.to(torch.bfloat16).float(), target=tb)
    assert abs(lbf.item() - l32b.item()) <= 1e-6 * l32b.item()
    assert torch.allclose(gbf, g32b, rtol=0, atol=1e-7 * g32b.abs().max().item() + 1e-9)


def test_autograd_training_reduces_loss(stda):
    """A few AdamW steps (lr 1e-3, weight decay 5e-4, Table of training
    settings) through the autograd function lower the MSE on a fixed batch."""
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.uniform(0, 1, (4, 3, 32, 32)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0.3, 0.7, (4, 1, 32, 32)).astype(np.float32)).cuda()
    ctx = stda.Context(32, 32, 4, "fp32", 0)
    theta = torch.from_numpy(ctx.get_params()).cuda().requires_grad_(True)
    opt = torch.optim.AdamW([theta], lr=1e-3, weight_decay=5e-4)
    losses = []
    for _ in range(8):
        z = stda.stda_apply(x, theta, ctx)
        loss = torch.mean((z - t) ** 2)
        opt.zero_grad()
        loss.backward()
        opt.step()
        ctx.set_params(theta.detach().cpu().numpy())
        losses.append(loss.item())
    assert losses[-1] < 0.9 * losses[0], losses
