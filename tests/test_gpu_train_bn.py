"""Training step with BatchNorm in training mode (stda_backward_bn, batch
statistics over all windows and pixels) against the FP64 oracle's batch
training step: loss to 1e-5 relative, every parameter tensor's gradient to
2e-4 of its largest magnitude (as for the running-statistics step), the BN
statistics to 1e-5 of their largest magnitude."""
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


def data(seed, B, H, W):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0, 1, (B, 3, H, W)).astype(np.float32), rng.uniform(0.2, 0.8, (B, H, W)).astype(np.float32))


@pytest.mark.parametrize("B,H,W", [(3, 24, 40), (5, 32, 32), (2, 64, 48)])
def test_batch_bn_step_matches_oracle(stda, weights, B, H, W):
    x, t = data(B + H, B, H, W)
    loss_ref, g_ref, st_ref = O.loss_grad_bn(*weights, x, t, mode=1)
    ctx = stda.Context(H, W, B, "fp32", 0)
    loss, gp, st = ctx.backward_bn(torch.from_numpy(x).cuda(), target=torch.from_numpy(t)[:, None].cuda().contiguous())
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    g = gp.cpu().numpy().astype(np.float64)
    for name, (o, n) in I.param_offsets().items():
        assert np.max(np.abs(g[o:o + n] - g_ref[o:o + n])) <= GRAD_RTOL * np.abs(g_ref[o:o + n]).max() + 1e-9, name
    s = st.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(s - st_ref)) <= 1e-5 * np.abs(st_ref).max()


def test_running_mode_equals_stda_backward(stda):
    x, t = data(1, 3, 32, 32)
    ctx = stda.Context(32, 32, 3, "fp32", 0)
    xc, tc = torch.from_numpy(x).cuda(), torch.from_numpy(t)[:, None].cuda().contiguous()
    l0, g0, _, _ = ctx.backward(xc, target=tc)
    l1, g1, st = ctx.backward_bn(xc, target=tc, mode="running")
    assert torch.equal(g0, g1) and l0.item() == l1.item()
    assert np.array_equal(st.cpu().numpy(), ctx.get_buffers())


def test_batch_statistics_normalise_the_stem(stda, weights):
    """The stem BN's batch mean / variance are those of the stem conv output
    over the whole batch (cross-checked in FP64 with the conv run by torch)."""
    import torch.nn.functional as F

    x, t = data(2, 4, 16, 24)
    ctx = stda.Context(16, 24, 4, "fp32", 0)
    _, _, st = ctx.backward_bn(torch.from_numpy(x).cuda(), target=torch.from_numpy(t)[:, None].cuda().contiguous())
    o, n = I.param_offsets()["stem.w"]
    su = F.conv2d(torch.tensor(x.astype(np.float64)), torch.tensor(weights[0][o:o + n].astype(np.float64)).view(8, 3, 3, 3),
                  padding=1)
    s = st.cpu().numpy()
    np.testing.assert_allclose(s[:8], su.mean(dim=(0, 2, 3)).numpy(), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(s[8:16], su.var(dim=(0, 2, 3), unbiased=False).numpy(), rtol=1e-5)
