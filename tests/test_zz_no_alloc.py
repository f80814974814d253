"""The no-allocation entry point, stda_forward_static, for callers that
cannot allocate device memory (real-time pipelines that forbid allocation
after start-up, plug-ins whose host owns all device buffers). It must give
the same denoised maps as the context-based stda_forward, call after call,
although every call reuses one static device array, and match the FP64
oracle; it takes up to 65,536 map pixels per call.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2307_09063_gb300 import inputs as I

pytestmark = pytest.mark.gpu
FP32_RTOL = 1e-4


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


@pytest.fixture(scope="module")
def dev_weights():
    params, buffers = I.init_params(0)
    return params, buffers, torch.from_numpy(params).cuda(), torch.from_numpy(buffers).cuda()


def test_static_forward_matches_context_forward_two_calls_in_a_row(stda, dev_weights):
    _, _, d_params, d_buffers = dev_weights
    ctx = stda.Context(64, 64, 4, "fp32", 0)
    rng = np.random.default_rng(2024)
    for B, H, W in [(2, 64, 64), (4, 32, 48)]:
        x = torch.from_numpy(rng.uniform(0, 1, (B, 3, H, W)).astype(np.float32)).cuda()
        ref = ctx.forward(x)
        got = stda.forward_static(d_params, d_buffers, x)
        torch.cuda.synchronize()
        rel = ((got - ref).abs() / ref.abs()).max().item()
        assert rel <= FP32_RTOL, rel


@pytest.mark.parametrize("B,H,W", [(1, 256, 256), (16, 64, 64)])
def test_static_forward_at_its_pixel_limit_matches_oracle(stda, dev_weights, B, H, W):
    """Exactly 65,536 pixels per call: accepted, equal to stda_forward and,
    on one window, to the FP64 oracle."""
    params, buffers, d_params, d_buffers = dev_weights
    assert B * H * W == 65536
    rng = np.random.default_rng(B * H)
    x = rng.uniform(0, 1, (B, 3, H, W)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    got = stda.forward_static(d_params, d_buffers, xd)
    ref_ctx = stda.Context(H, W, B, "fp32", 0).forward(xd)
    torch.cuda.synchronize()
    assert ((got - ref_ctx).abs() / ref_ctx.abs()).max().item() <= FP32_RTOL
    k = B - 1
    ref = O.forward(params, buffers, x[k])
    assert np.max(np.abs(got[k, 0].cpu().numpy() - ref) / ref) <= FP32_RTOL


def test_static_forward_rejects_sizes_beyond_its_array(stda):
    d = torch.zeros(1, device="cuda")
    lib = stda.lib()
    for B, H, W in [(1, 512, 256), (1, 256, 264), (17, 64, 64)]:
        x = torch.zeros((B, 3, H, W), device="cuda")
        y = torch.zeros((B, 1, H, W), device="cuda")
        st = lib.stda_forward_static(stda._ptr(d), stda._ptr(d), stda._ptr(x), stda._ptr(y), B, H, W,
                                     stda._stream())
        assert st == stda.ERR_SHAPE


def test_static_forward_binding_refuses_short_parameters(stda, dev_weights):
    _, _, d_params, d_buffers = dev_weights
    x = torch.zeros((1, 3, 32, 32), device="cuda")
    with pytest.raises(stda.StdaError):
        stda.forward_static(d_params[:-1], d_buffers, x)
    with pytest.raises(stda.StdaError):
        stda.forward_static(d_params, d_buffers.double(), x)
