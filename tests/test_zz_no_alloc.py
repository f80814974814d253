"""The no-allocation entry point, stda_forward_static, for callers that
cannot allocate device memory (real-time pipelines that forbid allocation
after start-up, plug-ins whose host owns all device buffers). It must give
the same denoised maps as the context-based stda_forward, call after call,
although every call reuses one static device array.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest
import torch

from paper_2307_09063_gb300 import inputs as I

pytestmark = pytest.mark.gpu
FP32_RTOL = 1e-4


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


def test_static_forward_matches_context_forward_two_calls_in_a_row(stda):
    params, buffers = I.init_params(0)
    d_params = torch.from_numpy(params).cuda()
    d_buffers = torch.from_numpy(buffers).cuda()
    ctx = stda.Context(64, 64, 4, "fp32", 0)
    rng = np.random.default_rng(2024)
    for B, H, W in [(2, 64, 64), (4, 32, 48)]:
        x = torch.from_numpy(rng.uniform(0, 1, (B, 3, H, W)).astype(np.float32)).cuda()
        ref = ctx.forward(x)
        got = stda.forward_static(d_params, d_buffers, x)
        torch.cuda.synchronize()
        rel = ((got - ref).abs() / ref.abs()).max().item()
        assert rel <= FP32_RTOL, rel


def test_static_forward_rejects_sizes_beyond_its_array(stda):
    d = torch.zeros(1, device="cuda")
    lib = stda.lib()
    x = torch.zeros((1, 3, 512, 256), device="cuda")
    y = torch.zeros((1, 1, 512, 256), device="cuda")
    st = lib.stda_forward_static(stda._ptr(d), stda._ptr(d), stda._ptr(x), stda._ptr(y), 1, 512, 256,
                                 stda._stream())
    assert st == stda.ERR_SHAPE
