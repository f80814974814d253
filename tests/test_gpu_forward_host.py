"""stda_forward_host: the forward pass on host buffers (input copied in on
an internal stream into one of two staging buffers, forward on the caller's
stream, output stored straight into page-locked host memory or copied back
from a staging buffer) gives exactly the device-buffer forward's result, for
back-to-back calls that overlap, pinned or pageable memory."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_host_forward_equals_device_forward(stda, prec):
    B, H, W = 7, 64, 96
    ctx = stda.Context(H, W, B, prec, 0)
    g = torch.Generator(device="cpu").manual_seed(11)
    x = torch.rand((B, 3, H, W), generator=g).to(ctx.io_dtype)
    ref = ctx.forward(x.cuda()).cpu()
    y = ctx.forward_host(x.pin_memory())
    torch.cuda.synchronize()
    assert torch.equal(y, ref)


def test_host_forward_back_to_back_calls(stda):
    """Five calls queued without synchronising: each call's input copy may run
    during the previous call's kernels and the staging buffers alternate."""
    B, H, W = 5, 32, 64
    ctx = stda.Context(H, W, B, "bf16", 0)
    g = torch.Generator(device="cpu").manual_seed(12)
    xs = [torch.rand((B, 3, H, W), generator=g).to(torch.bfloat16) for _ in range(5)]
    refs = [ctx.forward(x.cuda()).cpu() for x in xs]
    torch.cuda.synchronize()
    outs = [ctx.forward_host(x.pin_memory()) for x in xs]
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    # one output buffer reused by consecutive calls ends with the last result
    o = torch.empty((B, 1, H, W), dtype=torch.bfloat16).pin_memory()
    for x in xs[:3]:
        ctx.forward_host(x.pin_memory(), o)
    torch.cuda.synchronize()
    assert torch.equal(o, refs[2])


def test_host_forward_direct_and_staged_outputs(stda):
    """A 16-byte aligned pinned output is written by the output kernel itself;
    a pinned output at an 8-byte offset and a pageable one go through the
    staging buffer and the copy back. All three equal the device forward,
    also when the calls alternate without synchronising."""
    B, H, W = 3, 64, 64
    ctx = stda.Context(H, W, B, "bf16", 0)
    g = torch.Generator(device="cpu").manual_seed(14)
    xs = [torch.rand((B, 3, H, W), generator=g).to(torch.bfloat16) for _ in range(3)]
    refs = [ctx.forward(x.cuda()).cpu() for x in xs]
    torch.cuda.synchronize()
    n = B * H * W
    aligned = torch.empty((B, 1, H, W), dtype=torch.bfloat16).pin_memory()
    buf = torch.empty(n + 8, dtype=torch.bfloat16).pin_memory()
    offset = buf[4:4 + n].view(B, 1, H, W)
    assert aligned.data_ptr() % 16 == 0 and offset.data_ptr() % 16 == 8
    pageable = torch.empty((B, 1, H, W), dtype=torch.bfloat16)
    outs = (aligned, offset, pageable)
    for _ in range(2):
        for x, o in zip(xs, outs):
            ctx.forward_host(x.pin_memory(), o)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)


def test_host_forward_pageable_and_smaller_batch(stda):
    B, H, W = 5, 32, 64
    ctx = stda.Context(H, W, B, "bf16", 0)
    g = torch.Generator(device="cpu").manual_seed(13)
    x = torch.rand((B, 3, H, W), generator=g).to(torch.bfloat16)
    ref = ctx.forward(x.cuda()).cpu()
    y = torch.empty((B, 1, H, W), dtype=torch.bfloat16)
    ctx.forward_host(x, y)  # pageable host memory
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    yd = ctx.forward_host(x[:2].contiguous().pin_memory())
    torch.cuda.synchronize()
    assert torch.equal(yd, ref[:2])


def test_host_forward_invalid_calls(stda):
    ctx = stda.Context(32, 32, 2, "fp32", 0)
    L, h, s = stda.lib(), ctx.h, stda._stream()
    x = torch.zeros((3, 3, 32, 32)).pin_memory()
    y = torch.zeros((3, 1, 32, 32)).pin_memory()
    p = stda._ptr
    assert L.stda_forward_host(h, p(x), p(y), 0, 32, 32, s) == stda.OK            # empty batch
    assert L.stda_forward_host(h, p(x), p(y), 3, 32, 32, s) == stda.ERR_SHAPE     # above max_batch
    assert L.stda_forward_host(h, p(x), p(y), 1, 12, 32, s) == stda.ERR_SHAPE     # not a multiple of 8
    assert L.stda_forward_host(h, None, p(y), 1, 32, 32, s) == stda.ERR_INVALID_ARG
    assert ctx.device_status() == stda.OK
