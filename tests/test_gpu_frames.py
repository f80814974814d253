"""Fusion variants with 2 or 4 stacked maps (Sec. IV-A, Eq. concat_operation
with T maps instead of three), through the C-ABI: the FP32 CUDA-core forward
against the FP64 oracle of the variant (max relative error 1e-4), and the
BF16 / FP8 tensor-core stems for 2, 3 and 4 maps against each other, bit for
bit, by zeroing the stem weights of the extra maps. (The BF16 bound of 2e-2
depends on how strongly a weight draw amplifies bf16 storage rounding, so
the tensor-core variants are checked exactly rather than against the oracle
with other weights.)"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2307_09063_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-4
LOWP_ATOL = 2e-2


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


def oracle_batch(params, bufs, x):
    return np.stack([O.forward_frames(params, bufs, xi) for xi in x])


@pytest.mark.parametrize("T,B,H,W", [(2, 2, 24, 40), (4, 2, 32, 48), (4, 1, 8, 8)])
def test_fp32_variant(stda, T, B, H, W):
    params, bufs = I.init_params(0, frames=T)
    x = np.random.default_rng(T * 10 + H).uniform(0, 1, (B, T, H, W)).astype(np.float32)
    ctx = stda.Context(H, W, B, "fp32", 0, frames=T)
    assert ctx.get_params().size == params.size
    got = ctx.forward(torch.from_numpy(x).cuda())[:, 0].cpu().numpy().astype(np.float64)
    ref = oracle_batch(params, bufs, x)
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= FP32_RTOL


def with_zero_stem_map(params_small, small, big, seed=0):
    """Parameters of the `big`-map network equal to the `small`-map network
    (same seed) plus zero stem weights for the extra maps."""
    pb, _ = I.init_params(seed, frames=big)
    ob, os_ = I.param_offsets(big), I.param_offsets(small)
    w = np.zeros((8, big, 9), np.float32)
    w[:, :small] = params_small[os_["stem.w"][0]:os_["stem.w"][0] + 72 * small].reshape(8, small, 9)
    pb = pb.copy()
    pb[ob["stem.w"][0]:ob["stem.w"][0] + 72 * big] = w.ravel()
    pb[ob["stem.bn.gamma"][0]:] = params_small[os_["stem.bn.gamma"][0]:]
    return pb


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("small,big", [(2, 3), (3, 4)])
def test_tensor_core_variant_reduces_bit_exactly(stda, prec, small, big):
    """The tensor-core stem for `big` maps with zero weights on the extra
    maps computes exactly what the `small`-map kernel computes (each extra
    product is an exact zero), whatever the extra maps hold."""
    B, H, W = 2, 64, 96
    ps, bufs = I.init_params(0, frames=small)
    pb = with_zero_stem_map(ps, small, big)
    x = torch.from_numpy(np.random.default_rng(big).uniform(0, 1, (B, big, H, W)).astype(np.float32))
    xb = x.to(torch.bfloat16).cuda()
    cb = stda.Context(H, W, B, prec, 0, frames=big)
    cb.set_params(pb)
    cs = stda.Context(H, W, B, prec, 0, frames=small)
    zb = cb.forward(xb)
    zs = cs.forward(xb[:, :small].contiguous())
    assert torch.equal(zb, zs)
    if prec == "bf16" and small == 3:
        # and the three-map network meets the BF16 bound against the oracle
        ref = np.stack([O.forward_frames(pb, bufs, xi) for xi in xb.float().cpu().numpy()])
        assert np.max(np.abs(zb[:, 0].float().cpu().numpy() - ref)) <= LOWP_ATOL


def test_three_maps_only_for_training_and_serving(stda):
    ctx = stda.Context(32, 32, 1, "fp32", 0, frames=4)
    x = torch.zeros(1, 4, 32, 32, device="cuda")
    with pytest.raises(stda.StdaError):
        ctx.backward(x, target=torch.zeros(1, 1, 32, 32, device="cuda"))
    frame = torch.zeros(32, 32, dtype=torch.bfloat16, device="cuda")
    bctx = stda.Context(32, 32, 1, "bf16", 0, frames=2)
    with pytest.raises(stda.StdaError):
        bctx.submit(0, frame, frame.clone())
