"""Structural re-parameterisation export (host only): the folded inference
network written by stda_reparam_export, run with PyTorch float64 library
convolutions, reproduces the multi-branch network of the FP64 oracle (BN
folding is an identity, Sec. IV-B; the only difference is the single float32
rounding of each exported weight)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from paper_2307_09063_gb300 import inputs as I
from paper_2307_09063_gb300 import stda as S


def folded_forward(net, x):  # x [frames][H][W]
    """The inference network of the export, from PyTorch float64 operators."""
    t = {k: torch.tensor(v.astype(np.float64)) for k, v in net.items()}
    a = torch.tensor(np.asarray(x, np.float64))[None]
    a = F.relu(F.conv2d(a, t["stem.weight"], t["stem.bias"], padding=1))
    skips = []
    for b in range(6):
        p, ci = f"blk{b}", I.CIN[b]
        x1 = F.relu(F.conv2d(a, t[p + ".dw.weight"], t[p + ".dw.bias"], padding=1, groups=ci))
        conv = F.conv2d if I.ENC[b] else F.conv_transpose2d
        main = conv(x1, t[p + ".main.weight"], t[p + ".main.bias"], stride=2, padding=1)
        res = conv(a, t[p + ".res.weight"], t[p + ".res.bias"], stride=2, padding=1)
        y = F.relu(main) + res
        g = y.mean(dim=(2, 3))
        y = y * torch.sigmoid(F.conv1d(g[:, None, :], t[p + ".eca.weight"], padding=1))[:, 0, :, None, None]
        if b == 3:
            y = y + skips[1]
        if b == 4:
            y = y + skips[0]
        if b < 2:
            skips.append(y)
        a = y
    return torch.sigmoid(F.conv2d(a, t["out.weight"], t["out.bias"], padding=1))[0, 0].numpy()


def test_count_and_shapes():
    n = sum(int(np.prod(s)) for _, s in S.reparam_shapes())
    assert n == S.lib().stda_reparam_count(3) == 136731
    assert S.lib().stda_reparam_count(4) == n + 72 and S.lib().stda_reparam_count(5) == 0
    params, bufs = I.init_params(0)
    net = S.reparam_export(params, bufs)
    assert all(np.all(np.isfinite(v)) for v in net.values())


@pytest.mark.parametrize("seed,H,W", [(0, 32, 24), (3, 16, 40)])
def test_folded_network_matches_multibranch_oracle(seed, H, W):
    params, bufs = I.init_params(seed)
    net = S.reparam_export(params, bufs)
    x = np.random.default_rng(seed).uniform(0, 1, (3, H, W))
    z = folded_forward(net, x)
    zr = O.forward(params, bufs, x)
    assert np.max(np.abs(z - zr)) <= 2e-6


def test_identity_bn_exposes_the_raw_branches():
    """With every BN the identity (gamma 1, beta 0, mean 0, var 1 - eps) the
    export must be the raw weights: stage-1 kernel = w3 (flipped in both axes
    for the decoder's transposed conv) with w1 + 1 added at the centre, main
    and residual convs unchanged, zero biases except the residual's."""
    params, bufs = I.init_params(1)
    off = I.param_offsets()
    for name, (o, n) in off.items():
        if name.endswith(".gamma"):
            params[o:o + n] = 1.0
        if name.endswith(".beta"):
            params[o:o + n] = 0.0
    k = 0
    for _, c in I.bn_table():
        bufs[k:k + c] = 0.0
        bufs[k + c:k + 2 * c] = np.float32(1.0 - 1e-5)
        k += 2 * c
    net = S.reparam_export(params, bufs)
    g = lambda n: params[off[n][0]:off[n][0] + off[n][1]]
    np.testing.assert_allclose(net["stem.weight"].ravel(), g("stem.w"), rtol=1e-6)
    for b in range(6):
        p, ci = f"blk{b}", I.CIN[b]
        w3 = g(p + ".w3").reshape(ci, 3, 3).astype(np.float64)
        if not I.ENC[b]:
            w3 = w3[:, ::-1, ::-1]
        ref = w3.copy()
        ref[:, 1, 1] += g(p + ".w1") + 1.0
        np.testing.assert_allclose(net[p + ".dw.weight"][:, 0], ref, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(net[p + ".main.weight"].ravel(), g(p + ".w2"), rtol=1e-6)
        np.testing.assert_array_equal(net[p + ".res.weight"].ravel(), g(p + ".rw"))
        np.testing.assert_array_equal(net[p + ".res.bias"], g(p + ".rb"))
        assert np.abs(net[p + ".main.bias"]).max() < 1e-6 and np.abs(net[p + ".dw.bias"]).max() < 1e-6


def test_bad_arguments():
    params, bufs = I.init_params(0)
    out = np.empty(10, np.float32)
    assert S.lib().stda_reparam_export(params.ctypes.data, bufs.ctypes.data, 3, out.ctypes.data, 10) == S.ERR_INVALID_ARG
    n = S.lib().stda_reparam_count(3)
    big = np.empty(n, np.float32)
    assert S.lib().stda_reparam_export(params.ctypes.data, bufs.ctypes.data, 0, big.ctypes.data, n) == S.ERR_INVALID_ARG


@pytest.mark.parametrize("T", [2, 4])
def test_folded_fusion_variant_matches_oracle(T):
    params, bufs = I.init_params(4, frames=T)
    net = S.reparam_export(params, bufs, frames=T)
    assert net["stem.weight"].shape == (8, T, 3, 3)
    x = np.random.default_rng(T).uniform(0, 1, (T, 16, 24))
    assert np.max(np.abs(folded_forward(net, x) - O.forward_frames(params, bufs, x))) <= 2e-6


def test_library_init_params_frames_bit_exact():
    for T in (2, 3, 4):
        p, b = S.init_params(9, frames=T)
        pr, br = I.init_params(9, frames=T)
        assert np.array_equal(p, pr) and np.array_equal(b, br)
