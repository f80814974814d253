"""CPU checks of the reduced-precision tolerance helper (tests/precision.py)."""
import numpy as np
import torch
import torch.nn.functional as F

import oracle as O
import precision as PR
from paper_2307_09063_gb300 import inputs as I


def test_logit_terms_constant_map_and_conv(weights):
    params, _ = weights
    o, s = I.param_offsets()["out.w"]
    w = params[o:o + s].astype(np.float64).reshape(1, 8, 3, 3)
    t = PR.logit_terms(params, np.full((8, 6, 5), 2.0))
    assert np.allclose(t[1:-1, 1:-1], 2.0 * np.abs(w).sum())
    assert np.allclose(t[0, 0], 2.0 * np.abs(w[0, :, 1:, 1:]).sum())  # corner: zero padding
    d3 = np.random.default_rng(0).normal(size=(8, 7, 9))
    ref = F.conv2d(torch.tensor(np.abs(d3))[None], torch.tensor(np.abs(w)), padding=1)[0, 0].numpy()
    assert np.allclose(PR.logit_terms(params, d3), ref)


def test_logit_terms_bound_the_oracle_logit(weights):
    """|logit - bias| <= T(p) at every pixel (triangle inequality), with the
    logit recovered from the oracle output."""
    params, buffers = weights
    x = np.random.default_rng(1).uniform(0, 1, (3, 32, 16)).astype(np.float32)
    z, blocks = O.forward(params, buffers, x, return_blocks=True)
    o, _ = I.param_offsets()["out.b"]
    logit = np.log(z / (1.0 - z)) - float(params[o])
    assert np.all(np.abs(logit) <= PR.logit_terms(params, blocks[5]) * (1 + 1e-9))


def test_bound_is_the_stated_tolerance_for_the_parity_weights(weights):
    """Seed 0 (the parity weights) on a 64 x 64 window: the bound is 2e-2."""
    params, buffers = weights
    w = I.WORKLOADS[1]
    noisy, _, _ = O.gen_window(0, w.cid, 0, w.gen, with_clean=False)
    z, blocks = O.forward(params, buffers, noisy.astype(np.float32), return_blocks=True)
    k = PR.kappa(params, blocks[5], z)
    assert 0 < k and PR.bound(k) == PR.ATOL
    assert PR.bound(1e3) == PR.GROWTH * PR.U_BF16 * 1e3


def test_sinr_cells_reproduce_the_oracle_sinr(weights):
    params, buffers = weights
    w = I.WORKLOADS[1]
    noisy, _, bins = O.gen_window(0, w.cid, 0, w.gen, with_clean=False)
    z, blocks = O.forward(params, buffers, noisy.astype(np.float32), return_blocks=True)
    o, n = PR.sinr_cells(bins, *z.shape)
    assert abs(10 * np.log10((z[o] ** 2).mean() / (z[n] ** 2).mean()) - O.sinr_db(z, bins)) < 1e-9
    assert PR.sinr_bound(params, blocks[5], z, bins) > 0


def test_fp32_bound_is_the_stated_tolerance_for_the_parity_weights(weights):
    params, buffers = weights
    x = np.random.default_rng(2).uniform(0, 1, (3, 64, 64)).astype(np.float32)
    z, blocks = O.forward(params, buffers, x, return_blocks=True)
    assert np.all(PR.fp32_rel_bound(params, blocks[5], z) == PR.RTOL_FP32)
