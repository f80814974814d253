"""Parity of the GPU range-Doppler generator with the FP64 oracle: target
counts and peak bins bit-exact, maps within FP32 / BF16 rounding."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2307_09063_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


def _check(stda, g, cid, windows, dtype, atol):
    w0, nb = min(windows), max(windows) - min(windows) + 1
    noisy, clean, bins, ntgt = stda.generate(g, 0, cid, w0, nb, dtype=dtype)
    torch.cuda.synchronize()
    for w in windows:
        on, oc, ob = O.gen_window(0, cid, w, g)
        k = w - w0
        assert int(ntgt[k]) == len(ob)
        assert np.array_equal(bins[k, :len(ob)].cpu().numpy(), ob)
        assert np.all(bins[k, len(ob):].cpu().numpy() == -1)
        assert np.max(np.abs(noisy[k].float().cpu().numpy() - on)) <= atol
        assert np.max(np.abs(clean[k, 0].float().cpu().numpy() - oc)) <= atol


def test_generator_64x64_fp32(stda):
    w = I.WORKLOADS[1]
    _check(stda, w.gen, w.cid, [0, 1, 2, 3], torch.float32, 2e-6)


def test_generator_256x128_fp32_sampled(stda):
    w = I.WORKLOADS[2]
    _check(stda, w.gen, w.cid, [0, 5, 37], torch.float32, 2e-6)


def test_generator_256x128_bf16_one_ulp(stda):
    w = I.WORKLOADS[2]
    _check(stda, w.gen, w.cid, [74, 75], torch.bfloat16, 2.0 ** -8 + 1e-9)


def test_generator_512x256_bins(stda):
    w = I.WORKLOADS[4]
    _check(stda, w.gen, w.cid, [111], torch.float32, 2e-6)


def test_generator_bins_many_windows_bit_exact(stda):
    """Counts and peak bins over 64 windows of the 256 x 128 workload."""
    w = I.WORKLOADS[2]
    _, _, bins, ntgt = stda.generate(w.gen, 0, w.cid, 0, 64, with_clean=False)
    bins, ntgt = bins.cpu().numpy(), ntgt.cpu().numpy()
    for k in range(64):
        sc = O.draw_scene(0, w.cid, k, w.gen)
        ob = O.peak_bins(w.gen, sc)
        assert ntgt[k] == sc.n_tgt
        assert np.array_equal(bins[k, :len(ob)], ob)


def test_generator_rejects_bad_config(stda):
    g = I.GenConfig(64, 16, 48, 64, 1, 1, 1, 1, 0, 0)  # P not a power of two
    with pytest.raises(stda.StdaError):
        stda.generate(g, 0, 0, 0, 1)
