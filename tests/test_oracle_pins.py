"""Pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: each check is a value the
paper prints (tests/golden/paper_tables.json), a closed form, an identity, a
library routine computing the same definition (PyTorch / NumPy in float64),
or brute force on a tiny input.
"""
import json
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from paper_2307_09063_gb300 import inputs as I
from torch_ref import torch_reference

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
rng = np.random.default_rng(1234)


# --------------------------------------------------------------------- RNG
def test_splitmix64_reference_outputs():
    """SplitMix64 seeded with 0: the published first outputs."""
    L = O.lib()
    g = 0x9E3779B97F4A7C15
    want = [int(h, 16) for h in GOLDEN["splitmix64_seed0"]["outputs"]]
    got = [int(L.orc_splitmix64((k * g) % 2**64)) for k in range(3)]
    assert got == want
    # the shared input module implements the same published function
    got_np = [int(v) for v in I.splitmix64(np.array([(k * g) % 2**64 for k in range(3)], dtype=np.uint64))]
    assert got_np == want


def test_uniform_draws_in_range_and_spread():
    L = O.lib()
    u = np.array([L.orc_u01(L.orc_key(0, 1, 0, 11, 0, i)) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.003


# ------------------------------------------------------------- radar table
def test_victim_radar_table_identities():
    """Table 'victim parameters': 64 samples, 128 chirps reproduce the printed
    range/velocity resolution and maxima within the table's rounding."""
    t = GOLDEN["victim_radar"]
    rres, rmax, vmax, vres = O.radar_helpers(t["samples_per_chirp"], t["chirps_per_frame"])
    assert abs(rres - t["range_resolution_m"]) < 0.01
    assert abs(rmax - t["max_range_m"]) < 0.1
    assert abs(vmax - t["max_velocity_mps"]) < 0.05
    assert abs(vres - t["velocity_resolution_mps"]) < 0.005
    # slope over the ADC window = bandwidth / window = 30 MHz/us
    assert abs(t["sweep_bandwidth_MHz"] / t["adc_window_us"] - 30.0) < 1e-9


# ------------------------------------------------------------------- DFT
@pytest.mark.parametrize("N,M,P,Q", [(16, 8, 16, 8), (16, 8, 32, 16), (12, 6, 16, 8)])
def test_rd_transform_equals_numpy_fft(N, M, P, Q):
    """Eqs. 'column transform' / 'row transform' with a Hann window and zero
    padding equal numpy's FFT of the windowed, padded matrix, Doppler-shifted."""
    s = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    hn = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(N) / (N - 1))
    hm = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(M) / (M - 1))
    ref = np.fft.fftshift(np.fft.fft2(s * hn[:, None] * hm[None, :], s=(P, Q)), axes=1)
    got = O.rd_complex(s, P, Q)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_rd_transform_parseval():
    N, M, P, Q = 32, 16, 64, 32
    s = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    hn = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(N) / (N - 1))
    hm = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(M) / (M - 1))
    y = O.rd_complex(s, P, Q)
    assert abs(np.sum(np.abs(y) ** 2) - P * Q * np.sum(np.abs(s * np.outer(hn, hm)) ** 2)) < 1e-8 * np.sum(
        np.abs(y) ** 2)


def _single_target_cfg(N=64, M=16, P=64, Q=64):
    return I.GenConfig(N, M, P, Q, 1, 1, 0, 0, 10.0, 10.0)


def _scene_with(g, r, d, f_phase=0.3):
    sc = O.Scene()
    sc.n_tgt = 1
    sc.r[0], sc.d[0], sc.delta[0] = r, d, 0.0
    for f in range(3):
        sc.phase[f][0] = f_phase
    sc.sigma = 0.0
    return sc


@pytest.mark.parametrize("r,d", [(10.0, 3.0), (37.0, -5.0), (2.0, 7.0), (61.0, -7.0)])
def test_single_target_on_grid_peak_closed_form(r, d):
    """Sec. III-B: the range peak sits at the beat frequency, the Doppler peak
    at the Doppler frequency. On grid, the peak magnitude is A * sum(w_n) *
    sum(w_m) = (N-1)/2 * (M-1)/2 for a symmetric Hann window."""
    g = _single_target_cfg()
    sc = _scene_with(g, r, d)
    s = O.if_signal(0, 0, 0, g, sc, 0, with_int=False, with_noise=False)
    y = O.rd_complex(s, g.P, g.Q)
    p, q = np.unravel_index(np.argmax(np.abs(y)), y.shape)
    bins = O.peak_bins(g, sc)
    assert (p, q) == tuple(bins[0])
    assert p == round(r * g.P / g.N) % g.P
    assert q == (round(d * g.Q / g.M) + g.Q // 2) % g.Q
    peak = (g.N - 1) / 2 * (g.M - 1) / 2
    assert abs(np.abs(y[p, q]) - peak) < 1e-9 * peak


@pytest.mark.parametrize("seed", range(6))
def test_single_target_off_grid_argmax(seed):
    """Off-grid tones (fraction <= 0.4 bin from the nearest cell) still peak
    at the closed-form rounded bin."""
    g = _single_target_cfg(N=64, M=32, P=128, Q=64)
    rr = np.random.default_rng(seed)
    while True:
        r = rr.uniform(3, 60)
        d = rr.uniform(-14, 14)
        fr, fd = r * g.P / g.N, d * g.Q / g.M
        if abs(fr - np.floor(fr + 0.5)) <= 0.4 and abs(fd - np.floor(fd + 0.5)) <= 0.4:
            break
    sc = _scene_with(g, r, d)
    y = O.rd_complex(O.if_signal(0, 0, 0, g, sc, 0, False, False), g.P, g.Q)
    assert tuple(np.unravel_index(np.argmax(np.abs(y)), y.shape)) == tuple(O.peak_bins(g, sc)[0])


def test_target_drifts_between_frames():
    """A target at range r at frame t sits at r - f * delta at frame t - f."""
    g = _single_target_cfg(N=64, M=16, P=64, Q=64)
    sc = _scene_with(g, 30.0, 4.0)
    sc.delta[0] = 3.0
    for f in range(3):
        y = O.rd_complex(O.if_signal(0, 0, 0, g, sc, f, False, False), g.P, g.Q)
        p, _ = np.unravel_index(np.argmax(np.abs(y)), y.shape)
        assert p == 30 - 3 * f


def test_noise_variance_and_mean():
    """v(n, m) is complex white Gaussian with E|v|^2 = sigma^2, zero mean."""
    g = I.GenConfig(128, 64, 128, 64, 1, 1, 0, 0, 6.0, 6.0)
    sc = O.draw_scene(0, 9, 0, g)
    sc.n_tgt = 0
    v = O.if_signal(0, 9, 0, g, sc, 0, with_int=False, with_noise=True)
    n = v.size
    s2 = 10 ** (-6.0 / 10)
    assert abs(np.mean(np.abs(v) ** 2) / s2 - 1) < 5 / np.sqrt(n)
    assert abs(np.mean(v.real)) < 5 * np.sqrt(s2 / 2 / n)
    assert abs(np.mean(v.real ** 2) - np.mean(v.imag ** 2)) < 10 * s2 / np.sqrt(n)
    # Gaussian: fourth moment of a real component is 3 sigma_r^4
    k = np.mean(v.real ** 4) / np.mean(v.real ** 2) ** 2
    assert abs(k - 3.0) < 0.2


def test_interferer_equal_slope_is_a_zero_range_ghost():
    """Sec. III-D scenario (1): identical chirp slopes give a constant
    dechirped tone, i.e. a ghost at zero beat frequency (range bin 0)."""
    g = I.GenConfig(64, 16, 64, 16, 0, 0, 1, 1, 40.0, 40.0, 10.0, 10.0, 1.0, 1.0)
    sc = O.draw_scene(0, 7, 0, g)
    s = O.if_signal(0, 7, 0, g, sc, 0, with_int=True, with_noise=False)
    y = np.abs(O.rd_complex(s, g.P, g.Q)) ** 2
    rows = y.sum(axis=1)
    # the Hann main lobe holds a DC tone in range bins -1, 0, 1
    assert np.argmax(rows) == 0
    assert rows[0] + rows[1] + rows[-1] > 0.999 * y.sum()
    assert np.allclose(np.abs(s), 10 ** 0.5)


def test_interferer_burst_is_short_and_centred():
    """A slope ratio kappa gives an IF sweep of (kappa - 1) * 0.192 cycles per
    sample^2; only |f| <= fs/2 passes the IF filter, so each chirp holds one
    contiguous burst of about 1 / |gamma| samples around the crossing."""
    g = I.GenConfig(256, 8, 256, 8, 0, 0, 1, 1, 40.0, 40.0, 0.0, 0.0, 2.0, 2.0)
    sc = O.draw_scene(0, 8, 0, g)
    s = O.if_signal(0, 8, 0, g, sc, 0, with_int=True, with_noise=False)
    nz = np.nonzero(np.abs(s[:, 0]) > 0)[0]
    assert len(nz) in (5, 6) and np.all(np.diff(nz) == 1)
    assert abs(nz.mean() - sc.nx[0][0]) < 1.0
    assert np.allclose(np.abs(s[nz, 0]), 1.0)


def test_lognorm_range_and_order():
    y = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    z = O.lognorm(y)
    assert z.min() == 0.0 and z.max() == 1.0
    order = np.argsort(np.abs(y))
    assert np.all(np.diff(z[order]) >= 0)
    assert np.all(O.lognorm(np.ones(7, dtype=complex)) == 0.0)


def test_generated_window_bins_and_counts():
    w = I.WORKLOADS[2]
    counts = set()
    for win in range(12):
        sc = O.draw_scene(0, 2, win, w.gen)
        counts.add(sc.n_tgt)
        assert w.gen.tmin <= sc.n_tgt <= w.gen.tmax
        for f in range(3):
            assert w.gen.imin <= sc.n_int[f] <= w.gen.imax
        assert 0.0 <= sc.snr_db <= 20.0
    assert len(counts) >= 4
    noisy, clean, bins = O.gen_window(0, 1, 0, I.WORKLOADS[1].gen)
    assert noisy.shape == (3, 64, 64) and clean.shape == (64, 64) and bins.shape == (2, 2)
    for m in list(noisy) + [clean]:
        assert m.min() == 0.0 and m.max() == 1.0
    # targets stand out of the clean map: SINR at the closed-form cells is high
    assert O.sinr_db(clean, bins) > 3.0


# --------------------------------------------------------------- metrics
def test_sinr_known_map():
    """Eq. (SINR): peak cells of 10 over a floor of 1 give 20 dB."""
    z = np.ones((32, 16))
    bins = np.array([[5, 5], [20, 10], [20, 10]])
    z[5, 5] = z[20, 10] = 10.0
    assert abs(O.sinr_db(z, bins) - 20.0) < 1e-12
    # the guard box keeps near-peak cells out of the noise set
    z[6, 6] = 100.0
    assert abs(O.sinr_db(z, bins) - 20.0) < 1e-12


def test_evm_known_values():
    c = rng.uniform(0.5, 1.0, (16, 16))
    bins = np.array([[1, 2], [7, 9]])
    assert O.evm(c, c, bins) == 0.0
    assert abs(O.evm(c, 0.5 * c, bins) - 0.5) < 1e-15


# ------------------------------------------------------ network primitives
CONV_CASES = [  # Ci, Co, k, stride, pad, groups, H, W
    (3, 8, 3, 1, 1, 1, 7, 9), (8, 8, 1, 1, 0, 8, 6, 5), (8, 8, 3, 1, 1, 8, 6, 5),
    (8, 16, 3, 2, 1, 1, 8, 10), (6, 4, 3, 2, 1, 2, 7, 7), (8, 1, 3, 1, 1, 1, 5, 4)]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv2d_equals_torch(case):
    Ci, Co, k, s, p, g, H, W = case
    x = rng.standard_normal((Ci, H, W))
    w = rng.standard_normal((Co, Ci // g, k, k))
    b = rng.standard_normal(Co)
    ref = F.conv2d(torch.tensor(x)[None], torch.tensor(w), torch.tensor(b), stride=s, padding=p, groups=g)[0]
    assert np.max(np.abs(O.conv2d(x, w, b, s, p, g) - ref.numpy())) < 1e-12


DECONV_CASES = [  # Ci, Co, k, stride, pad, groups, H, W
    (8, 8, 1, 1, 0, 8, 5, 6), (8, 8, 3, 1, 1, 8, 5, 6), (16, 8, 4, 2, 1, 1, 4, 5), (4, 6, 4, 2, 1, 2, 3, 3),
    (5, 3, 3, 2, 0, 1, 4, 4)]


@pytest.mark.parametrize("case", DECONV_CASES)
def test_conv_transpose2d_equals_torch(case):
    Ci, Co, k, s, p, g, H, W = case
    x = rng.standard_normal((Ci, H, W))
    w = rng.standard_normal((Ci, Co // g, k, k))
    b = rng.standard_normal(Co)
    ref = F.conv_transpose2d(torch.tensor(x)[None], torch.tensor(w), torch.tensor(b), stride=s, padding=p,
                             groups=g)[0]
    assert np.max(np.abs(O.conv_transpose2d(x, w, b, s, p, g) - ref.numpy())) < 1e-12


def test_deconv_equals_zero_insertion_then_flipped_conv():
    """Transposed conv (stride s, pad p, kernel k) = insert s-1 zeros between
    inputs, pad by k-1-p, and correlate with the spatially flipped kernel
    whose in/out channel axes are swapped (textbook identity)."""
    Ci, Co, k, s, p, H, W = 6, 4, 4, 2, 1, 5, 7
    x = rng.standard_normal((Ci, H, W))
    w = rng.standard_normal((Ci, Co, k, k))
    up = np.zeros((Ci, (H - 1) * s + 1, (W - 1) * s + 1))
    up[:, ::s, ::s] = x
    wf = np.ascontiguousarray(np.flip(w, axis=(2, 3)).transpose(1, 0, 2, 3))
    ref = O.conv2d(up, wf, None, 1, k - 1 - p, 1)
    assert np.max(np.abs(O.conv_transpose2d(x, w, None, s, p, 1) - ref)) < 1e-12


def test_eca_special_cases():
    """Eq. 'eca_process_equation': a zero 1-D kernel gives weight sigmoid(0) =
    1/2 exactly; a channel-constant map has GAP equal to that constant."""
    m = rng.standard_normal((8, 5, 6))
    assert np.array_equal(O.eca(m, np.zeros(3)), 0.5 * m)
    c = rng.uniform(0.2, 1.0, 8)
    mc = np.broadcast_to(c[:, None, None], (8, 4, 4)).copy()
    k3 = np.array([0.0, 1.0, 0.0])
    assert np.allclose(O.eca(mc, k3)[:, 0, 0], c / (1 + np.exp(-c)), rtol=0, atol=1e-15)


def test_eca_equals_torch():
    m = rng.standard_normal((16, 6, 5))
    k3 = rng.standard_normal(3)
    t = torch.tensor(m)[None]
    g = F.adaptive_avg_pool2d(t, 1)[:, :, 0, 0]
    s = torch.sigmoid(F.conv1d(g[:, None, :], torch.tensor(k3).view(1, 1, 3), padding=1))[:, 0]
    assert np.max(np.abs(O.eca(m, k3) - (t * s[:, :, None, None])[0].numpy())) < 1e-14


# ------------------------------------------------------------ whole network
def test_param_count_matches_paper():
    """Table 'performance_radar_stda': 0.14 M parameters."""
    n = O.num_params()
    assert n == I.NUM_PARAMS == 137915
    assert round(n / 1e6, 2) == GOLDEN["model"]["params_M"]
    assert O.num_buffers() == I.NUM_BUFFERS == 1360


@pytest.mark.parametrize("H,W", [(16, 16), (24, 40), (64, 64)])
def test_network_equals_torch_composition(weights, H, W):
    params, buffers = weights
    x = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    z, blocks = O.forward(params, buffers, x, return_blocks=True)
    zr, br = torch_reference(params, buffers, x)
    assert z.shape == (H, W)
    assert np.max(np.abs(z - zr)) < 1e-12
    for got, ref in zip(blocks, br):
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) < 1e-11 * max(1.0, np.abs(ref).max())


def test_network_block_shapes_follow_the_stage_equations(weights):
    """Encoder stage 2: c -> 2c, h -> h/2; decoder stage 2: 2c -> c, h/2 -> h."""
    params, buffers = weights
    x = rng.uniform(0, 1, (3, 32, 48)).astype(np.float32)
    _, blocks = O.forward(params, buffers, x, return_blocks=True)
    assert [b.shape for b in blocks] == [(16, 16, 24), (32, 8, 12), (64, 4, 6), (32, 8, 12), (16, 16, 24),
                                         (8, 32, 48)]


def test_network_rejects_shapes_not_multiple_of_8(weights):
    with pytest.raises(ValueError):
        O.forward(*weights, np.zeros((3, 12, 16), np.float32))


def test_batch_forward_equals_single(weights):
    params, buffers = weights
    x = rng.uniform(0, 1, (5, 3, 16, 24)).astype(np.float32)
    zb = O.forward_batch(params, buffers, x, nthreads=3)
    for b in range(5):
        assert np.array_equal(zb[b], O.forward(params, buffers, x[b]))


def test_output_is_not_degenerate(weights):
    """With the recorded output gain the sigmoid is neither flat nor saturated
    on a generated window, so tolerance checks are meaningful."""
    noisy, _, _ = O.gen_window(0, 1, 0, I.WORKLOADS[1].gen)
    z = O.forward(*weights, noisy.astype(np.float32))
    assert z.std() >= 0.05
    assert np.mean((z > 0.05) & (z < 0.95)) >= 0.5


# ------------------------------------------------------------------ CA-CFAR
def test_cacfar_closed_forms():
    """A single bright cell on a constant floor is the only detection; a
    constant map has none (every cell equals its training mean, and alpha >
    1); the CA-CFAR factor is N (pfa^(-1/N) - 1)."""
    z = np.full((24, 20), 0.1)
    det, n = O.cacfar(z, 2, 4, 1e-3)
    assert n == 0
    z[10, 7] = 1.0
    det, n = O.cacfar(z, 2, 4, 1e-3)
    assert n == 1 and det[10, 7] == 1
    # threshold closed form: interior cell, N = 13^2 - 5^2 = 144 training cells
    N = 144
    alpha = N * (1e-3 ** (-1.0 / N) - 1.0)
    z2 = np.full((24, 20), 0.1)
    z2[10, 7] = 0.1 * np.sqrt(alpha) * 1.001
    assert O.cacfar(z2, 2, 4, 1e-3)[0][10, 7] == 1
    z2[10, 7] = 0.1 * np.sqrt(alpha) * 0.999
    assert O.cacfar(z2, 2, 4, 1e-3)[0][10, 7] == 0
    bins = np.array([[10, 7], [3, 3], [10, 7]])
    assert O.detect_rate(det, bins) == 0.5
