"""Tolerance of the reduced-precision (BF16 / FP8) forward against the FP64
oracle, derived from first-order rounding-error propagation.

The output is z = sigmoid(l) with logit l = b + sum over 72 terms
w[c, tap] * D3[c, p + tap] (the output conv of the network, Sec. IV-A, on the
ECA-scaled map of decoder block 3). When every term carries a relative error
of at most e, |dl| <= e * T(p) with T(p) = sum |w[c, tap] * D3[c, p + tap]|,
and |dz| <= sigmoid'(l) * |dl| = z (1 - z) e T(p) to first order. In the
BF16 path every stored activation and weight is rounded to bf16 (unit
roundoff u = 2^-9); a term of the output conv reaches the logit through the
roundings of the block input staged for the MMAs, the stage-1 output, the
weights and the stored block output, so its relative error is taken as
GROWTH = 4 roundings, e = 4 u. Hence

    max |z_bf16 - z_oracle| <= max(2e-2, 4 u kappa),
    kappa = max over pixels of z (1 - z) T(p),

with kappa computed by the FP64 oracle from the same weights and input. For
the parity weights (seed 0) kappa is about 2.4, so the stated 2e-2 bound is
the one that applies; weight draws whose activations or logits grow larger
(random draws with saturated outputs) get the proportionally larger bound.
The two-term E4M3 path keeps bf16-level operands (two E4M3 terms, about
2^-8 relative) and is held to the same bound.
"""
import numpy as np

U_BF16 = 2.0 ** -9
GROWTH = 4.0
ATOL = 2e-2
U_FP32 = 2.0 ** -24
GROWTH_FP32 = 32.0
RTOL_FP32 = 1e-4


def logit_terms(params, d3, frames=3):
    """T(p) = sum over the output conv's 72 terms of |w * D3| (zero padding),
    for d3 [8][H][W] (float64, ECA-scaled decoder-3 output)."""
    from paper_2307_09063_gb300 import inputs as I

    o, s = I.param_offsets(frames)["out.w"]
    w = np.abs(np.asarray(params[o:o + s], np.float64)).reshape(8, 3, 3)
    a = np.abs(np.asarray(d3, np.float64))
    C, H, W = a.shape
    pad = np.zeros((C, H + 2, W + 2))
    pad[:, 1:-1, 1:-1] = a
    t = np.zeros((H, W))
    for c in range(C):
        for ky in range(3):
            for kx in range(3):
                t += w[c, ky, kx] * pad[c, ky:ky + H, kx:kx + W]
    return t


def kappa(params, d3, z, frames=3):
    """max over pixels of z (1 - z) T(p) for the oracle output z [H][W]."""
    z = np.asarray(z, np.float64)
    return float(np.max(z * (1.0 - z) * logit_terms(params, d3, frames)))


def bound(k):
    """The reduced-precision tolerance for a window of sensitivity k."""
    return max(ATOL, GROWTH * U_BF16 * k)


def fp32_rel_bound(params, d3, z, frames=3):
    """Per-pixel relative tolerance of the FP32 path: max(1e-4, 32 u32 (1 - z)
    T(p)). The relative error of z = sigmoid(l) is (1 - z) |dl|; in FP32 the
    terms of the logit carry the roundings of stored activations plus those
    of sums of up to 576 products (about sqrt(576) = 24 roundings), taken as
    32 roundings of u32 = 2^-24. The bound exceeds 1e-4 only where |l| runs
    into the hundreds (saturated outputs of badly scaled weight draws)."""
    z = np.asarray(z, np.float64)
    return np.maximum(RTOL_FP32, GROWTH_FP32 * U_FP32 * (1.0 - z) * logit_terms(params, d3, frames))


def sinr_cells(bins, H, W, guard=2):
    """Masks of the SINR cell sets of Eq. (SINR): the distinct peak cells and
    the cells outside every (2 guard + 1)^2 box around a peak."""
    o = np.zeros((H, W), bool)
    n = np.ones((H, W), bool)
    for p, q in np.asarray(bins).reshape(-1, 2):
        o[p, q] = True
        n[max(0, p - guard):p + guard + 1, max(0, q - guard):q + guard + 1] = False
    return o, n


def sinr_bound(params, d3, z, bins, frames=3):
    """First-order bound of the output-SINR change (dB) when every output
    pixel moves by at most e_i = 4 u z(1-z) T(p) (the logit bound above) plus
    u z (the bf16 rounding of the output itself): |d(z^2)| <= 2 z e per
    cell, relative to the mean z^2 of each cell set."""
    z = np.asarray(z, np.float64)
    e = GROWTH * U_BF16 * z * (1.0 - z) * logit_terms(params, d3, frames) + U_BF16 * z
    o, n = sinr_cells(bins, *z.shape)
    dz2 = 2.0 * z * e
    return float(10.0 / np.log(10.0) * (dz2[o].sum() / (z[o] ** 2).sum() + dz2[n].sum() / (z[n] ** 2).sum()))
