"""Pins of the oracle's fusion variants (Sec. IV-A, Eq. concat_operation
with T = 2 or 4 stacked maps instead of 3): against an independent PyTorch
float64 composition, the three-map network, and the reduction T=4 -> T=3
when the fourth map's stem weights are zero."""
import numpy as np
import pytest

import oracle as O
from paper_2307_09063_gb300 import inputs as I
from torch_ref import torch_reference


@pytest.mark.parametrize("T", [2, 4])
def test_variant_matches_torch_composition(T):
    params, bufs = I.init_params(5, frames=T)
    assert params.size == O.num_params_frames(T)
    x = np.random.default_rng(T).uniform(0, 1, (T, 24, 32)).astype(np.float32)
    z = O.forward_frames(params, bufs, x)
    zt, _ = torch_reference(params, bufs, x)
    assert np.max(np.abs(z - zt)) <= 1e-12


def test_three_maps_is_the_paper_network():
    params, bufs = I.init_params(2)
    x = np.random.default_rng(0).uniform(0, 1, (3, 16, 24)).astype(np.float32)
    assert np.array_equal(O.forward_frames(params, bufs, x), O.forward(params, bufs, x))


def test_zero_fourth_map_weights_reduce_to_three_maps():
    p3, bufs = I.init_params(7)
    p4, _ = I.init_params(7, frames=4)
    o3, o4 = I.param_offsets(3), I.param_offsets(4)
    w3 = p3[o3["stem.w"][0]:o3["stem.w"][0] + 216].reshape(8, 3, 9)
    w4 = np.zeros((8, 4, 9), np.float32)
    w4[:, :3] = w3
    p4 = p4.copy()
    p4[o4["stem.w"][0]:o4["stem.w"][0] + 288] = w4.ravel()
    p4[o4["stem.bn.gamma"][0]:] = p3[o3["stem.bn.gamma"][0]:]
    x = np.random.default_rng(1).uniform(0, 1, (4, 16, 16)).astype(np.float32)
    z4 = O.forward_frames(p4, bufs, x)
    z3 = O.forward(p3, bufs, x[:3])
    assert np.max(np.abs(z4 - z3)) <= 1e-14
