"""GPU evaluation (stda_metrics) against the oracle on the same maps: SINR
and EVM equal to FP64 rounding, CA-CFAR detections bit-exact."""
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


@pytest.mark.parametrize("cid", [1, 2])
def test_metrics_match_oracle(stda, weights, cid):
    w = I.WORKLOADS[cid]
    g = w.gen
    maps, cleans, binsl = [], [], []
    for k in range(3):
        noisy, clean, bins = O.gen_window(0, cid, k, g)
        den = O.forward(*weights, noisy.astype(np.float32))
        maps += [noisy[0], den]
        cleans += [clean, clean]
        binsl += [bins, bins]
    B = len(maps)
    m = np.stack(maps).astype(np.float32)
    c = np.stack(cleans).astype(np.float32)
    bins = np.full((B, 16, 2), -1, np.int32)
    ntgt = np.zeros(B, np.int32)
    for i, b in enumerate(binsl):
        bins[i, :len(b)] = b
        ntgt[i] = len(b)
    sinr, evm, rate, det = stda.metrics(torch.from_numpy(m).cuda(), torch.from_numpy(bins).cuda(),
                                        torch.from_numpy(ntgt).cuda(), clean=torch.from_numpy(c).cuda(),
                                        want_det=True)
    torch.cuda.synchronize()
    for i in range(B):
        mi, ci, bi = m[i].astype(np.float64), c[i].astype(np.float64), binsl[i]
        assert abs(sinr[i].item() - O.sinr_db(mi, bi)) <= 1e-9
        assert abs(evm[i].item() - O.evm(ci, mi, bi)) <= 1e-12
        dref, _ = O.cacfar(mi, 2, 4, 1e-3)
        assert np.array_equal(det[i].cpu().numpy(), dref)
        assert rate[i].item() == pytest.approx(O.detect_rate(dref, bi), abs=1e-7)


def test_metrics_rejects_bad_arguments(stda):
    x = torch.zeros((1, 16, 16), device="cuda")
    b = torch.zeros((1, 16, 2), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(stda.StdaError):
        stda.metrics(x, b, n, pfa=1.5)
