"""Serving: per-radar frame rings, continuous batching of mixed map sizes,
memory-based admission. Each served output must equal the same window
denoised alone (windows are independent in the network), and match the
oracle within the BF16 bound."""
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


def frame_pool(stda, H, W, n=4):
    g = I.SERVING_SIZES[(H, W)]
    noisy, _, _, _ = stda.generate(g, 0, I.SERVING_CID, H * 1000 + W, n, dtype=torch.bfloat16, with_clean=False)
    return [noisy[i, f].contiguous() for i in range(n) for f in range(3)]


def test_served_outputs_equal_windows_run_alone(stda, weights):
    sizes = [(128, 64)] * 3 + [(256, 128)] * 2 + [(512, 256)]  # the 3:2:1 mix
    pools = {s: frame_pool(stda, *s) for s in set(sizes)}
    ctx = stda.Context(512, 256, 8, "bf16", 0)
    nframes = 6
    frames, outs, events, expect = {}, {}, {}, {}
    rng = np.random.default_rng(0)
    order = [(r, k) for k in range(nframes) for r in range(len(sizes))]
    # interleave radars, flush at random points
    for r, k in order:
        H, W = sizes[r]
        f = pools[(H, W)][(r * 5 + k) % len(pools[(H, W)])]
        frames[(r, k)] = f
        out = torch.full((H, W), float("nan"), dtype=torch.bfloat16, device="cuda")
        ev = torch.cuda.Event()
        st = ctx.submit(r, f, out, ev)
        if k < 2:
            assert st == stda.WARMUP
            continue
        assert st == stda.OK
        outs[(r, k)], events[(r, k)] = out, ev
        if rng.uniform() < 0.3:
            ctx.flush()
    ctx.flush()
    torch.cuda.synchronize()
    alone = stda.Context(512, 256, 1, "bf16", 0)
    for (r, k), out in outs.items():
        assert events[(r, k)].query()
        x = torch.stack([frames[(r, k)], frames[(r, k - 1)], frames[(r, k - 2)]])[None].contiguous()
        ref = alone.forward(x)[0, 0]
        assert torch.equal(out, ref), (r, k)
    # one served window against the oracle
    r, k = 5, nframes - 1
    x = torch.stack([frames[(r, k)], frames[(r, k - 1)], frames[(r, k - 2)]]).float().cpu().numpy()
    zr = O.forward(*weights, x)
    assert np.max(np.abs(outs[(r, k)].float().cpu().numpy() - zr)) <= 2e-2
    assert ctx.device_status() == stda.OK


def test_admission_by_memory_budget_and_release(stda):
    pool = frame_pool(stda, 128, 64, n=1)
    probe = stda.Context(128, 64, 1, "bf16", 0)
    out = torch.empty((128, 64), dtype=torch.bfloat16, device="cuda")
    probe.submit(0, pool[0], out)
    one_radar = probe.serve_bytes()  # ring + the size class buffers
    ring = 3 * 128 * 64 * 2
    ctx = stda.Context(128, 64, 1, "bf16", 0, mem_budget_bytes=one_radar + ring // 2)
    assert ctx.submit(1, pool[0], out) == stda.WARMUP
    assert ctx.submit(2, pool[0], out) == stda.ERR_BUSY  # no room for a second ring
    assert ctx.serve_radars() == 1
    ctx.serve_close(1)
    assert ctx.serve_radars() == 0
    assert ctx.submit(2, pool[0], out) == stda.WARMUP  # admitted once memory freed up


def test_radar_cannot_change_size(stda):
    ctx = stda.Context(256, 128, 1, "bf16", 0)
    a = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros((256, 128), dtype=torch.bfloat16, device="cuda")
    assert ctx.submit(7, a, a.clone()) == stda.WARMUP
    with pytest.raises(stda.StdaError):
        ctx.submit(7, b, b.clone())
