"""Serving: per-radar frame rings, continuous batching of mixed map sizes
into one graph launch per flush, memory-based admission. Each served output
must equal the same window denoised alone (windows are independent in the
network), and match the oracle within the BF16 bound."""
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


def test_frames_submitted_while_a_flush_is_in_flight(stda):
    """The next frames of the same radars are submitted right after each
    flush, without waiting for it: the ring copies wait only for the
    flush's gathers, and every output still equals the window alone."""
    sizes = [(256, 128), (128, 64)]
    pools = {s: frame_pool(stda, *s) for s in sizes}
    ctx = stda.Context(256, 128, 4, "bf16", 0)
    alone = stda.Context(256, 128, 1, "bf16", 0)
    hist, outs = {}, []
    for k in range(8):
        for r, (H, W) in enumerate(sizes):
            f = pools[(H, W)][(3 * r + k) % len(pools[(H, W)])]
            hist.setdefault(r, []).append(f)
            out = torch.full((H, W), float("nan"), dtype=torch.bfloat16, device="cuda")
            st = ctx.submit(r, f, out)
            if k >= 2:
                assert st == stda.OK
                outs.append((r, k, out))
        ctx.flush()  # no synchronisation before the next submits
    torch.cuda.synchronize()
    for r, k, out in outs:
        x = torch.stack([hist[r][k], hist[r][k - 1], hist[r][k - 2]])[None].contiguous()
        assert torch.equal(out, alone.forward(x)[0, 0]), (r, k)
    assert ctx.device_status() == stda.OK


def _event_ms(a, b):
    """cudaEventElapsedTime of two events (the library records the end
    events, so torch's own bookkeeping does not know them)."""
    import ctypes
    import glob

    for path in ["libcudart.so"] + sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*")):
        try:
            rt = ctypes.CDLL(path)
            break
        except OSError:
            continue
    ms = ctypes.c_float()
    assert rt.cudaEventElapsedTime(ctypes.byref(ms), ctypes.c_void_p(a.cuda_event), ctypes.c_void_p(b.cuda_event)) == 0
    return ms.value


def _flush_ms(stda, ctx, jobs, reps=7):
    """Median time from a flush to the completion of its last window, for
    jobs [(radar, frame, out)] submitted (as third frames) just before it."""
    times = []
    for _ in range(reps):
        start = torch.cuda.Event(enable_timing=True)
        ends = []
        for r, f, out in jobs:
            ev = torch.cuda.Event(enable_timing=True)
            assert ctx.submit(r, f, out, ev) == stda.OK
            ends.append(ev)
        start.record()
        ctx.flush()
        torch.cuda.synchronize()
        times.append(max(_event_ms(start, e) for e in ends))
    return float(np.median(times))


def test_two_map_sizes_overlap_in_one_flush(stda):
    """One flush launches both sizes' branches of the graph together: the
    flush with both sizes pending finishes well before the two sizes run
    one after the other would."""
    a, b = (512, 256), (256, 128)
    pa, pb = frame_pool(stda, *a, n=1), frame_pool(stda, *b, n=1)
    ctx = stda.Context(512, 256, 2, "bf16", 0)
    oa = torch.empty(a, dtype=torch.bfloat16, device="cuda")
    ob = torch.empty(b, dtype=torch.bfloat16, device="cuda")
    for k in range(2):  # warm both rings (and create both size classes)
        ctx.submit(0, pa[k], oa)
        ctx.submit(1, pb[k], ob)
    t_a = _flush_ms(stda, ctx, [(0, pa[2], oa)])
    t_b = _flush_ms(stda, ctx, [(1, pb[2], ob)])
    t_ab = _flush_ms(stda, ctx, [(0, pa[2], oa), (1, pb[2], ob)])
    print(f"flush ms: 512x256 alone {t_a:.3f}, 256x128 alone {t_b:.3f}, both {t_ab:.3f}")
    assert t_ab < 0.9 * (t_a + t_b)
    assert ctx.device_status() == stda.OK


def test_admission_while_a_flush_is_in_flight(stda):
    """A new radar refused for memory while another radar's window is being
    served is admitted once that radar closes (the close waits for its
    flush)."""
    pool = frame_pool(stda, 128, 64, n=1)
    probe = stda.Context(128, 64, 1, "bf16", 0)
    out = torch.empty((128, 64), dtype=torch.bfloat16, device="cuda")
    probe.submit(0, pool[0], out)
    budget = probe.serve_bytes() + 3 * 128 * 64 * 2 // 2
    ctx = stda.Context(128, 64, 1, "bf16", 0, mem_budget_bytes=budget)
    for k in range(3):
        ctx.submit(1, pool[k], out)
    ctx.flush()  # radar 1's window in flight
    assert ctx.submit(2, pool[0], out) == stda.ERR_BUSY
    ctx.serve_close(1)
    assert ctx.submit(2, pool[0], out) == stda.WARMUP
    assert ctx.device_status() == stda.OK
