#!/usr/bin/env python
"""Radar-STDA denoising throughput on GB300.

One step = one forward pass of the whole network (stem, three encoder and
three decoder blocks with ECA and skips, output conv) over one batch of
synthetic three-frame range-Doppler windows resident in HBM. Default
workload: 256 windows of 3 x 256 x 128 maps in BF16 (FP32 accumulation).

Prints one JSON line (rank 0). With --impl reference, times the FP64 CPU
oracle on the host cores instead (the only arm available: the paper ships
no code), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "denoised RD frames/s (3-frame windows) fwd & fwd+bwd, % HBM roofline; p99 ms"
UNIT = "frames/s"

# Multiply-accumulates per full-resolution output pixel of each kernel of the
# forward pass (plain count of the layers it computes, no halo recompute):
#   enc1_stem: stem 3->8 (216) + block-1 stage 1 dw (72) + stage 2 2x(9*8*16)/4
#   enc2: dw 16*9/4 + 2x(9*16*32)/16; enc3: dw 32*9/16 + 2x(9*32*64)/64
#   dec1: dw 64*9/64 + 2x(4*64*32)/16; dec2: dw 32*9/16 + 2x(4*32*16)/4
#   dec3: dw 16*9/4 + 2x(4*16*8); out: 8*9.
KERNEL_MACS_PER_PX = {"enc1_stem": 864, "enc2": 612, "enc3": 594, "dec1": 1033, "dec2": 1042,
                      "dec3": 1060, "out": 72}
MACS_PER_PX = sum(KERNEL_MACS_PER_PX.values())  # 5277
# Of those, the dense stage-2 convolutions and the stem (216 MAC/px) run on the
# tensor cores in the bf16 / fp8 paths; the depthwise stage 1 and the output
# conv stay on the FP32 FMA pipe.
KERNEL_TC_MACS_PER_PX = {"enc1_stem": 792, "enc2": 576, "enc3": 576, "dec1": 1024, "dec2": 1024, "dec3": 1024,
                         "out": 0}
FP32_LANES_PER_SM = 128


def ffma_peak_tflops(sm_count: int, sm_max_mhz: float) -> float:
    """FP32 FMA peak from the unit counts and the clock: SMs x 128 lanes x
    2 FLOP x maximum SM clock (152 SMs at 2070 MHz: 80.5 TFLOP/s)."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_max_mhz / 1e6
FP8_OVER_BF16 = 4.5 / 2.25  # nominal dense ratio


def dist_env():
    """(world, rank, local rank) of this process (torchrun sets the
    variables; a plain run is world 1, rank 0)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def first_window(rank: int, per_rank: int) -> int:
    """Windows are sharded by rank with no exchange: rank r generates and
    denoises windows r * per_rank .. (r + 1) * per_rank - 1."""
    return rank * per_rank


def reduce_max(value: float, dist, device) -> float:
    """The largest of every rank's value (the job's time is its slowest
    rank's); the value itself without torch.distributed."""
    if not dist:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, per_rank: int, steps: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the
    slowest rank's time."""
    return world * per_rank * steps / (max_ms / 1e3)


def ncu_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu record of this
    workload (profiles/traffic.json), or None when there is none or a kernel
    source changed since the capture (its sha256 differs)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(workload)
        if not rec or rec.get("kernel") != kernel:
            return None
        for src, digest in rec["sources"].items():
            with open(os.path.join(ROOT, src), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        return int(rec["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def workload(name):
    from paper_2307_09063_gb300 import inputs as I

    for w in I.WORKLOADS.values():
        if w.name == name:
            return w
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_windows(w, n):
    """The first min(n, cores) windows of workload w from the oracle's own
    generator (untimed; threads over windows), rounded to the workload's
    input type, repeated up to n windows (the forward's cost does not depend
    on the values)."""
    import concurrent.futures as cf

    import oracle as O

    k = max(1, min(n, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=k) as ex:
        maps = list(ex.map(lambda i: O.gen_window(0, w.cid, i, w.gen, with_clean=False)[0], range(k)))
    x = np.stack(maps).astype(np.float32)
    if w.precision != "fp32":
        import torch

        x = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    return np.concatenate([x] * ((n + k - 1) // k))[:n], k


def cpu_baseline(w, target_s=15.0):
    """The FP64 oracle timed on this host's cores on a bounded sample of the
    workload's own windows."""
    import oracle as O
    from paper_2307_09063_gb300 import inputs as I

    cores = os.cpu_count() or 1
    params, buffers = I.init_params(0)
    g = w.gen
    x1, _ = oracle_windows(w, 1)
    t0 = time.perf_counter()
    O.forward_batch(params, buffers, x1, nthreads=1)
    t1 = time.perf_counter() - t0
    n = int(max(cores, min(8 * cores, target_s / max(t1, 1e-3))))
    n = max(cores, (n // cores) * cores)
    x, k = oracle_windows(w, n)
    t0 = time.perf_counter()
    O.forward_batch(params, buffers, x, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": min(cores, n), "kind": "oracle",
            "sample": f"{n} windows of 3x{g.P}x{g.Q} ({k} distinct windows of the workload from the oracle's "
                      f"generator, repeated), FP64 forward, {dt:.2f} s wall on {min(cores, n)} threads"}


def run_reference(args, w, rank):
    if rank != 0:
        return
    import oracle as O
    from paper_2307_09063_gb300 import inputs as I

    O.build()
    cores = os.cpu_count() or 1
    params, buffers = I.init_params(0)
    g = w.gen
    x, _ = oracle_windows(w, cores)
    for _ in range(args.warmup):
        O.forward_batch(params, buffers, x[:1], nthreads=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.forward_batch(params, buffers, x, nthreads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = cores * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (the workload's seeded FMCW windows, oracle generator)",
            "config": {"workload": w.name, "batch": w.batch, "H": g.P, "W": g.Q, "precision": "f64 oracle",
                       "step": f"{cores} windows (one per host core) of the {w.batch}-window batch"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} windows per step x {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(seconds=3.0, warm=1.0, streams=512, rate=20.0, flush_ms=0.25, seed=0):
    """Real-time serving simulation: `streams` radars (map sizes 128x64,
    256x128, 512x256 in a 3:2:1 mix) deliver frames at Poisson times (rate
    per radar); the host loop submits arrived frames, flushes every
    `flush_ms`, and polls completion events. Latency = time from a frame's
    scheduled arrival to the host seeing its denoised map done."""
    import collections

    import torch

    from paper_2307_09063_gb300 import inputs as I
    from paper_2307_09063_gb300 import stda

    kinds = [(128, 64), (256, 128), (512, 256)]
    n_small, n_mid = streams * 3 // 6, streams * 2 // 6
    size_of = [kinds[0]] * n_small + [kinds[1]] * n_mid + [kinds[2]] * (streams - n_small - n_mid)
    rng = np.random.default_rng(seed)
    total = warm + seconds
    arr = []
    for sidx in range(streams):
        t = rng.exponential(1.0 / rate)
        while t < total:
            arr.append((t, sidx))
            t += rng.exponential(1.0 / rate)
    arr.sort()
    pools = {}
    for (H, W) in kinds:
        g = I.SERVING_SIZES[(H, W)]
        x, _, _, _ = stda.generate(g, 0, I.SERVING_CID, 0, 8, dtype=torch.bfloat16, with_clean=False)
        pools[(H, W)] = [x[i, f] for i in range(8) for f in range(3)]
    outs = {k: [torch.empty(k, dtype=torch.bfloat16, device="cuda") for _ in range(64)] for k in kinds}
    ctx = stda.Context(512, 256, 1, "bf16", 0)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    counts = [0] * streams
    fifo = {k: collections.deque() for k in kinds}
    free_events = [torch.cuda.Event() for _ in range(4096)]
    lat, done_frames, waiting = [], 0, []
    ptr, last_flush, nsub = 0, 0.0, 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while ptr < len(arr) and arr[ptr][0] <= now:
            ta, sidx = arr[ptr]
            ptr += 1
            H, W = size_of[sidx]
            k = counts[sidx]
            counts[sidx] += 1
            frame = pools[(H, W)][(sidx * 7 + k) % len(pools[(H, W)])]
            out = outs[(H, W)][nsub % 64]
            ev = free_events.pop() if free_events else torch.cuda.Event()
            st = ctx.submit(sidx, frame, out, ev, stream)
            nsub += 1
            if st == stda.OK:
                waiting.append(((H, W), ev, ta))
            else:
                free_events.append(ev)
        if waiting and (now - last_flush) * 1e3 >= flush_ms:
            # `done` is recorded when a window's batch is launched: only
            # flushed windows can be polled
            ctx.flush(stream)
            last_flush = now
            for key, ev, ta in waiting:
                fifo[key].append((ev, ta))
            waiting.clear()
        for q in fifo.values():
            while q and q[0][0].query():
                ev, ta = q.popleft()
                tdone = time.perf_counter() - t0
                if ta >= warm:
                    lat.append(tdone - ta)
                    done_frames += 1
                free_events.append(ev)
        if ptr >= len(arr):
            ctx.flush(stream)
            for key, ev, ta in waiting:
                fifo[key].append((ev, ta))
            waiting.clear()
            if all(not q for q in fifo.values()):
                break
    elapsed = seconds
    lat_ms = np.array(lat) * 1e3
    # saturation: every radar submits its next frame back to back (round
    # robin); flushes happen when a size class holds 64 windows or a radar
    # comes round again with its window still pending
    sat_frames, nsub0 = 0, nsub
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    while sat_frames < 40 * streams:
        for sidx in range(streams):
            H, W = size_of[sidx]
            k = counts[sidx]
            counts[sidx] += 1
            frame = pools[(H, W)][(sidx * 7 + k) % len(pools[(H, W)])]
            if ctx.submit(sidx, frame, outs[(H, W)][nsub % 64], None, stream) == stda.OK:
                sat_frames += 1
            nsub += 1
    ctx.flush(stream)
    torch.cuda.synchronize()
    sat = sat_frames / (time.perf_counter() - t1)
    return {"value": done_frames / elapsed, "unit": UNIT, "offered_frames_per_s": streams * rate,
            "saturation_frames_per_s": sat, "saturation_frames": sat_frames,
            "streams": streams, "mix": "128x64 : 256x128 : 512x256 = 3:2:1", "seconds": seconds,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "max_ms": float(lat_ms.max()), "frames": int(done_frames), "flush_ms": flush_ms,
            "latency": "scheduled arrival -> completion event observed by the host loop",
            "serve_bytes": ctx.serve_bytes()}



def train_leg(args, rank, world, dist, dev, stream, flush, barrier, stda):
    """The fwd+bwd training step on 64 windows of 3 x 256 x 128 (MSE against the
    clean maps), BN with running statistics and in training mode."""
    import torch

    wt = workload("train_bf16_b64_3x256x128")
    gt = wt.gen
    tctx = stda.Context(gt.P, gt.Q, wt.batch, "bf16", 0)
    tx, tclean, _, _ = stda.generate(gt, 0, wt.cid, first_window(rank, wt.batch), wt.batch, dtype=torch.bfloat16)
    for _ in range(2):
        tctx.backward(tx, target=tclean)
    def time_steps(step):
        tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.train_steps)]
        barrier()
        for i in range(args.train_steps):
            flush.fill_(i & 0xFF)
            tev[i][0].record(stream)
            step()
            tev[i][1].record(stream)
        barrier()
        tms = [a.elapsed_time(b) for a, b in tev]
        return reduce_max(sum(tms), dist, dev), tms

    ttot, tms = time_steps(lambda: tctx.backward(tx, target=tclean))
    tctx.backward_bn(tx, target=tclean, mode="batch")
    btot, _ = time_steps(lambda: tctx.backward_bn(tx, target=tclean, mode="batch"))
    # algorithmic FLOPs of one step: forward, input gradients and weight
    # gradients each cost the forward's multiply-accumulates (3 x 5277 MAC
    # per pixel), all on the FP32 FMA pipe
    _, mhz, ffma_peak = device_peaks(dev)
    tflops = 2.0 * 3 * MACS_PER_PX * wt.batch * gt.P * gt.Q / (ttot / args.train_steps / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": tflops, "peak": ffma_peak, "unit": "TFLOP/s", "frac": tflops / ffma_peak,
            "traffic": None, "flops_per_step": 2.0 * 3 * MACS_PER_PX * wt.batch * gt.P * gt.Q,
            "peak_source": f"FP32 FMA at {mhz:.0f} MHz (derived)",
            "note": "whole step: forward + input gradients + weight gradients = 3 x the forward MACs"}
    train = {"value": whole_job_rate(world, wt.batch, args.train_steps, ttot), "unit": UNIT, "roofline": roof,
             "ms_per_step": ttot / args.train_steps, "p99_ms": float(np.percentile(tms, 99)),
             "workload": wt.name, "batch": wt.batch, "steps": args.train_steps,
             "step": "forward with tape + adjoint + MSE vs clean maps, FP32 arithmetic on CUDA cores, bf16 I/O",
             "l2": "flushed between timed steps",
             "bn_batch_statistics": {"value": whole_job_rate(world, wt.batch, args.train_steps, btot),
                                     "ms_per_step": btot / args.train_steps,
                                     "step": "the same with BatchNorm in training mode (batch statistics)"}}
    del tctx
    return train


def device_peaks(dev):
    """(SM count of the device, maximum SM clock in MHz, FP32 FMA peak in
    TFLOP/s derived from them)."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return sms, mhz, ffma_peak_tflops(sms, mhz)


def forward_leg(stda, w, steps, warmup, ctx_env, keep=False):
    """Times `steps` forward passes of workload w (batch resident in HBM, L2
    flushed between steps) with CUDA events on the launching stream, with
    per-kernel event times from the library; returns the measurement (and,
    with keep, the context and tensors for the end-to-end leg)."""
    import torch

    rank, world, dist, dev, stream, flush, barrier, local = ctx_env
    g = w.gen
    B, H, W = w.batch, g.P, g.Q
    dtype = torch.float32 if w.precision == "fp32" else torch.bfloat16
    ctx = stda.Context(H, W, B, w.precision, 0)
    x, _, _, _ = stda.generate(g, 0, w.cid, first_window(rank, B), B, dtype=dtype, with_clean=False)
    out = torch.empty((B, 1, H, W), dtype=dtype, device=dev)
    torch.cuda.synchronize()
    for _ in range(warmup):
        ctx.forward(x, out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        for i in range(steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            ctx.forward(x, out)
            ev[i][1].record(stream)
        barrier()
    launches = ctx.launch_count() - launches0
    assert ctx.device_status() == stda.OK
    # per-kernel times in a second pass of the same steps (the library's
    # event pairs around every launch stay out of the timed region above)
    ctx.profile(True)
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ctx.forward(x, out)
    kt = ctx.profile_read()
    ctx.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = reduce_max(sum(step_ms), dist, dev)
    ms_per_step = tot_ms / steps
    res = {"value": whole_job_rate(world, B, steps, tot_ms), "unit": UNIT, "ms_per_step": ms_per_step,
           "steps": steps, "warmup": warmup,
           "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
           "config": {"workload": w.name, "batch": B, "H": H, "W": W, "precision": w.precision,
                      "accumulate": "fp32", "l2": "flushed (256 MB write) between timed steps"},
           "gpu_launches": int(launches), "clocks": clk.summary()}
    res.update(rooflines(w, kt, ms_per_step, dev))
    if keep:
        return res, (ctx, x, out, dtype)
    del ctx, x, out
    torch.cuda.empty_cache()
    return res


def rooflines(w, kt, ms_per_step, dev):
    """HBM fraction of the step, the dominant kernel's roofline (tensor pipe
    and FP32 FMA pipe; the larger fraction names the bound) and the whole
    step against the binding compute roofline."""
    hbm_gbs, bf16_tf, _, peak_src = load_peaks()
    sms, mhz, ffma_peak = device_peaks(dev)
    g = w.gen
    B, H, W = w.batch, g.P, g.Q
    esz = 4 if w.precision == "fp32" else 2
    px = B * H * W
    bytes_per_step = B * 4 * H * W * esz  # 3 input maps + 1 output map per window
    hbm_achieved = bytes_per_step / (ms_per_step / 1e3) / 1e9
    name = max(kt, key=lambda k: kt[k][0])
    k_ms, k_n = kt[name]
    k_avg_s = k_ms / max(k_n, 1) / 1e3
    tc = w.precision != "fp32"
    tc_macs = KERNEL_TC_MACS_PER_PX[name] if tc else 0
    fma_macs = KERNEL_MACS_PER_PX[name] - tc_macs
    alu_tf = 2.0 * fma_macs * px / k_avg_s / 1e12
    tc_tf = 2.0 * tc_macs * px / k_avg_s / 1e12
    tc_peak = bf16_tf * (FP8_OVER_BF16 if w.precision.startswith("fp8") else 1.0)
    fr_alu, fr_tc = alu_tf / ffma_peak, tc_tf / tc_peak
    shares = {k: round(v[0] / max(sum(u[0] for u in kt.values()), 1e-12), 4) for k, v in kt.items()}
    fma_src = f"FP32 FMA: {sms} SMs x 128 lanes x 2 FLOP x {mhz:.0f} MHz (derived)"
    if fr_tc > fr_alu:
        bound, ach, peak, psrc = "tensor", tc_tf, tc_peak, (
            f"{peak_src} bf16 burst {bf16_tf} TFLOP/s" + (" x 2 (fp8/bf16 nominal)" if tc_peak != bf16_tf else ""))
    else:
        bound, ach, peak, psrc = "alu", alu_tf, ffma_peak, fma_src
    roofline = {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": ncu_traffic(w.name, name), "peak_source": psrc,
                "alu": {"achieved": alu_tf, "peak": ffma_peak, "frac": fr_alu, "flops_per_launch": 2.0 * fma_macs * px},
                "tensor": {"achieved": tc_tf, "peak": tc_peak, "frac": fr_tc, "flops_per_launch": 2.0 * tc_macs * px},
                "avg_launch_ms": k_avg_s * 1e3, "time_shares": shares}
    tc_total = sum(KERNEL_TC_MACS_PER_PX.values()) if tc else 0
    t_tensor_us = 2.0 * tc_total * px / (tc_peak * 1e12) * 1e6
    t_fma_us = 2.0 * (MACS_PER_PX - tc_total) * px / (ffma_peak * 1e12) * 1e6
    step_roofline = {"t_tensor_us": t_tensor_us, "t_fma_us": t_fma_us, "bound_us": max(t_tensor_us, t_fma_us),
                     "measured_us": ms_per_step * 1e3, "frac": max(t_tensor_us, t_fma_us) / (ms_per_step * 1e3),
                     "peaks": f"tensor {tc_peak:.0f} TFLOP/s, FP32 FMA {ffma_peak:.1f} TFLOP/s"}
    return {"hbm": {"achieved_gbs": hbm_achieved, "peak_gbs": hbm_gbs, "frac": hbm_achieved / hbm_gbs,
                    "bytes_per_step": bytes_per_step, "peak_source": peak_src},
            "compute": {"macs_per_px": MACS_PER_PX, "tflops": 2.0 * MACS_PER_PX * px / (ms_per_step / 1e3) / 1e12},
            "roofline": roofline, "step_roofline": step_roofline}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bf16_b256_3x256x128",
                    help="bf16_b256_3x256x128 | fp8_b1024_3x512x256 | fp32_b1_3x64x64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the fwd+bwd training-step measurement")
    ap.add_argument("--train-steps", type=int, default=5)
    ap.add_argument("--train-only", action="store_true", help="run only the training-step measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving latency measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other forward workloads (FP32 1 x 3x64x64, FP8 1024 x 3x512x256)")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_env()
    if args.workload == "serving":
        return main_serving(args, world, rank, local)
    w = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w, rank)

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2307_09063_gb300 import build as Bld

    Bld.build()
    from paper_2307_09063_gb300 import stda

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    if args.train_only:
        # the training leg alone (for launch lists of the training kernels)
        train = train_leg(args, rank, world, dist, dev, stream, flush, barrier, stda)
        if rank == 0:
            print(json.dumps({"train_fwd_bwd": train}))
        if dist:
            dist.destroy_process_group()
        return

    env = (rank, world, dist, dev, stream, flush, barrier, local)
    main_res, (ctx, x, out, dtype) = forward_leg(stda, w, args.steps, args.warmup, env, keep=True)
    g = w.gen
    B, H, W = w.batch, g.P, g.Q
    esz = 4 if w.precision == "fp32" else 2

    # end to end through the public API on host buffers (stda_forward_host):
    # every step copies its pinned host input to the device, denoises it and
    # delivers the output to pinned host memory (the output kernel stores it
    # there directly); a step's input copy overlaps the previous step's
    # kernels, so the K steps are timed as one region (events on the
    # launching stream around all of them, every transfer inside it)
    xh = x.cpu().pin_memory()
    oh = torch.empty((B, 1, H, W), dtype=dtype).pin_memory()
    for _ in range(2):  # allocates the two staging pairs (and captures each one's forward)
        ctx.forward_host(xh, oh)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ctx.forward_host(xh, oh)
    e1.record(stream)
    barrier()
    e2e_ms = reduce_max(e0.elapsed_time(e1), dist, dev)
    e2e_value = whole_job_rate(world, B, args.steps, e2e_ms)
    del ctx, x, out
    torch.cuda.empty_cache()

    # the other forward workloads: FP32 batch 1 (3 x 64 x 64) and FP8 1024 x 3 x 512 x 256
    configs = {}
    if not args.no_configs:
        for name, steps in (("fp32_b1_3x64x64", 50), ("fp8_b1024_3x512x256", 5)):
            if name != w.name:
                configs[name] = forward_leg(stda, workload(name), steps, 3, env)

    # fwd + bwd: the training step (stda_backward, MSE against the clean maps)
    # on 64 windows of 3 x 256 x 128, one step per timed iteration
    train = None
    if not args.no_train:
        train = train_leg(args, rank, world, dist, dev, stream, flush, barrier, stda)

    line = {"metric": METRIC, "value": main_res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3x2"}.get(w.precision, w.precision),
            "data": "synthetic (seeded FMCW targets, interferers, noise; GPU generator)",
            "config": dict(main_res["config"], parallelism=f"replicas x{world}"),
            "p50_ms": main_res["p50_ms"], "p99_ms": main_res["p99_ms"],
            "hbm": main_res["hbm"], "compute": main_res["compute"], "roofline": main_res["roofline"],
            "step_roofline": main_res["step_roofline"],
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(xh.numel() * esz),
                    "d2h_bytes_per_step": int(oh.numel() * esz),
                    "call": "stda_forward_host on pinned host buffers; each step's input copy overlaps the previous step's kernels; the output kernel stores the result straight into the pinned host output; L2 flush inside the region"},
            "clocks": main_res["clocks"], "gpu_launches": main_res["gpu_launches"]}
    if configs:
        line["configs"] = configs
    if train:
        line["train_fwd_bwd"] = train
    if not args.no_serving:
        line["serving"] = run_serving(seconds=2.0, warm=1.0)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main_serving(args, world, rank, local):
    """--workload serving: the real-time serving simulation alone."""
    import torch

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the serving loop has no CPU counterpart; "
                              "the oracle arm times the forward workloads"}), flush=True)
        return
    torch.cuda.set_device(local)
    from paper_2307_09063_gb300 import build as Bld

    Bld.build()
    with ClockSampler(local) as clk:
        r = run_serving(seconds=args.serve_seconds, warm=1.0)
    line = {"metric": METRIC, "value": r["value"] * world, "unit": UNIT, "n_gpus": world, "steps": r["frames"],
            "warmup": 1, "ms_per_step": r["p50_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded FMCW frames, GPU generator)",
            "config": {"workload": "serving_512_streams_20fps_mixed", "streams": r["streams"], "mix": r["mix"],
                       "arrivals": "Poisson, 20 frames/s per radar", "parallelism": f"replicas x{world}"},
            "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "serving": r, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
