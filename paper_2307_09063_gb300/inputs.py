"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method itself: only the workload
shapes and value ranges, a counter-based random number generator (SplitMix64,
Steele, Lea & Flood 2014, used as a stateless hash), and the random
initialisation of the network's parameters and batch-norm running
statistics. Both the oracle and the CUDA library receive what it produces;
the CUDA library also re-implements the same parameter initialisation from
the same published generator so that ``stda_create`` can build weights from
a seed without Python.
"""
from __future__ import annotations

import dataclasses

import numpy as np

MASK64 = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output function on uint64 numpy values (wrapping)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = x + _GOLDEN
        x = (x ^ (x >> np.uint64(30))) * _M1
        x = (x ^ (x >> np.uint64(27))) * _M2
        return x ^ (x >> np.uint64(31))


def key(seed, cid, w, tag, i1, i2):
    """Hash chain over (seed, workload id, window, tag, i1, i2); each may be an array."""
    u = lambda v: np.asarray(v, dtype=np.uint64)
    h = splitmix64(u(seed))
    for v in (cid, w, tag, i1, i2):
        h = splitmix64(h ^ u(v))
    return h


def u01(k):
    """Uniform double in [0, 1): (k >> 11) * 2^-53."""
    return (np.asarray(k, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# --------------------------------------------------------------------------
# Workloads: three-frame range-Doppler windows. H = range bins (P), W =
# Doppler bins (Q). N samples per chirp, M chirps per frame.
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class GenConfig:
    N: int
    M: int
    P: int
    Q: int
    tmin: int
    tmax: int
    imin: int
    imax: int
    snr_min: float
    snr_max: float
    inr_min: float = 0.0
    inr_max: float = 30.0
    kmin: float = 0.5
    kmax: float = 2.0

    @property
    def H(self):
        return self.P

    @property
    def W(self):
        return self.Q


@dataclasses.dataclass(frozen=True)
class Workload:
    cid: int
    name: str
    gen: GenConfig
    batch: int
    precision: str  # "fp32" | "bf16" | "fp8"


WORKLOADS = {
    1: Workload(1, "fp32_b1_3x64x64", GenConfig(64, 16, 64, 64, 2, 2, 1, 1, 10.0, 10.0), 1, "fp32"),
    2: Workload(2, "bf16_b256_3x256x128", GenConfig(256, 128, 256, 128, 1, 8, 1, 3, 0.0, 20.0), 256, "bf16"),
    3: Workload(3, "train_bf16_b64_3x256x128", GenConfig(256, 128, 256, 128, 1, 8, 1, 3, 0.0, 20.0), 64, "bf16"),
    4: Workload(4, "fp8_b1024_3x512x256", GenConfig(512, 256, 512, 256, 1, 16, 1, 4, 0.0, 20.0), 1024, "fp8"),
}

# Serving map sizes (H x W) and their generator shapes, 3:2:1 mix.
SERVING_SIZES = {
    (128, 64): GenConfig(128, 64, 128, 64, 1, 8, 1, 3, 0.0, 20.0),
    (256, 128): GenConfig(256, 128, 256, 128, 1, 8, 1, 3, 0.0, 20.0),
    (512, 256): GenConfig(512, 256, 512, 256, 1, 16, 1, 4, 0.0, 20.0),
}
SERVING_CID = 5

# Small generator shapes used by tests (several tiles and a ragged tail).
def small_gen(H, W, tmin=1, tmax=4, imin=1, imax=2):
    return GenConfig(H, W, H, W, tmin, tmax, imin, imax, 0.0, 20.0)


def parity_windows(B, k=8):
    """The sampled windows of a batch that are checked one by one."""
    return sorted({(37 * i) % B for i in range(k)})


# --------------------------------------------------------------------------
# Parameter initialisation. Every value is U(lo, hi) drawn from key(seed, 0,
# 0, TAG, tensor id, element index), computed in float64, rounded to float32.
# --------------------------------------------------------------------------
TAG_WEIGHT = 20
TAG_BN_MEAN = 21
TAG_BN_VAR = 22

ENC = (1, 1, 1, 0, 0, 0)
CIN = (8, 16, 32, 64, 32, 16)
OUT_GAIN = 3.0  # output-conv gain: keeps the sigmoid output spread out (std ~0.2)


def _cout(b):
    return 2 * CIN[b] if ENC[b] else CIN[b] // 2


FRAMES = 3  # maps per window (Eq. concat_operation); the fusion variants take 2 or 4


def param_table(frames: int = FRAMES):
    """Canonical parameter tensors: list of (name, size, lo, hi). `frames`
    input maps per window set the stem's input channels."""
    t = []

    def conv(name, size, fan):
        bound = float(np.sqrt(6.0 / fan))
        t.append((name, size, -bound, bound))

    def bn(name, c):
        t.append((name + ".gamma", c, 0.8, 1.2))
        t.append((name + ".beta", c, -0.1, 0.1))

    conv("stem.w", 8 * frames * 9, frames * 9)
    bn("stem.bn", 8)
    for b in range(6):
        ci, co = CIN[b], _cout(b)
        p = f"blk{b}"
        conv(p + ".w1", ci, 1)
        bn(p + ".bn1", ci)
        conv(p + ".w3", 9 * ci, 9)
        bn(p + ".bn2", ci)
        bn(p + ".bn3", ci)
        if ENC[b]:
            dense, fan = co * ci * 9, ci * 9
        else:
            dense, fan = ci * co * 16, ci * 16 // 4
        conv(p + ".w2", dense, fan)
        bn(p + ".bn", co)
        conv(p + ".rw", dense, fan)
        t.append((p + ".rb", co, -0.05, 0.05))
        t.append((p + ".eca", 3, -0.577, 0.577))
    conv("out.w", 72, 72)
    t.append(("out.b", 1, -0.05, 0.05))
    return t


def bn_table():
    """BN running statistics: list of (name, channels) in buffer order."""
    t = [("stem.bn", 8)]
    for b in range(6):
        ci, co = CIN[b], _cout(b)
        t += [(f"blk{b}.bn1", ci), (f"blk{b}.bn2", ci), (f"blk{b}.bn3", ci), (f"blk{b}.bn", co)]
    return t


NUM_PARAMS = sum(s for _, s, _, _ in param_table())
NUM_BUFFERS = 2 * sum(c for _, c in bn_table())


def init_params(seed: int = 0, frames: int = FRAMES):
    """(params float32[NUM_PARAMS], buffers float32[NUM_BUFFERS]) from a seed
    (NUM_PARAMS of the 3-map network; the stem grows with `frames`)."""
    out = []
    for tid, (name, size, lo, hi) in enumerate(param_table(frames)):
        u = u01(key(seed, 0, 0, TAG_WEIGHT, tid, np.arange(size)))
        v = lo + (hi - lo) * u
        if name == "out.w":
            v = v * OUT_GAIN
        out.append(v.astype(np.float32))
    params = np.concatenate(out)
    bufs = []
    for bid, (name, c) in enumerate(bn_table()):
        mu = -0.1 + 0.2 * u01(key(seed, 0, 0, TAG_BN_MEAN, bid, np.arange(c)))
        var = 0.8 + 0.4 * u01(key(seed, 0, 0, TAG_BN_VAR, bid, np.arange(c)))
        bufs += [mu.astype(np.float32), var.astype(np.float32)]
    return params, np.concatenate(bufs)


def param_offsets(frames: int = FRAMES):
    """name -> (offset, size) in the flat parameter blob."""
    off, d = 0, {}
    for name, size, _, _ in param_table(frames):
        d[name] = (off, size)
        off += size
    return d
