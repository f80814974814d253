"""Radar-STDA oracle — TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU implementation of the paper's generator (Sec. III), network
(Sec. IV) and metrics (Sec. V-B), written in C (stda_oracle.c) and loaded
here through ctypes. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the CUDA library
shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stda_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so integer decisions
    taken in floating point are the same on every IEEE-754 host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "stda_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class GenCfg(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("P", ctypes.c_int), ("Q", ctypes.c_int),
                ("tmin", ctypes.c_int), ("tmax", ctypes.c_int), ("imin", ctypes.c_int), ("imax", ctypes.c_int),
                ("snr_min", ctypes.c_double), ("snr_max", ctypes.c_double),
                ("inr_min", ctypes.c_double), ("inr_max", ctypes.c_double),
                ("kmin", ctypes.c_double), ("kmax", ctypes.c_double)]


MAX_TGT = 16
MAX_INT = 4


class Scene(ctypes.Structure):
    _fields_ = [("n_tgt", ctypes.c_int),
                ("r", ctypes.c_double * MAX_TGT), ("d", ctypes.c_double * MAX_TGT),
                ("delta", ctypes.c_double * MAX_TGT), ("phase", (ctypes.c_double * MAX_TGT) * 3),
                ("n_int", ctypes.c_int * 3),
                ("kappa", (ctypes.c_double * MAX_INT) * 3), ("nx", (ctypes.c_double * MAX_INT) * 3),
                ("amp_i", (ctypes.c_double * MAX_INT) * 3),
                ("snr_db", ctypes.c_double), ("sigma", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)
_U64 = ctypes.c_uint64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_splitmix64.restype = _U64
            L.orc_splitmix64.argtypes = [_U64]
            L.orc_key.restype = _U64
            L.orc_key.argtypes = [_U64] * 6
            L.orc_u01.restype = ctypes.c_double
            L.orc_u01.argtypes = [_U64]
            L.orc_draw_scene.argtypes = [_U64, _U64, _U64, ctypes.POINTER(GenCfg), ctypes.POINTER(Scene)]
            L.orc_if_signal.argtypes = [_U64, _U64, _U64, ctypes.POINTER(GenCfg), ctypes.POINTER(Scene),
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            L.orc_rd_complex.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            L.orc_lognorm.argtypes = [_D, _D, ctypes.c_int, _D]
            L.orc_peak_bins.restype = ctypes.c_int
            L.orc_peak_bins.argtypes = [ctypes.POINTER(GenCfg), ctypes.POINTER(Scene), _I]
            L.orc_gen_window.restype = ctypes.c_int
            L.orc_gen_window.argtypes = [_U64, _U64, _U64, ctypes.POINTER(GenCfg), _D, _D, _I]
            L.orc_radar_helpers.argtypes = [ctypes.c_int, ctypes.c_int, _D]
            L.orc_num_params.restype = ctypes.c_int
            L.orc_num_buffers.restype = ctypes.c_int
            L.orc_forward.restype = ctypes.c_int
            L.orc_forward.argtypes = [_F, _F, _F, ctypes.c_int, ctypes.c_int, _D, _D]
            L.orc_forward_batch.restype = ctypes.c_int
            L.orc_forward_batch.argtypes = [_F, _F, _F, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int]
            L.orc_conv2d.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
            L.orc_conv_transpose2d.argtypes = L.orc_conv2d.argtypes
            L.orc_eca.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
            L.orc_cacfar.restype = ctypes.c_int
            L.orc_cacfar.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_ubyte)]
            L.orc_detect_rate.restype = ctypes.c_double
            L.orc_detect_rate.argtypes = [ctypes.POINTER(ctypes.c_ubyte), ctypes.c_int, ctypes.c_int, _I, ctypes.c_int]
            L.orc_sinr_db.restype = ctypes.c_double
            L.orc_sinr_db.argtypes = [_D, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int, ctypes.c_int]
            L.orc_evm.restype = ctypes.c_double
            L.orc_evm.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int]
            L.orc_loss_grad.restype = ctypes.c_double
            L.orc_loss_grad.argtypes = [_F, _F, _F, _F, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int]
            L.orc_adjoint.restype = ctypes.c_int
            L.orc_adjoint.argtypes = [_F, _F, _F, _D, ctypes.c_int, ctypes.c_int, _D, _D]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def gen_cfg(g) -> GenCfg:
    """ctypes config from an inputs.GenConfig (or any object with the fields)."""
    return GenCfg(g.N, g.M, g.P, g.Q, g.tmin, g.tmax, g.imin, g.imax, g.snr_min, g.snr_max,
                  g.inr_min, g.inr_max, g.kmin, g.kmax)


# ---------------------------------------------------------------- generator
def draw_scene(seed, cid, w, g) -> Scene:
    sc = Scene()
    lib().orc_draw_scene(seed, cid, w, ctypes.byref(gen_cfg(g)), ctypes.byref(sc))
    return sc


def if_signal(seed, cid, w, g, sc, f, with_int=True, with_noise=True):
    re = np.empty((g.N, g.M))
    im = np.empty((g.N, g.M))
    lib().orc_if_signal(seed, cid, w, ctypes.byref(gen_cfg(g)), ctypes.byref(sc), f, int(with_int),
                        int(with_noise), _p(re, _D), _p(im, _D))
    return re + 1j * im


def rd_complex(s, P, Q):
    s = np.asarray(s, dtype=np.complex128)
    N, M = s.shape
    re, im = _f64(s.real), _f64(s.imag)
    yr = np.empty((P, Q))
    yi = np.empty((P, Q))
    lib().orc_rd_complex(_p(re, _D), _p(im, _D), N, M, P, Q, _p(yr, _D), _p(yi, _D))
    return yr + 1j * yi


def lognorm(y):
    y = np.asarray(y, dtype=np.complex128)
    re, im = _f64(y.real), _f64(y.imag)
    z = np.empty(y.shape)
    lib().orc_lognorm(_p(re, _D), _p(im, _D), y.size, _p(z, _D))
    return z


def peak_bins(g, sc):
    b = np.zeros((MAX_TGT, 2), dtype=np.int32)
    n = lib().orc_peak_bins(ctypes.byref(gen_cfg(g)), ctypes.byref(sc), _p(b, _I))
    return b[:n].copy()


def gen_window(seed, cid, w, g, with_clean=True):
    """(noisy[3][P][Q], clean[P][Q] or None, bins[n][2]) in float64."""
    noisy = np.empty((3, g.P, g.Q))
    clean = np.empty((g.P, g.Q)) if with_clean else None
    b = np.zeros((MAX_TGT, 2), dtype=np.int32)
    n = lib().orc_gen_window(seed, cid, w, ctypes.byref(gen_cfg(g)), _p(noisy, _D),
                             _p(clean, _D) if with_clean else None, _p(b, _I))
    return noisy, clean, b[:n].copy()


def radar_helpers(N, M):
    o = np.empty(4)
    lib().orc_radar_helpers(N, M, _p(o, _D))
    return o


# ------------------------------------------------------------------ network
def num_params():
    return lib().orc_num_params()


def num_buffers():
    return lib().orc_num_buffers()


BLOCK_SHAPES = [(16, 2), (32, 4), (64, 8), (32, 4), (16, 2), (8, 1)]  # (C, downsample)


def forward(params, buffers, x, return_blocks=False):
    """x[3][H][W] -> z[H][W] (float64); optionally the six block outputs."""
    params, buffers, x = _f32(params), _f32(buffers), _f32(x)
    _, H, W = x.shape
    out = np.empty((H, W))
    blocks = None
    if return_blocks:
        tot = sum(c * (H // s) * (W // s) for c, s in BLOCK_SHAPES)
        blocks = np.empty(tot)
    rc = lib().orc_forward(_p(params, _F), _p(buffers, _F), _p(x, _F), H, W, _p(out, _D),
                           _p(blocks, _D) if return_blocks else None)
    if rc:
        raise ValueError(f"oracle forward rejected shape {H}x{W}")
    if not return_blocks:
        return out
    res, off = [], 0
    for c, s in BLOCK_SHAPES:
        n = c * (H // s) * (W // s)
        res.append(blocks[off:off + n].reshape(c, H // s, W // s))
        off += n
    return out, res


def num_params_frames(frames):
    return lib().orc_num_params_frames(frames)


def forward_frames(params, buffers, x):
    """Fusion variant (Sec. IV-A): x[T][H][W] with T = 2..4 stacked maps,
    params of that variant (stem W[8][T][3][3]) -> z[H][W] (float64)."""
    params, buffers, x = _f32(params), _f32(buffers), _f32(x)
    T, H, W = x.shape
    assert params.size == num_params_frames(T)
    out = np.empty((H, W))
    rc = lib().orc_forward_frames(_p(params, _F), _p(buffers, _F), _p(x, _F), T, H, W, _p(out, _D))
    if rc:
        raise ValueError(f"oracle forward rejected {T} frames of {H}x{W}")
    return out


def forward_batch(params, buffers, x, nthreads=None):
    """x[B][3][H][W] -> z[B][H][W] (float64), POSIX threads over windows."""
    params, buffers, x = _f32(params), _f32(buffers), _f32(x)
    B, _, H, W = x.shape
    out = np.empty((B, H, W))
    nt = nthreads or os.cpu_count() or 1
    rc = lib().orc_forward_batch(_p(params, _F), _p(buffers, _F), _p(x, _F), B, H, W, _p(out, _D), nt)
    if rc:
        raise ValueError(f"oracle forward rejected shape {H}x{W}")
    return out


def loss_grad_bn(params, buffers, x, target, mode=1):
    """MSE loss, dL/dtheta [num_params] and the BN statistics used
    ([num_buffers], BN-buffer layout) of a batch x[B][3][H][W] against
    target[B][H][W], with BN in training mode (mode 1: batch statistics) or
    with the running statistics (mode 0)."""
    params, buffers, x, target = _f32(params), _f32(buffers), _f32(x), _f32(target)
    B, _, H, W = x.shape
    g = np.empty(num_params())
    st = np.empty(num_buffers())
    lib().orc_loss_grad_bn.restype = ctypes.c_double
    loss = lib().orc_loss_grad_bn(_p(params, _F), _p(buffers, _F), _p(x, _F), _p(target, _F), B, H, W, mode,
                                  _p(g, _D), _p(st, _D))
    if np.isnan(loss):
        raise ValueError(f"oracle rejected shape {H}x{W}")
    return loss, g, st


def conv2d(x, w, bias, stride, pad, groups):
    x, w = _f64(x), _f64(w)
    Ci, H, W = x.shape
    Co, _, k, _ = w.shape
    Ho, Wo = (H + 2 * pad - k) // stride + 1, (W + 2 * pad - k) // stride + 1
    y = np.empty((Co, Ho, Wo))
    b = None if bias is None else _f64(bias)
    lib().orc_conv2d(_p(x, _D), Ci, H, W, _p(w, _D), None if b is None else _p(b, _D), Co, k, stride, pad,
                     groups, _p(y, _D))
    return y


def conv_transpose2d(x, w, bias, stride, pad, groups):
    x, w = _f64(x), _f64(w)
    Ci, H, W = x.shape
    _, cog, k, _ = w.shape
    Co = cog * groups
    Ho, Wo = (H - 1) * stride - 2 * pad + k, (W - 1) * stride - 2 * pad + k
    y = np.empty((Co, Ho, Wo))
    b = None if bias is None else _f64(bias)
    lib().orc_conv_transpose2d(_p(x, _D), Ci, H, W, _p(w, _D), None if b is None else _p(b, _D), Co, k,
                               stride, pad, groups, _p(y, _D))
    return y


def eca(m, k3):
    m = _f64(m).copy()
    C, h, w = m.shape
    k3 = _f64(k3)
    lib().orc_eca(_p(m, _D), C, h, w, _p(k3, _D))
    return m


def adjoint(params, buffers, x, gout):
    """(dL/dtheta [num_params], dL/dx [3][H][W]) of one window given dL/dz."""
    params, buffers, x = _f32(params), _f32(buffers), _f32(x)
    _, H, W = x.shape
    g = _f64(gout)
    gp = np.empty(num_params())
    gi = np.empty((3, H, W))
    if lib().orc_adjoint(_p(params, _F), _p(buffers, _F), _p(x, _F), _p(g, _D), H, W, _p(gp, _D), _p(gi, _D)):
        raise ValueError("oracle adjoint rejected the shape")
    return gp, gi


def loss_grad(params, buffers, x, target, nthreads=None):
    """(MSE loss, dL/dtheta) over a batch x[B][3][H][W], target[B][H][W]."""
    params, buffers, x, t = _f32(params), _f32(buffers), _f32(x), _f32(target)
    B, _, H, W = x.shape
    gp = np.empty(num_params())
    loss = lib().orc_loss_grad(_p(params, _F), _p(buffers, _F), _p(x, _F), _p(t, _F), B, H, W, _p(gp, _D),
                               nthreads or os.cpu_count() or 1)
    return loss, gp


# ------------------------------------------------------------------ metrics
def sinr_db(z, bins, guard=2):
    z = _f64(z)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    return lib().orc_sinr_db(_p(z, _D), z.shape[0], z.shape[1], _p(b, _I), len(b), guard)


def evm(clean, est, bins):
    c, e = _f64(clean), _f64(est)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    return lib().orc_evm(_p(c, _D), _p(e, _D), c.shape[0], c.shape[1], _p(b, _I), len(b))


def cacfar(z, guard=2, train=4, pfa=1e-3):
    """(detections [P][Q] uint8, count) of CA-CFAR on map z."""
    z = _f64(z)
    det = np.zeros(z.shape, dtype=np.uint8)
    n = lib().orc_cacfar(_p(z, _D), z.shape[0], z.shape[1], guard, train, pfa,
                         det.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return det, n


def detect_rate(det, bins):
    det = np.ascontiguousarray(det, dtype=np.uint8)
    b = np.ascontiguousarray(bins, dtype=np.int32)
    return lib().orc_detect_rate(det.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), det.shape[0], det.shape[1],
                                 _p(b, _I), len(b))
