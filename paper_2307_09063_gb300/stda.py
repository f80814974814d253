"""Thin Python binding of libstda (argument marshalling only).

Every step of the computation runs in the library's CUDA kernels; PyTorch
tensors only carry device memory and streams. Loading fails loudly when
libstda.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstda.so")

OK, ERR_INVALID_ARG, ERR_SHAPE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_UNSUPPORTED, WARMUP = range(9)
FP32, BF16, FP8_E4M3, FP8_E4M3_FAST = 0, 1, 2, 3
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8_E4M3, "fp8_fast": FP8_E4M3_FAST}
MAX_TGT = 16


class StdaError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"libstda status {status}: {msg}")


class Config(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("max_batch", ctypes.c_int), ("prec", ctypes.c_int),
                ("weight_seed", ctypes.c_uint64), ("mem_budget_bytes", ctypes.c_size_t), ("frames", ctypes.c_int)]


class GenConfig(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("P", ctypes.c_int), ("Q", ctypes.c_int),
                ("tmin", ctypes.c_int), ("tmax", ctypes.c_int), ("imin", ctypes.c_int), ("imax", ctypes.c_int),
                ("snr_min", ctypes.c_double), ("snr_max", ctypes.c_double),
                ("inr_min", ctypes.c_double), ("inr_max", ctypes.c_double),
                ("kmin", ctypes.c_double), ("kmax", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p


def lib():
    """The loaded libstda (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libstda.so is missing ({LIB_PATH}); build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        L.stda_status_string.restype = ctypes.c_char_p
        L.stda_status_string.argtypes = [ctypes.c_int]
        L.stda_num_params.restype = ctypes.c_size_t
        L.stda_num_buffers.restype = ctypes.c_size_t
        L.stda_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_VP)]
        L.stda_destroy.argtypes = [_VP]
        for n in ("stda_get_params", "stda_set_params", "stda_get_buffers", "stda_set_buffers"):
            getattr(L, n).argtypes = [_VP, _VP, ctypes.c_size_t]
        L.stda_init_params.argtypes = [ctypes.c_uint64, _VP, _VP]
        L.stda_reparam_count.restype = ctypes.c_size_t
        L.stda_reparam_count.argtypes = [ctypes.c_int]
        L.stda_reparam_export.argtypes = [_VP, _VP, ctypes.c_int, _VP, ctypes.c_size_t]
        L.stda_num_params_frames.restype = ctypes.c_size_t
        L.stda_num_params_frames.argtypes = [ctypes.c_int]
        L.stda_init_params_frames.argtypes = [ctypes.c_uint64, ctypes.c_int, _VP, _VP]
        L.stda_forward.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]
        L.stda_forward_host.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]
        L.stda_device_status.argtypes = [_VP]
        L.stda_set_wait_limit.argtypes = [_VP, ctypes.c_uint32]
        L.stda_last_error.restype = ctypes.c_char_p
        L.stda_last_error.argtypes = [_VP]
        L.stda_backward.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, _VP]
        L.stda_backward_bn.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _VP, _VP]
        L.stda_metrics.argtypes = [_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _VP, _VP, _VP, _VP,
                                   _VP]
        L.stda_submit.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP]
        L.stda_flush.argtypes = [_VP, _VP]
        L.stda_serve_close.argtypes = [_VP, ctypes.c_int, _VP]
        L.stda_serve_bytes.restype = ctypes.c_size_t
        L.stda_serve_bytes.argtypes = [_VP]
        L.stda_serve_radars.restype = ctypes.c_int
        L.stda_serve_radars.argtypes = [_VP]
        L.stda_forward_static.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]
        L.stda_profile.argtypes = [_VP, ctypes.c_int]
        L.stda_profile_read.restype = ctypes.c_int
        L.stda_profile_read.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int]
        L.stda_launch_count.restype = ctypes.c_uint64
        L.stda_launch_count.argtypes = [_VP]
        L.stda_generate.argtypes = [ctypes.POINTER(GenConfig), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]
        _lib = L
    return _lib


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def num_params():
    return int(lib().stda_num_params())


def num_buffers():
    return int(lib().stda_num_buffers())


def init_params(seed=0, frames=3):
    """Host-side: the parameters and BN buffers stda_create draws from a seed
    for a context of `frames` stacked maps per window."""
    p = np.empty(int(lib().stda_num_params_frames(frames)), np.float32)
    b = np.empty(num_buffers(), np.float32)
    st = lib().stda_init_params_frames(seed, frames, p.ctypes.data, b.ctypes.data)
    if st != OK:
        raise StdaError(st)
    return p, b


def reparam_shapes(frames=3):
    """(name, shape) of the re-parameterised inference network, in the order
    of stda_reparam_export (PyTorch Conv2d / ConvTranspose2d / Conv1d
    weight layouts)."""
    cin, enc = (8, 16, 32, 64, 32, 16), (1, 1, 1, 0, 0, 0)
    t = [("stem.weight", (8, frames, 3, 3)), ("stem.bias", (8,))]
    for b in range(6):
        ci = cin[b]
        co = 2 * ci if enc[b] else ci // 2
        conv = (co, ci, 3, 3) if enc[b] else (ci, co, 4, 4)
        t += [(f"blk{b}.dw.weight", (ci, 1, 3, 3)), (f"blk{b}.dw.bias", (ci,)),
              (f"blk{b}.main.weight", conv), (f"blk{b}.main.bias", (co,)),
              (f"blk{b}.res.weight", conv), (f"blk{b}.res.bias", (co,)),
              (f"blk{b}.eca.weight", (1, 1, 3))]
    return t + [("out.weight", (1, 8, 3, 3)), ("out.bias", (1,))]


def reparam_export(params, buffers, frames=3):
    """Host-side: the re-parameterised inference network (every BN folded,
    stage-1 branches merged) as {name: float32 array}, through
    stda_reparam_export."""
    n = int(lib().stda_reparam_count(frames))
    out = np.empty(n, np.float32)
    p = np.ascontiguousarray(params, np.float32)
    b = np.ascontiguousarray(buffers, np.float32)
    st = lib().stda_reparam_export(p.ctypes.data, b.ctypes.data, frames, out.ctypes.data, n)
    if st != OK:
        raise StdaError(st)
    d, off = {}, 0
    for name, shape in reparam_shapes(frames):
        k = int(np.prod(shape))
        d[name] = out[off:off + k].reshape(shape)
        off += k
    assert off == n
    return d


class Context:
    """One libstda context: folded weights and activation scratch on the
    current CUDA device for up to max_batch windows of H x W."""

    def __init__(self, H, W, max_batch, precision="fp32", weight_seed=0, mem_budget_bytes=0, frames=3):
        self.precision = precision
        self.prec = PRECISIONS[precision]
        self.H, self.W, self.max_batch, self.frames = H, W, max_batch, frames
        cfg = Config(H, W, max_batch, self.prec, weight_seed, mem_budget_bytes, frames)
        h = _VP()
        st = lib().stda_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise StdaError(st, lib().stda_status_string(st).decode())
        self.h = h

    @property
    def io_dtype(self):
        import torch

        return torch.float32 if self.prec == FP32 else torch.bfloat16

    def close(self):
        if getattr(self, "h", None):
            lib().stda_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise StdaError(st, lib().stda_last_error(self.h).decode())

    def get_params(self):
        a = np.empty(int(lib().stda_num_params_frames(self.frames)), np.float32)
        self._check(lib().stda_get_params(self.h, a.ctypes.data, a.size))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, np.float32)
        self._check(lib().stda_set_params(self.h, a.ctypes.data, a.size))

    def get_buffers(self):
        a = np.empty(num_buffers(), np.float32)
        self._check(lib().stda_get_buffers(self.h, a.ctypes.data, a.size))
        return a

    def set_buffers(self, a):
        a = np.ascontiguousarray(a, np.float32)
        self._check(lib().stda_set_buffers(self.h, a.ctypes.data, a.size))

    def forward_raw(self, x, out, B, H, W, stream=None):
        """stda_forward on existing device tensors; returns the status."""
        return lib().stda_forward(self.h, _ptr(x), _ptr(out), B, H, W, _stream(stream))

    def forward(self, x, out=None, stream=None):
        """x: CUDA tensor [B][frames][H][W] (float32 for fp32, bfloat16 otherwise)."""
        import torch

        assert x.is_cuda and x.is_contiguous() and x.dtype == self.io_dtype and x.dim() == 4 and x.shape[1] == self.frames
        B, _, H, W = x.shape
        if out is None:
            out = torch.empty((B, 1, H, W), dtype=x.dtype, device=x.device)
        self._check(self.forward_raw(x, out, B, H, W, stream))
        return out

    def forward_host(self, x, out=None, stream=None):
        """stda_forward_host: x a CPU tensor [B][frames][H][W] (pinned for
        overlapped copies) whose contents are final, out a CPU tensor
        [B][1][H][W] (allocated pinned if None), complete once `stream` (the
        current stream if None) is synchronised."""
        import torch

        assert not x.is_cuda and x.is_contiguous() and x.dtype == self.io_dtype and x.dim() == 4
        assert x.shape[1] == self.frames
        B, _, H, W = x.shape
        if out is None:
            out = torch.empty((B, 1, H, W), dtype=x.dtype).pin_memory()
        assert not out.is_cuda and out.is_contiguous() and out.dtype == x.dtype and out.numel() == B * H * W
        self._check(lib().stda_forward_host(self.h, _ptr(x), _ptr(out), B, H, W, _stream(stream)))
        return out

    def backward(self, x, target=None, gout=None, want_gin=False, want_out=False, stream=None):
        """stda_backward: (loss or None, dL/dtheta [137915] float, dL/dx or None,
        z or None) for x [B][3][H][W] and either target [B][1][H][W] (MSE) or
        gout [B][1][H][W] (float dL/dz)."""
        import torch

        B, _, H, W = x.shape
        dev = x.device
        gp = torch.empty(num_params(), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev) if target is not None else None
        gin = torch.empty((B, 3, H, W), dtype=torch.float32, device=dev) if want_gin else None
        out = torch.empty((B, 1, H, W), dtype=torch.float32, device=dev) if want_out else None
        st = lib().stda_backward(self.h, _ptr(x), _ptr(target), _ptr(gout), _ptr(gp), _ptr(loss), _ptr(gin),
                                 _ptr(out), B, H, W, _stream(stream))
        self._check(st)
        return loss, gp, gin, out

    def backward_bn(self, x, target=None, gout=None, mode="batch", stream=None):
        """stda_backward_bn: (loss or None, dL/dtheta [137915] float, BN
        statistics [1360] float) with BN in training mode ("batch": batch
        statistics) or inference form ("running")."""
        import torch

        B, _, H, W = x.shape
        dev = x.device
        gp = torch.empty(num_params(), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev) if target is not None else None
        stats = torch.empty(num_buffers(), dtype=torch.float32, device=dev)
        st = lib().stda_backward_bn(self.h, _ptr(x), _ptr(target), _ptr(gout), _ptr(gp), _ptr(loss), None, None,
                                    B, H, W, {"running": 0, "batch": 1}[mode], _ptr(stats), _stream(stream))
        self._check(st)
        return loss, gp, stats

    # ----------------------------------------------------------- serving
    def submit(self, radar, frame, out, done=None, stream=None):
        """stda_submit: frame / out are bf16 [H][W] CUDA tensors; done an
        optional torch.cuda.Event. Returns the status (OK, WARMUP or BUSY)."""
        H, W = frame.shape[-2:]
        if done is not None and done.cuda_event == 0:
            # torch creates its CUDA event lazily, at the first record: create
            # it here, or the library would receive a null event
            done.record()
        ev = ctypes.c_void_p(done.cuda_event) if done is not None else None
        st = lib().stda_submit(self.h, radar, H, W, _ptr(frame), _ptr(out), ev, _stream(stream))
        if st not in (OK, WARMUP, ERR_BUSY):
            self._check(st)
        return st

    def flush(self, stream=None):
        self._check(lib().stda_flush(self.h, _stream(stream)))

    def serve_close(self, radar, stream=None):
        self._check(lib().stda_serve_close(self.h, radar, _stream(stream)))

    def serve_bytes(self):
        return int(lib().stda_serve_bytes(self.h))

    def serve_radars(self):
        return int(lib().stda_serve_radars(self.h))

    def profile(self, enable=True):
        self._check(lib().stda_profile(self.h, int(enable)))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since the last read."""
        n = 32
        names = (ctypes.c_char_p * n)()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        k = lib().stda_profile_read(self.h, names, ms, cnt, n)
        if k < 0:
            raise StdaError(ERR_CUDA, "profile_read failed")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(k)}

    def launch_count(self):
        return int(lib().stda_launch_count(self.h))

    def device_status(self):
        """The device-side error word (OK or ERR_TIMEOUT), cleared by the read."""
        return lib().stda_device_status(self.h)

    def set_wait_limit(self, polls=1 << 22):
        """Bound of the tensor-core kernels' tile waits (0: give up at once,
        for tests of the timeout path)."""
        self._check(lib().stda_set_wait_limit(self.h, polls))


def forward_static(d_params, d_buffers, x, out=None, stream=None):
    """stda_forward_static: the FP32 forward without a context or any device
    allocation (for callers that cannot allocate); all tensors on the GPU."""
    import torch

    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.dim() == 4 and x.shape[1] == 3
    for t, n in ((d_params, num_params()), (d_buffers, num_buffers())):
        # the library reads exactly n floats from each: anything else is an
        # out-of-bounds device read, so refuse it here
        if not (t.is_cuda and t.device == x.device and t.dtype == torch.float32 and t.is_contiguous()
                and t.numel() == n):
            raise StdaError(ERR_INVALID_ARG, f"forward_static: parameters must be {n} contiguous float32 "
                                             f"values on {x.device}")
    B, _, H, W = x.shape
    if out is None:
        out = torch.empty((B, 1, H, W), dtype=torch.float32, device=x.device)
    st = lib().stda_forward_static(_ptr(d_params), _ptr(d_buffers), _ptr(x), _ptr(out), B, H, W, _stream(stream))
    if st != OK:
        raise StdaError(st, lib().stda_status_string(st).decode())
    return out


def gen_config(g) -> GenConfig:
    return GenConfig(g.N, g.M, g.P, g.Q, g.tmin, g.tmax, g.imin, g.imax, g.snr_min, g.snr_max, g.inr_min,
                     g.inr_max, g.kmin, g.kmax)


def generate(g, seed, cid, w0, B, dtype=None, with_clean=True, device="cuda", stream=None):
    """GPU generator: (noisy [B][3][P][Q], clean [B][1][P][Q] | None, bins [B][16][2], ntgt [B])."""
    import torch

    dtype = dtype or torch.float32
    noisy = torch.empty((B, 3, g.P, g.Q), dtype=dtype, device=device)
    clean = torch.empty((B, 1, g.P, g.Q), dtype=dtype, device=device) if with_clean else None
    bins = torch.empty((B, MAX_TGT, 2), dtype=torch.int32, device=device)
    ntgt = torch.empty((B,), dtype=torch.int32, device=device)
    cfg = gen_config(g)
    st = lib().stda_generate(ctypes.byref(cfg), seed, cid, w0, B, int(dtype == torch.bfloat16), _ptr(noisy),
                             _ptr(clean), _ptr(bins), _ptr(ntgt), _stream(stream))
    if st != OK:
        raise StdaError(st, lib().stda_status_string(st).decode())
    return noisy, clean, bins, ntgt


def _autograd_function():
    import torch

    class STDAFunction(torch.autograd.Function):
        """z = Radar-STDA(x; theta) through libstda: forward on the context's
        kernels, backward with stda_backward (the exact adjoint). `params`
        must hold the context's current parameters (it only routes the
        gradient to the caller's master copy)."""

        @staticmethod
        def forward(fctx, x, params, ctx):
            fctx.save_for_backward(x)
            fctx.stda = ctx
            return ctx.forward(x.contiguous())

        @staticmethod
        def backward(fctx, gout):
            (x,) = fctx.saved_tensors
            _, gp, gin, _ = fctx.stda.backward(x.contiguous(), gout=gout.float().contiguous(),
                                               want_gin=fctx.needs_input_grad[0])
            gx = gin.to(x.dtype) if gin is not None else None
            return gx, gp, None

    return STDAFunction


def stda_apply(x, params, ctx):
    """Differentiable application of the denoiser (see STDAFunction)."""
    return _autograd_function().apply(x, params, ctx)


def metrics(maps, bins, ntgt, clean=None, guard=2, cfar_guard=2, cfar_train=4, pfa=1e-3, want_det=False,
            stream=None):
    """stda_metrics on CUDA tensors maps / clean [B][(1)][H][W] (float or
    bf16), bins [B][16][2], ntgt [B]: (sinr [B] f64, evm [B] f64 | None,
    detection rate [B] f32, detections [B][H][W] u8 | None)."""
    import torch

    B, H, W = maps.shape[0], maps.shape[-2], maps.shape[-1]
    dev = maps.device
    bf16 = int(maps.dtype == torch.bfloat16)
    sinr = torch.empty(B, dtype=torch.float64, device=dev)
    evm = torch.empty(B, dtype=torch.float64, device=dev) if clean is not None else None
    rate = torch.empty(B, dtype=torch.float32, device=dev)
    det = torch.empty((B, H, W), dtype=torch.uint8, device=dev) if want_det else None
    st = lib().stda_metrics(_ptr(maps), _ptr(clean), bf16, _ptr(bins), _ptr(ntgt), B, H, W, guard, cfar_guard,
                            cfar_train, pfa, _ptr(sinr), _ptr(evm), _ptr(rate), _ptr(det), _stream(stream))
    if st != OK:
        raise StdaError(st, lib().stda_status_string(st).decode())
    return sinr, evm, rate, det
