"""FP64 CPU oracle for Noise2Fast (arXiv 2108.10209) -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``oracle/liboracle.so`` (plain C, see ``oracle.c``). Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this package;
the library under ``paper_2108_10209_gb300`` never does, and the two share no code.

Arrays are float64 numpy arrays in NCHW order; 3x3 weights are [C_out][C_in][3][3].
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

LAYERS = 8
# Methods, first paragraph: 32, 32, then three doublings of a pair of layers.
WIDTHS_PLIT = (32, 32, 64, 64, 128, 128, 256, 256)
# The constant-64 reading of the same paragraph (kept beside the literal one).
WIDTHS_W64 = (64,) * 8

THETA, GRAD, ADAM_M, ADAM_V, ACT, DELTA, Z, DZ, PAIR_IN, PAIR_TGT, SUM, VBEST = range(12)

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    """Loads (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_splitmix64_at.restype = C.c_uint64
        L.orc_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_param_count.restype = C.c_size_t
        L.orc_param_count.argtypes = [C.POINTER(C.c_int)]
        L.orc_param_count_c.restype = C.c_size_t
        L.orc_param_count_c.argtypes = [C.POINTER(C.c_int), C.c_int]
        L.orc_init_params_c.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_uint64, _dp]
        L.orc_net_forward_c.argtypes = [C.POINTER(C.c_int), C.c_int, _dp, _dp, C.c_int, C.c_int,
                                        C.c_void_p, C.c_void_p]
        L.orc_init_params.argtypes = [C.POINTER(C.c_int), C.c_uint64, _dp]
        L.orc_checker.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_conv3x3_fwd.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_int, _dp]
        L.orc_conv3x3_dgrad.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, C.c_int, _dp]
        L.orc_conv3x3_wgrad.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp]
        L.orc_head_fwd.argtypes = [_dp, C.c_int, C.c_int, _dp, C.c_double, _dp]
        L.orc_sigmoid.restype = C.c_double
        L.orc_sigmoid.argtypes = [C.c_double]
        L.orc_loss.restype = C.c_double
        L.orc_loss.argtypes = [_dp, _dp, C.c_int, C.c_int, _dp]
        L.orc_adam.argtypes = [_dp, _dp, _dp, _dp, C.c_size_t, C.c_long, C.c_double, C.c_double,
                               C.c_double, C.c_double]
        L.orc_stop_init.argtypes = [C.c_void_p]
        L.orc_threads.restype = C.c_int
        L.orc_threads.argtypes = []
        L.orc_stop_update.restype = C.c_int
        L.orc_stop_update.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int]
        L.orc_job_new.restype = C.c_void_p
        L.orc_job_new.argtypes = [_dp, C.c_int, C.c_int, C.c_void_p]
        L.orc_job_set_theta.argtypes = [C.c_void_p, _dp]
        L.orc_job_step.restype = C.c_double
        L.orc_job_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_job_validate.restype = C.c_double
        L.orc_job_validate.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_job_epoch.restype = C.c_double
        L.orc_job_epoch.argtypes = [C.c_void_p]
        L.orc_job_run.argtypes = [C.c_void_p, _dp]
        L.orc_job_get.restype = C.c_size_t
        L.orc_job_get.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.orc_job_info.argtypes = [C.c_void_p] + [C.c_void_p] * 8
        L.orc_job_free.argtypes = [C.c_void_p]
        L.orc_net_forward.argtypes = [C.POINTER(C.c_int), _dp, _dp, C.c_int, C.c_int, C.c_void_p,
                                      C.c_void_p]
        L.orc_max_project.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp]
        L.orc_quad.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _widths(w):
    w = tuple(int(v) for v in w)
    assert len(w) == LAYERS
    return (C.c_int * LAYERS)(*w)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def splitmix64_at(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64_at(seed, k))


def param_count(widths=WIDTHS_PLIT, channels: int = 1) -> int:
    return int(lib().orc_param_count_c(_widths(widths), max(1, channels)))


def init_params(widths=WIDTHS_PLIT, seed: int = 0, channels: int = 1) -> np.ndarray:
    th = np.zeros(param_count(widths, channels), np.float64)
    lib().orc_init_params_c(_widths(widths), max(1, channels), seed, th)
    return th


def unpack(widths, theta, channels: int = 1):
    """Splits a flat parameter vector into [(W_l, b_l)] * 8 + [(w_head, b_head)] views."""
    out, off, cin = [], 0, max(1, channels)
    for cout in widths:
        n = cout * cin * 9
        out.append((theta[off:off + n].reshape(cout, cin, 3, 3), theta[off + n:off + n + cout]))
        off += n + cout
        cin = cout
    out.append((theta[off:off + cin], theta[off + cin:off + cin + 1]))
    assert off + cin + 1 == theta.size
    return out


def checker(x):
    x = _f64(x)
    H, W = x.shape
    up_e = np.zeros((H, W // 2)); up_o = np.zeros((H, W // 2))
    lf_e = np.zeros((H // 2, W)); lf_o = np.zeros((H // 2, W))
    lib().orc_checker(x, H, W, up_e, up_o, lf_e, lf_o)
    return up_e, up_o, lf_e, lf_o


def quad(x):
    """Ablation Study's Quad downsampling: (TL, TR, BL, BR), each floor(H/2) x floor(W/2)."""
    x = _f64(x)
    H, W = x.shape
    outs = [np.zeros((H // 2, W // 2)) for _ in range(4)]
    lib().orc_quad(x, H, W, *outs)
    return tuple(outs)


def conv3x3_fwd(inp, wt, b, relu=True):
    inp, wt, b = _f64(inp), _f64(wt), _f64(b)
    cin, h, w = inp.shape
    cout = wt.shape[0]
    assert wt.shape == (cout, cin, 3, 3) and b.shape == (cout,)
    out = np.zeros((cout, h, w))
    lib().orc_conv3x3_fwd(inp, cin, h, w, wt, b, cout, int(relu), out)
    return out


def conv3x3_dgrad(dout, wt):
    dout, wt = _f64(dout), _f64(wt)
    cout, h, w = dout.shape
    cin = wt.shape[1]
    din = np.zeros((cin, h, w))
    lib().orc_conv3x3_dgrad(dout, cout, h, w, wt, cin, din)
    return din


def conv3x3_wgrad(dout, inp):
    dout, inp = _f64(dout), _f64(inp)
    cout, h, w = dout.shape
    cin = inp.shape[0]
    dw = np.zeros((cout, cin, 3, 3)); db = np.zeros(cout)
    lib().orc_conv3x3_wgrad(dout, cout, h, w, inp, cin, dw, db)
    return dw, db


def head_fwd(a, w, b):
    a, w = _f64(a), _f64(w)
    c, h, ww = a.shape
    z = np.zeros((h, ww))
    lib().orc_head_fwd(a, c, h * ww, w, float(b), z)
    return z


def sigmoid(z: float) -> float:
    return float(lib().orc_sigmoid(z))


def loss(z, y, kind=0):
    z, y = _f64(z), _f64(y)
    dz = np.zeros_like(z)
    L = lib().orc_loss(z, y, z.size, kind, dz)
    return float(L), dz


def adam(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    for a in (theta, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(theta, g, m, v, theta.size, t, lr, b1, b2, eps)


class _Stop(C.Structure):
    _fields_ = [("best", C.c_double), ("since", C.c_int), ("epoch", C.c_int), ("stopped", C.c_int)]


class StopRule:
    """The paper's patience rule: see ``orc_stop_update``."""

    def __init__(self, patience=100, incl_best=False):
        self.s = _Stop()
        self.patience, self.incl_best = patience, int(incl_best)
        lib().orc_stop_init(C.byref(self.s))

    def update(self, score: float) -> bool:
        return bool(lib().orc_stop_update(C.byref(self.s), score, self.patience, self.incl_best))

    @property
    def stopped(self):
        return bool(self.s.stopped)

    @property
    def since(self):
        return self.s.since

    @property
    def epoch(self):
        return self.s.epoch

    @property
    def best(self):
        return self.s.best


class _Params(C.Structure):
    _fields_ = [("widths", C.c_int * LAYERS), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("patience", C.c_int),
                ("max_epochs", C.c_int), ("fixed_steps", C.c_int), ("loss_kind", C.c_int),
                ("incl_best", C.c_int), ("seed", C.c_uint64), ("channels", C.c_int),
                ("target", C.c_int), ("downsample", C.c_int), ("exact", C.c_int)]


@dataclasses.dataclass
class Params:
    widths: tuple = WIDTHS_PLIT
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    patience: int = 100
    max_epochs: int = 0
    fixed_steps: int = -1
    loss_kind: int = 0
    incl_best: bool = False
    seed: int = 0

    channels: int = 1   # input channels C_0 (Fig. 2a caption: inputs may be multi-channel)
    target: int = 0     # the predicted channel (one output channel per network)
    downsample: int = 0  # 0 checkerboard, 1 Quad (Ablation Study)
    exact: bool = False  # Exact (Ablation Study): x carries the clean target plane last

    def _c(self):
        return _Params(_widths(self.widths), self.lr, self.beta1, self.beta2, self.eps,
                       self.patience, self.max_epochs, self.fixed_steps, self.loss_kind,
                       int(self.incl_best), self.seed, self.channels, self.target,
                       self.downsample, int(self.exact))


class Job:
    """One image's whole Noise2Fast run, stepped from Python."""

    def __init__(self, x, params: Params = Params()):
        """x: (H, W), or (C_0, H, W) planes when params.channels = C_0 > 1."""
        x = _f64(x)
        if x.ndim == 2:
            x = x[None]
        c0 = max(1, params.channels)
        assert x.shape[0] == c0 + int(params.exact) and 0 <= params.target < c0
        _, self.H, self.W = x.shape
        x = np.ascontiguousarray(x)
        self.params = params
        self._p = params._c()
        self.h = lib().orc_job_new(x, self.H, self.W, C.byref(self._p))
        self.np = param_count(params.widths, params.channels)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_job_free(self.h)
            self.h = None

    def set_theta(self, theta):
        theta = _f64(theta)
        assert theta.size == self.np
        lib().orc_job_set_theta(self.h, theta)

    def step(self, pair: int) -> float:
        return float(lib().orc_job_step(self.h, pair))

    def validate(self):
        v = np.zeros((self.H, self.W))
        s = lib().orc_job_validate(self.h, v.ctypes.data)
        return float(s), v

    def epoch(self) -> float:
        return float(lib().orc_job_epoch(self.h))

    def run(self):
        out = np.zeros((self.H, self.W))
        lib().orc_job_run(self.h, out)
        return out

    def get(self, what: int, layer: int = 0) -> np.ndarray:
        n = lib().orc_job_get(self.h, what, layer, None)
        out = np.zeros(n)
        lib().orc_job_get(self.h, what, layer, out.ctypes.data)
        return out

    def info(self) -> dict:
        t = C.c_long(); ep = C.c_int(); since = C.c_int(); stopped = C.c_int(); capped = C.c_int()
        best = C.c_double(); last = C.c_double(); dims = (C.c_int * 4)()
        lib().orc_job_info(self.h, C.byref(t), C.byref(ep), C.byref(since), C.byref(stopped),
                           C.byref(capped), C.byref(best), C.byref(last), dims)
        return dict(t=t.value, epoch=ep.value, since=since.value, stopped=bool(stopped.value),
                    capped=bool(capped.value), best=best.value, last_loss=last.value,
                    dims=tuple(dims))


def net_forward(widths, theta, img):
    """img: (h, w), or (C_0, h, w) planes."""
    img = _f64(img)
    if img.ndim == 2:
        img = img[None]
    c0, h, w = img.shape
    img = np.ascontiguousarray(img)
    v = np.zeros((h, w)); z = np.zeros((h, w))
    lib().orc_net_forward_c(_widths(widths), c0, _f64(theta), img, h, w, v.ctypes.data,
                            z.ctypes.data)
    return v, z


def denoise_channels(x, params: Params = Params()):
    """A multi-channel image (C, H, W) the way Fig. 2a's caption describes RGB: every channel
    predicted by its own network that sees all C input channels. Returns (C, H, W)."""
    x = _f64(x)
    c0 = x.shape[0]
    return np.stack([denoise(x, dataclasses.replace(params, channels=c0, target=t))[0]
                     for t in range(c0)])


def denoise(x, params: Params = Params()):
    """The whole procedure on one image; returns (output, info)."""
    j = Job(x, params)
    out = j.run()
    return out, j.info()


def threads() -> int:
    """Threads the oracle's parallel loops use (OMP_NUM_THREADS as read when it was loaded)."""
    return int(lib().orc_threads())


def max_project(vol):
    """Maximum projection along Z of a (Z, H, W) volume (Methods, fluorescence microscopy)."""
    vol = _f64(vol)
    Z, H, W = vol.shape
    out = np.zeros((H, W))
    lib().orc_max_project(vol, Z, H, W, out)
    return out


def denoise_stack(vol, params: Params = Params()):
    """A Z-stack as the paper processes one: every slice denoised as its own image with the same
    parameters, then max projected. Returns (denoised slices, projection)."""
    outs = np.stack([denoise(np.asarray(s), params)[0] for s in vol])
    return outs, max_project(outs)
