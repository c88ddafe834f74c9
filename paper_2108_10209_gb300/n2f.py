"""Python binding of the C ABI in ``include/n2f.h`` (ctypes; argument marshalling only).

Every step of the denoising path runs in ``libn2f.so``; this module only converts Python
arguments (numpy arrays, torch CUDA tensors, streams) into the plain pointers and sizes the
C functions take. If the library has not been built, importing this module raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# N2F_LIBRARY=checked loads the checked build (libn2f_checked.so: bounds-checked kernel indexes,
# see n2f_check_status); anything else, or unset, the normal library
LIB_PATH = os.path.join(_HERE, "libn2f_checked.so" if os.environ.get("N2F_LIBRARY") == "checked"
                        else "libn2f.so")

N2F_OK, N2F_EINVAL, N2F_ETOOBIG, N2F_EAGAIN, N2F_ENOENT = 0, -1, -2, -3, -4
N2F_ETIMEDOUT, N2F_ENONFINITE, N2F_EDEVICE, N2F_ENOMEM, N2F_ECANCELED, N2F_ENOTSUP = (
    -5, -6, -7, -8, -9, -10)
N2F_FP32, N2F_BF16 = 0, 1
N2F_LOSS_BCE, N2F_LOSS_MSE = 0, 1
N2F_WIDTHS_PLIT, N2F_WIDTHS_W64 = 0, 1
N2F_ENGINE_AUTO, N2F_ENGINE_SIMT, N2F_ENGINE_TC = 0, 1, 2
N2F_DOWN_CHECKER, N2F_DOWN_QUAD = 0, 1
N2F_QUEUED, N2F_RUNNING, N2F_DONE, N2F_FAILED, N2F_CANCELED = range(5)
(N2F_X_THETA, N2F_X_GRAD, N2F_X_ADAM_M, N2F_X_ADAM_V, N2F_X_ACT, N2F_X_DELTA) = range(6)
N2F_X_DZ, N2F_X_PAIR, N2F_X_VAL, N2F_X_SUM, N2F_X_OUT, N2F_X_HIST, N2F_X_VBEST = (
    7, 8, 9, 10, 11, 12, 13)
N2F_HIST_CAP = 4096
(N2F_K_NONE, N2F_K_CONV_FWD, N2F_K_CONV_DGRAD, N2F_K_CONV_WGRAD, N2F_K_FIRST, N2F_K_HEAD,
 N2F_K_ADAM, N2F_K_CONV) = range(8)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("device", C.c_int), ("hbm_budget_bytes", C.c_uint64),
                ("max_slots", C.c_uint32), ("lookahead", C.c_uint32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p), ("profile_kernel", C.c_int32),
                ("use_graphs", C.c_int32), ("group_size", C.c_uint32), ("autotune", C.c_int32),
                ("profile_every", C.c_uint32)]


class Params(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("patience", C.c_uint32),
                ("max_epochs", C.c_uint32), ("fixed_steps", C.c_int32), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("loss", C.c_int32), ("widths", C.c_int32),
                ("incl_best", C.c_int32), ("engine", C.c_int32), ("channels", C.c_int32),
                ("target_channel", C.c_int32), ("downsample", C.c_int32), ("exact", C.c_int32),
                ("overlap", C.c_int32)]


class Status(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("state", C.c_int32), ("error", C.c_int32),
                ("epoch", C.c_uint32), ("steps", C.c_uint32), ("since", C.c_uint32),
                ("stopped", C.c_uint32), ("H", C.c_uint32), ("W", C.c_uint32),
                ("best_mse", C.c_double), ("last_mse", C.c_double), ("last_loss", C.c_double), ("device_ms", C.c_double),
                ("compute_ms", C.c_double), ("latency_ms", C.c_double), ("t_start_ms", C.c_double),
                ("t_done_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "struct_size"}


class CtxStats(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kernel_launches", C.c_uint64),
                ("bytes_resident", C.c_uint64), ("jobs_queued", C.c_uint32),
                ("jobs_running", C.c_uint32), ("jobs_done", C.c_uint32),
                ("prof_launches", C.c_uint64), ("prof_ms", C.c_double), ("prof_flops", C.c_double),
                ("prof_bytes", C.c_double)]


# name -> (restype, argtypes); the exported C ABI, one line per function of include/n2f.h
_P, _I, _Z, _U64, _D = C.c_void_p, C.c_int, C.c_size_t, C.c_uint64, C.c_double
SIGNATURES = {
    "n2f_config_default": (None, [C.POINTER(Config)]),
    "n2f_params_default": (None, [C.POINTER(Params)]),
    "n2f_strerror": (C.c_char_p, [_I]),
    "n2f_create": (_I, [C.POINTER(_P), C.POINTER(Config)]),
    "n2f_destroy": (None, [_P]),
    "n2f_submit": (_I, [_P, _P, _I, _I, C.POINTER(Params), C.POINTER(_U64)]),
    "n2f_submit_device": (_I, [_P, _P, _I, _I, C.POINTER(Params), C.POINTER(_U64)]),
    "n2f_submit_u16": (_I, [_P, _P, _I, _I, C.POINTER(Params), C.POINTER(_U64)]),
    "n2f_job_bytes": (_I, [_I, _I, C.POINTER(Params), C.POINTER(_U64)]),
    "n2f_poll": (_I, [_P, _U64, C.POINTER(Status)]),
    "n2f_wait": (_I, [_P, _U64, _I]),
    "n2f_result": (_I, [_P, _U64, _P, _Z]),
    "n2f_result_device": (_I, [_P, _U64, _P, _Z]),
    "n2f_cancel": (_I, [_P, _U64]),
    "n2f_history": (_I, [_P, _U64, _P, _Z, C.POINTER(_Z), C.POINTER(C.c_uint32)]),
    "n2f_stats": (_I, [_P, C.POINTER(CtxStats)]),
    "n2f_trainer_create": (_I, [C.POINTER(_P), _P, _I, _I, C.POINTER(Params), _P]),
    "n2f_trainer_destroy": (None, [_P]),
    "n2f_trainer_step": (_I, [_P, _I]),
    "n2f_trainer_validate": (_I, [_P]),
    "n2f_trainer_epoch": (_I, [_P]),
    "n2f_trainer_run": (_I, [_P, _I]),
    "n2f_trainer_finish": (_I, [_P]),
    "n2f_trainer_set_theta": (_I, [_P, _P, _Z]),
    "n2f_trainer_export": (_I, [_P, _I, _I, _P, _Z, C.POINTER(_Z)]),
    "n2f_trainer_status": (_I, [_P, C.POINTER(Status)]),
    "n2f_trainer_launches": (_U64, [_P]),
    "n2f_trainer_import": (_I, [_P, _I, _I, _P, _Z]),
    "n2f_trainer_set_progress": (_I, [_P, C.c_uint32, C.c_uint32, C.c_uint32, _D]),
    "n2f_param_count": (_Z, [_I]),
    "n2f_checker_gather": (_I, [_P, _I, _I, _P, _P, _P, _P, _P]),
    "n2f_max_project": (_I, [_P, _I, _I, _I, _P, _P]),
    "n2f_pack_cg": (_I, [_P, _I, _I, _I, _I, _P, _P]),
    "n2f_unpack_cg": (_I, [_P, _I, _I, _I, _I, _P, _P]),
    "n2f_conv3x3": (_I, [_I, _I, _I, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P]),
    "n2f_conv3x3_wgrad": (_I, [_I, _I, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "n2f_conv3x3_wgrad_noalloc": (_I, [_I, _I, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "n2f_umma_gemm": (_I, [_I, _I, _I, _I, _I, _P, _Z, C.c_uint32, C.c_uint32, C.c_uint32, _P, _Z,
                           C.c_uint32, C.c_uint32, C.c_uint32, _P, _P]),
    "n2f_wait_probe": (_I, [C.c_uint32, _P]),
    "n2f_check_status": (_I, [C.POINTER(_U64), C.POINTER(_I), _I]),
}

_lib = None


def lib():
    """Loads ``libn2f.so``; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class N2FError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().n2f_strerror(code)
        super().__init__(f"{where}: {code} ({msg.decode() if msg else '?'})")


def check(code, where=""):
    if code != N2F_OK:
        raise N2FError(code, where)
    return code


def params(**kw) -> Params:
    p = Params()
    lib().n2f_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def job_bytes(H: int, W: int, p: Params | None = None) -> int:
    """Device bytes a job holds while admitted (``n2f_job_bytes``): what the context counts
    against its HBM budget."""
    n = C.c_uint64()
    check(lib().n2f_job_bytes(H, W, C.byref(p) if p else None, C.byref(n)), "n2f_job_bytes")
    return int(n.value)


def param_count(widths=N2F_WIDTHS_PLIT) -> int:
    return int(lib().n2f_param_count(widths))


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return C.c_void_p(t.data_ptr())


# ---- job API ---------------------------------------------------------------------------------

def image_planes(p: Params | None) -> int:
    """Planes of H x W floats a submitted image holds: the input channels (0 means 1), plus the
    clean plane of the Exact ablation."""
    if p is None:
        return 1
    return max(1, int(p.channels)) + (1 if p.exact else 0)


def _check_device_image(dimage, p: Params | None, device: int):
    """n2f_submit_device takes no element count: the library copies image_planes(p) * H * W
    floats from the pointer. Raises ValueError unless dimage is a contiguous float32 tensor of
    exactly that many elements (shape (H, W) or (planes, H, W)) on the context's device."""
    import torch
    if not isinstance(dimage, torch.Tensor):
        raise ValueError("dimage: a torch tensor is required")
    if dimage.dtype != torch.float32:
        raise ValueError(f"dimage: dtype {dimage.dtype}, torch.float32 required")
    if dimage.dim() not in (2, 3):
        raise ValueError(f"dimage: shape {tuple(dimage.shape)}, (H, W) or (planes, H, W) required")
    H, W = dimage.shape[-2:]
    need = image_planes(p) * H * W
    if dimage.numel() != need:
        raise ValueError(f"dimage: {dimage.numel()} elements, {need} required "
                         f"({image_planes(p)} planes of {H} x {W})")
    if not dimage.is_contiguous():
        raise ValueError("dimage: must be contiguous")
    if dimage.device.type != "cuda" or dimage.device.index != device:
        raise ValueError(f"dimage: on {dimage.device}, cuda:{device} required")


class Context:
    """A scheduler context (``n2f_create``); device memory comes from torch's caching allocator
    unless ``torch_alloc=False`` (then the library calls cudaMalloc itself)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_slots: int = 0,
                 lookahead: int = 0, torch_alloc: bool = True, profile_kernel: int = 0,
                 use_graphs: bool = True, group_size: int = 0, autotune: bool = False,
                 profile_every: int = 0):
        cfg = Config()
        lib().n2f_config_default(C.byref(cfg))
        cfg.device = device
        if hbm_budget_bytes:
            cfg.hbm_budget_bytes = hbm_budget_bytes
        if max_slots:
            cfg.max_slots = max_slots
        if lookahead:
            cfg.lookahead = lookahead
        cfg.profile_kernel = profile_kernel
        cfg.use_graphs = int(use_graphs)
        cfg.group_size = group_size
        cfg.autotune = int(autotune)
        cfg.profile_every = profile_every
        self.device = device
        self._keep = []
        self._dev_inputs = {}  # job -> device image tensor, held until the job is collected
        if torch_alloc:
            import torch

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device=device)
                except Exception:
                    return None

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [a, f]
            cfg.alloc, cfg.free = a, f
        self.h = C.c_void_p()
        check(lib().n2f_create(C.byref(self.h), C.byref(cfg)), "n2f_create")

    def close(self):
        if getattr(self, "h", None):
            lib().n2f_destroy(self.h)
            self.h = None
            self._dev_inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, image: np.ndarray, p: Params | None = None) -> int:
        """image: (H, W), or (planes, H, W): the p.channels input planes, then the clean plane
        when p.exact (Ablation Study)."""
        img = np.ascontiguousarray(image, dtype=np.float32)
        H, W = img.shape[-2:]
        job = C.c_uint64()
        check(lib().n2f_submit(self.h, img.ctypes.data_as(C.c_void_p), H, W,
                               C.byref(p) if p else None, C.byref(job)), "n2f_submit")
        return job.value

    def submit_u16(self, image: np.ndarray, p: Params | None = None) -> int:
        img = np.ascontiguousarray(image, dtype=np.uint16)
        H, W = img.shape
        job = C.c_uint64()
        check(lib().n2f_submit_u16(self.h, img.ctypes.data_as(C.c_void_p), H, W,
                                   C.byref(p) if p else None, C.byref(job)), "n2f_submit_u16")
        return job.value

    def submit_device(self, dimage, p: Params | None = None) -> int:
        """dimage: a contiguous float32 CUDA tensor (H, W), or (planes, H, W). The library copies
        it on the job's own stream once the job is admitted, with no ordering against torch's
        streams: torch's current stream on that device is synchronised here (a tensor written on
        another stream needs that stream synchronised first), and the tensor is held, and must
        not be written, until the job's result is collected."""
        import torch
        H, W = dimage.shape[-2:]
        _check_device_image(dimage, p, self.device)
        torch.cuda.current_stream(dimage.device).synchronize()
        job = C.c_uint64()
        check(lib().n2f_submit_device(self.h, _ptr(dimage), H, W, C.byref(p) if p else None,
                                      C.byref(job)), "n2f_submit_device")
        self._dev_inputs[job.value] = dimage
        return job.value

    def poll(self, job: int) -> Status:
        st = Status()
        st.struct_size = C.sizeof(Status)
        check(lib().n2f_poll(self.h, job, C.byref(st)), "n2f_poll")
        if st.state >= N2F_DONE:
            # a final state: the library no longer reads a device input of this job
            self._dev_inputs.pop(job, None)
        return st

    def wait(self, job: int, timeout_ms: int = -1) -> int:
        rc = lib().n2f_wait(self.h, job, timeout_ms)
        if rc == N2F_OK:
            self._dev_inputs.pop(job, None)
        return rc

    def _collected(self, job: int, rc: int) -> int:
        # any other outcome means the job reached a final state (its copy of the input is done)
        if rc not in (N2F_EAGAIN, N2F_EINVAL):
            self._dev_inputs.pop(job, None)
        return rc

    def result(self, job: int, shape) -> np.ndarray:
        out = np.empty(shape, np.float32)
        rc = lib().n2f_result(self.h, job, out.ctypes.data_as(C.c_void_p), out.size)
        check(self._collected(job, rc), "n2f_result")
        return out

    def result_device(self, job: int, dout) -> None:
        rc = lib().n2f_result_device(self.h, job, _ptr(dout), dout.numel())
        check(self._collected(job, rc), "n2f_result_device")

    def history(self, job: int):
        """The job's validation scores, one per epoch (``n2f_history``): returns (scores as a
        float64 array, 1-based epoch of the first score). Available once the job is DONE and
        until its result is collected."""
        n, first = C.c_size_t(), C.c_uint32()
        check(lib().n2f_history(self.h, job, None, 0, C.byref(n), C.byref(first)), "n2f_history")
        out = np.empty(n.value, np.float64)
        check(lib().n2f_history(self.h, job, out.ctypes.data_as(C.c_void_p), out.size,
                                C.byref(n), C.byref(first)), "n2f_history")
        return out, int(first.value)

    def cancel(self, job: int) -> int:
        """Cancels the job; its device input (submit_device) is released by the next poll or
        wait that sees it final, or when the context closes."""
        return lib().n2f_cancel(self.h, job)

    def stats(self) -> dict:
        st = CtxStats()
        st.struct_size = C.sizeof(CtxStats)
        check(lib().n2f_stats(self.h, C.byref(st)), "n2f_stats")
        return {k: getattr(st, k) for k, _ in st._fields_ if k != "struct_size"}


def denoise(image: np.ndarray, p: Params | None = None, ctx: Context | None = None) -> np.ndarray:
    """One image through the whole path (submit, wait, result); (H, W), or (C_0, H, W) planes
    with p.channels = C_0 (the result is the predicted plane, (H, W))."""
    own = ctx is None
    ctx = ctx or Context()
    try:
        j = ctx.submit(image, p)
        ctx.wait(j)
        return ctx.result(j, image.shape[-2:])
    finally:
        if own:
            ctx.close()


def denoise_channels(image: np.ndarray, p: Params | None = None,
                     ctx: Context | None = None) -> np.ndarray:
    """A multi-channel image (C, H, W), e.g. RGB, the way Fig. 2a's caption describes it: one
    network per output channel, each seeing all C input channels. The C jobs run concurrently.
    Returns (C, H, W)."""
    own = ctx is None
    ctx = ctx or Context()
    try:
        c0 = image.shape[0]
        base = p if p is not None else params()
        jobs = []
        for t in range(c0):
            q = Params.from_buffer_copy(base)
            q.channels, q.target_channel = c0, t
            jobs.append(ctx.submit(image, q))
        outs = []
        for j in jobs:
            ctx.wait(j)
            outs.append(ctx.result(j, image.shape[-2:]))
        return np.stack(outs)
    finally:
        if own:
            ctx.close()


# ---- trainer API -----------------------------------------------------------------------------

class Trainer:
    """One job's device state stepped from Python (``n2f_trainer_*``)."""

    def __init__(self, image: np.ndarray, p: Params | None = None, stream=None):
        img = np.ascontiguousarray(image, dtype=np.float32)
        self.H, self.W = img.shape[-2:]
        self.h = C.c_void_p()
        check(lib().n2f_trainer_create(C.byref(self.h), img.ctypes.data_as(C.c_void_p), self.H,
                                       self.W, C.byref(p) if p else None,
                                       _stream_ptr(stream) if stream is not False else None),
              "n2f_trainer_create")

    def close(self):
        if getattr(self, "h", None):
            lib().n2f_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, pair: int):
        check(lib().n2f_trainer_step(self.h, pair), "n2f_trainer_step")

    def validate(self):
        check(lib().n2f_trainer_validate(self.h), "n2f_trainer_validate")

    def epoch(self):
        check(lib().n2f_trainer_epoch(self.h), "n2f_trainer_epoch")

    def run(self, max_epochs: int = 0):
        check(lib().n2f_trainer_run(self.h, max_epochs), "n2f_trainer_run")

    def finish(self):
        check(lib().n2f_trainer_finish(self.h), "n2f_trainer_finish")

    def set_theta(self, theta: np.ndarray):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        check(lib().n2f_trainer_set_theta(self.h, th.ctypes.data_as(C.c_void_p), th.size),
              "n2f_trainer_set_theta")

    def export(self, what: int, index: int = 0) -> np.ndarray:
        n = C.c_size_t()
        check(lib().n2f_trainer_export(self.h, what, index, None, 0, C.byref(n)), "export size")
        out = np.empty(n.value, np.float64)
        check(lib().n2f_trainer_export(self.h, what, index, out.ctypes.data_as(C.c_void_p),
                                       out.size, C.byref(n)), "n2f_trainer_export")
        return out

    def status(self) -> Status:
        st = Status()
        st.struct_size = C.sizeof(Status)
        check(lib().n2f_trainer_status(self.h, C.byref(st)), "n2f_trainer_status")
        return st

    def import_(self, what: int, values: np.ndarray):
        """Loads THETA, ADAM_M, ADAM_V, SUM or VBEST from host values (``n2f_trainer_import``)."""
        a = np.ascontiguousarray(values, dtype=np.float64).ravel()
        check(lib().n2f_trainer_import(self.h, what, 0, a.ctypes.data_as(C.c_void_p), a.size),
              "n2f_trainer_import")

    def set_progress(self, steps: int, epoch: int, since: int, best: float):
        """Adam step count and stopping-rule counters (``n2f_trainer_set_progress``)."""
        check(lib().n2f_trainer_set_progress(self.h, steps, epoch, since, float(best)),
              "n2f_trainer_set_progress")

    def launches(self) -> int:
        return int(lib().n2f_trainer_launches(self.h))


# ---- op-level entry points (torch CUDA tensors in, on the current stream) --------------------

def checker_gather(x, stream=None):
    import torch
    H, W = x.shape
    ue = torch.empty((H, W // 2), dtype=torch.float32, device=x.device)
    uo = torch.empty_like(ue)
    le = torch.empty((H // 2, W), dtype=torch.float32, device=x.device)
    lo = torch.empty_like(le)
    check(lib().n2f_checker_gather(_ptr(x), H, W, _ptr(ue), _ptr(uo), _ptr(le), _ptr(lo),
                                   _stream_ptr(stream)), "n2f_checker_gather")
    return ue, uo, le, lo


def max_project(vol, stream=None):
    """Maximum projection along Z of a contiguous float32 CUDA tensor (Z, H, W) (n2f_max_project)."""
    import torch
    Z, H, W = vol.shape
    out = torch.empty((H, W), dtype=torch.float32, device=vol.device)
    check(lib().n2f_max_project(_ptr(vol), Z, H, W, _ptr(out), _stream_ptr(stream)),
          "n2f_max_project")
    return out


def denoise_stack(vol: np.ndarray, p: Params | None = None, ctx: Context | None = None):
    """A Z-stack the way the paper processes one (Methods, fluorescence microscopy): every slice
    is submitted as its own job (all in flight at once, admitted by the context's budget), the
    denoised slices are gathered on the device and max projected there. Returns the slices
    (Z, H, W) and the projection (H, W) as float32 CUDA tensors on the context's device."""
    import torch
    own = ctx is None
    ctx = ctx or Context()
    try:
        Z, H, W = vol.shape
        dev = torch.device("cuda", ctx.device)
        jobs = [ctx.submit(np.ascontiguousarray(vol[z], dtype=np.float32), p) for z in range(Z)]
        slices = torch.empty((Z, H, W), dtype=torch.float32, device=dev)
        for z, j in enumerate(jobs):
            ctx.wait(j)
            ctx.result_device(j, slices[z])
        with torch.cuda.device(dev):
            proj = max_project(slices)
            torch.cuda.current_stream(dev).synchronize()
        return slices, proj
    finally:
        if own:
            ctx.close()


def pack_cg(nchw, precision=N2F_FP32, stream=None):
    import torch
    Cc, H, W = nchw.shape
    es = 2 if precision == N2F_BF16 else 4
    out = torch.empty(Cc * H * W * es, dtype=torch.uint8, device=nchw.device)
    check(lib().n2f_pack_cg(_ptr(nchw), Cc, H, W, precision, _ptr(out), _stream_ptr(stream)),
          "n2f_pack_cg")
    return out


def unpack_cg(cg, Cc, H, W, precision=N2F_FP32, stream=None):
    import torch
    out = torch.empty((Cc, H, W), dtype=torch.float32, device=cg.device)
    check(lib().n2f_unpack_cg(_ptr(cg), Cc, H, W, precision, _ptr(out), _stream_ptr(stream)),
          "n2f_unpack_cg")
    return out


def conv3x3(mode, inp_cg, cin, cout, H, W, w, b=None, mask_cg=None, precision=N2F_FP32,
            engine=N2F_ENGINE_AUTO, stream=None):
    """mode 0: forward (returns C_out CG map); mode 1: dgrad (inp has C_out, returns C_in)."""
    import torch
    es = 2 if precision == N2F_BF16 else 4
    cres = cout if mode == 0 else cin
    out = torch.empty(cres * H * W * es, dtype=torch.uint8, device=inp_cg.device)
    check(lib().n2f_conv3x3(mode, engine, precision, _ptr(inp_cg), cin, cout, H, W, _ptr(w),
                            _ptr(b) if b is not None else None,
                            _ptr(mask_cg) if mask_cg is not None else None, _ptr(out),
                            _stream_ptr(stream)), "n2f_conv3x3")
    return out


def conv3x3_wgrad(dout_cg, in_cg, cin, cout, H, W, precision=N2F_FP32, engine=N2F_ENGINE_AUTO,
                  stream=None):
    import torch
    dw = torch.empty((cout, cin, 3, 3), dtype=torch.float32, device=dout_cg.device)
    db = torch.empty((cout,), dtype=torch.float32, device=dout_cg.device)
    check(lib().n2f_conv3x3_wgrad(engine, precision, _ptr(dout_cg), _ptr(in_cg), cin, cout, H, W,
                                  _ptr(dw), _ptr(db), _stream_ptr(stream)), "n2f_conv3x3_wgrad")
    return dw, db


def umma_gemm(A_img, a_lbo, a_sbo, a_kstep, B_img, b_lbo, b_sbo, b_kstep, N, K, tf32=False,
              a_mn=0, b_mn=0, stream=None):
    """Diagnostic single-tile tcgen05 GEMM on shared-memory operand images (uint8 CUDA tensors)."""
    import torch
    D = torch.empty((128, N), dtype=torch.float32, device=A_img.device)
    check(lib().n2f_umma_gemm(int(tf32), N, K, a_mn, b_mn, _ptr(A_img), A_img.numel(), a_lbo,
                              a_sbo, a_kstep, _ptr(B_img), B_img.numel(), b_lbo, b_sbo, b_kstep,
                              _ptr(D), _stream_ptr(stream)), "n2f_umma_gemm")
    return D


def check_status(clear: bool = True):
    """Checked build only: (indexes found out of range since the last clear, first failing site
    as file * 100000 + line); raises N2FError(N2F_ENOTSUP) with the normal library."""
    n, site = C.c_uint64(), C.c_int()
    check(lib().n2f_check_status(C.byref(n), C.byref(site), int(clear)), "n2f_check_status")
    return int(n.value), int(site.value)


def wait_probe(limit_ms: int, stream=None) -> int:
    """Failure-detection check: a kernel waits on a barrier nothing completes; returns the
    library's code (N2F_ETIMEDOUT when the bounded wait gave up, as it must)."""
    return int(lib().n2f_wait_probe(int(limit_ms), _stream_ptr(stream)))


def _need_layout(name, t, dtype=None, shape=None, nbytes=None):
    """Raises ValueError unless t is a contiguous tensor of the given dtype and shape (or of at
    least nbytes bytes), naming the first mismatch."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, {dtype} required")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, {tuple(shape)} required")
    if nbytes is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{name}: {t.numel() * t.element_size()} bytes, {nbytes} required")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")


def _need_current_device(name, t):
    import torch
    if t.device.type != "cuda" or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {t.device}, the current CUDA device is required")


def conv3x3_wgrad_noalloc(dout_cg, in_cg, cin, cout, H, W, dw, db, precision=N2F_FP32,
                          engine=N2F_ENGINE_AUTO, stream=None):
    """n2f_conv3x3_wgrad_noalloc into caller-provided dw [C_out][C_in][3][3] and db [C_out]
    (contiguous float32 tensors on the current CUDA device, where the kernels run); the library
    allocates nothing for the call. dout_cg and in_cg are CG maps of C_out and C_in channels
    (at least C * H * W elements of the precision). Raises ValueError before the call when a
    tensor does not fit, since the kernels write dw and db without knowing their size."""
    import torch
    es = 2 if precision == N2F_BF16 else 4
    _need_layout("dw", dw, torch.float32, (cout, cin, 3, 3))
    _need_layout("db", db, torch.float32, (cout,))
    _need_layout("dout_cg", dout_cg, nbytes=cout * H * W * es)
    _need_layout("in_cg", in_cg, nbytes=cin * H * W * es)
    for name, t in (("dw", dw), ("db", db), ("dout_cg", dout_cg), ("in_cg", in_cg)):
        _need_current_device(name, t)
    check(lib().n2f_conv3x3_wgrad_noalloc(engine, precision, _ptr(dout_cg), _ptr(in_cg), cin, cout,
                                          H, W, _ptr(dw), _ptr(db), _stream_ptr(stream)),
          "n2f_conv3x3_wgrad_noalloc")
