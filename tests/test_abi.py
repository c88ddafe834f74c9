"""The C-ABI library loads without a GPU and exports every entry point of include/n2f.h, and the
Python binding's struct layouts agree with what a C compiler makes of the header."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "n2f.h")


@pytest.fixture(scope="module")
def n2f():
    import __graft_entry__ as g
    g.build_library()
    from paper_2108_10209_gb300 import n2f as mod
    mod.lib()
    return mod


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(n2f_[a-z0-9_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_function_is_exported_and_bound(n2f):
    names = declared_functions()
    assert len(names) >= 30
    L = C.CDLL(n2f.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
        assert name in n2f.SIGNATURES, name
    assert set(n2f.SIGNATURES) == set(names)


def test_struct_layouts_match_the_header(n2f):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "n2f.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(n2f_config), sizeof(n2f_params), sizeof(n2f_status),
         sizeof(n2f_ctx_stats));
  printf("%zu %zu %zu %zu %zu\n", offsetof(n2f_params, seed), offsetof(n2f_params, engine),
         offsetof(n2f_status, t_done_ms), offsetof(n2f_params, eps),
         offsetof(n2f_params, patience));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HDR), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:4] == [C.sizeof(n2f.Config), C.sizeof(n2f.Params), C.sizeof(n2f.Status),
                         C.sizeof(n2f.CtxStats)]
    assert sizes[4:] == [n2f.Params.seed.offset, n2f.Params.engine.offset,
                         n2f.Status.t_done_ms.offset, n2f.Params.eps.offset,
                         n2f.Params.patience.offset]


def test_defaults_follow_the_methods_section(n2f):
    p = n2f.params()
    # Adam's constants are held in double, exactly as the oracle's (Kingma & Ba's defaults)
    assert p.lr == 1e-3 and p.patience == 100 and p.fixed_steps == -1
    assert p.precision == n2f.N2F_FP32 and p.loss == n2f.N2F_LOSS_BCE
    assert p.beta1 == 0.9 and p.beta2 == 0.999 and p.eps == 1e-8


def test_param_counts_agree_with_the_oracle(n2f):
    import oracle
    assert n2f.param_count(n2f.N2F_WIDTHS_PLIT) == oracle.param_count(oracle.WIDTHS_PLIT)
    assert n2f.param_count(n2f.N2F_WIDTHS_W64) == oracle.param_count(oracle.WIDTHS_W64)


def test_error_strings(n2f):
    L = n2f.lib()
    for code in range(0, -11, -1):
        assert L.n2f_strerror(code)


def _no_gpu():
    import torch
    return not torch.cuda.is_available()


# The argument checks return before any CUDA call. The pointers below are placeholders that no
# call may dereference, so the test runs only where there is no GPU: a missing check then ends in
# a failed CUDA call (another error code), never in a device access.
@pytest.mark.skipif(not _no_gpu(), reason="placeholder pointers: run without a GPU only")
def test_op_level_argument_checks(n2f):
    L = n2f.lib()
    P = C.c_void_p(256)  # placeholder, never dereferenced
    E = n2f.N2F_EINVAL
    F32, TC = n2f.N2F_FP32, n2f.N2F_ENGINE_TC
    # precision outside the two forms
    assert L.n2f_pack_cg(P, 8, 4, 4, 7, P, None) == E
    assert L.n2f_unpack_cg(P, 8, 4, 4, -1, P, None) == E
    assert L.n2f_conv3x3(0, TC, 2, P, 32, 32, 8, 8, P, P, None, P, None) == E
    assert L.n2f_conv3x3_wgrad(TC, 5, P, P, 32, 32, 8, 8, P, P, None) == E
    assert L.n2f_conv3x3_wgrad_noalloc(TC, 5, P, P, 32, 32, 8, 8, P, P, None) == E
    # engine outside enum n2f_engine, mode other than 0 / 1, channel counts, sizes
    assert L.n2f_conv3x3(0, 3, F32, P, 32, 32, 8, 8, P, P, None, P, None) == E
    assert L.n2f_conv3x3(2, TC, F32, P, 32, 32, 8, 8, P, P, P, P, None) == E
    assert L.n2f_conv3x3(1, TC, F32, P, 32, 32, 8, 8, P, None, None, P, None) == E  # no mask
    assert L.n2f_conv3x3(0, TC, F32, P, 12, 32, 8, 8, P, P, None, P, None) == E
    assert L.n2f_conv3x3_wgrad(-1, F32, P, P, 32, 32, 8, 8, P, P, None) == E
    assert L.n2f_conv3x3_wgrad(TC, F32, P, P, 32, 32, 0, 8, P, P, None) == E
    assert L.n2f_pack_cg(P, 6, 4, 4, F32, P, None) == E      # C not a multiple of G = 4
    assert L.n2f_pack_cg(P, 12, 4, 4, n2f.N2F_BF16, P, None) == E  # G = 8 for bf16
    assert L.n2f_checker_gather(P, 1, 8, P, P, P, P, None) == E
    assert L.n2f_max_project(P, 0, 4, 4, P, None) == E
    assert L.n2f_wait_probe(0, None) == E and L.n2f_wait_probe(10001, None) == E


@pytest.mark.parametrize("bad", [
    dict(precision=2), dict(loss=5), dict(widths=3), dict(engine=4), dict(engine=-1),
    dict(lr=0.0), dict(lr=float("nan")), dict(beta1=1.0), dict(beta2=-0.5), dict(eps=0.0),
    dict(patience=0), dict(incl_best=1, patience=1), dict(channels=5), dict(channels=-1),
    dict(channels=3, target_channel=3), dict(target_channel=1), dict(downsample=9),
    dict(exact=2), dict(struct_size=8)])
def test_trainer_rejects_parameters_before_touching_the_device(n2f, bad):
    # a valid host image (room for every plane any of these parameter sets could ask for): the
    # parameter check runs before the first CUDA call, so this runs with or without a GPU
    img = np.random.default_rng(0).random(6 * 8 * 8).astype(np.float32)
    tr = C.c_void_p()
    p = n2f.params(**bad)
    rc = n2f.lib().n2f_trainer_create(C.byref(tr), img.ctypes.data, 8, 8, C.byref(p), None)
    assert rc == n2f.N2F_EINVAL and not tr.value


@pytest.mark.parametrize("H,W,poison", [(1, 8, None), (8, 1, None), (0, 0, None), (8, 8, 17),
                                         (1 << 16, 1 << 15, None)])
def test_trainer_rejects_images_before_touching_the_device(n2f, H, W, poison):
    img = np.zeros(64, np.float32)
    if poison is not None:
        img[poison] = np.inf
    tr = C.c_void_p()
    rc = n2f.lib().n2f_trainer_create(C.byref(tr), img.ctypes.data, H, W, None, None)
    assert rc == n2f.N2F_EINVAL and not tr.value


def test_normal_build_has_no_checks(n2f):
    # n2f_check_status answers N2F_ENOTSUP in libn2f.so before touching any device
    n, site = C.c_uint64(7), C.c_int(7)
    assert n2f.lib().n2f_check_status(C.byref(n), C.byref(site), 0) == n2f.N2F_ENOTSUP
    assert n2f.lib().n2f_check_status(None, C.byref(site), 0) == n2f.N2F_EINVAL


def test_overlap_holds_its_own_validation_buffers(n2f):
    """n2f_job_bytes (what admission counts) includes what overlapped validation adds: the
    validation ping-pong pair (2 x 256 channels x H x W), no longer aliasing the training
    activations, and the weight snapshot (theta and the forward weight copies); fixed-step jobs
    never overlap and hold nothing more."""
    H, W = 64, 96
    count = n2f.param_count()
    for precision, es in ((n2f.N2F_FP32, 4), (n2f.N2F_BF16, 2)):
        a = n2f.job_bytes(H, W, n2f.params(precision=precision))
        b = n2f.job_bytes(H, W, n2f.params(precision=precision, overlap=1))
        vb = 2 * 256 * H * W * es
        # snapshot: theta (4 B) + SIMT forward copies (4 B per weight, the biases and head
        # excluded) + the tensor-core copies where the driver's tensor-map encoder is present
        # (2 B per weight, float32 form also the 2-byte lo parts), alignment, a saved job state
        assert vb + 7 * count <= b - a <= vb + 12 * count + 64 * 256, (precision, b - a)
        fa = n2f.job_bytes(H, W, n2f.params(precision=precision, fixed_steps=5))
        fb = n2f.job_bytes(H, W, n2f.params(precision=precision, fixed_steps=5, overlap=1))
        assert fa == fb
    with pytest.raises(n2f.N2FError):
        n2f.job_bytes(H, W, n2f.params(overlap=2))
