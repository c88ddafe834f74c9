"""The Ablation Study's variants through the C ABI against the FP64 oracle: Quad 2x2
downsampling (pairs TL->TR, TR->BR, BR->BL, BL->TL) and Exact targets x_tgt - (s_tgt - s_in)
from the clean image."""
import numpy as np
import pytest

import oracle
from gpu_util import MAXABS_TOL, PSNR_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


def _img(h, w, seed):
    from paper_2108_10209_gb300 import synth
    clean = synth.blobs(h, w, seed=seed)
    return clean, (clean + synth.rng(seed + 1).normal(0, 0.1, (h, w))).astype(np.float32)


@pytest.mark.parametrize("H,W", [(2, 2), (32, 32), (7, 9), (66, 130)])
def test_quad_sub_images_bit_exact(n2f, H, W):
    x = np.random.default_rng(H * 7 + W).normal(size=(H, W)).astype(np.float32)
    tr = n2f.Trainer(x, n2f.params(downsample=n2f.N2F_DOWN_QUAD, widths=1))
    tl, trr, bl, br = oracle.quad(x.astype(np.float64))
    for k, ref in enumerate((tl, trr, br, bl)):
        assert np.array_equal(tr.export(n2f.N2F_X_PAIR, k), ref.ravel())


@pytest.mark.parametrize("downsample,exact", [(1, 0), (0, 1), (1, 1)])
def test_fixed_steps_against_oracle(n2f, downsample, exact):
    from paper_2108_10209_gb300 import synth
    clean, x = _img(32, 32, 21)
    img = np.stack([x, clean.astype(np.float32)]) if exact else x
    out = n2f.denoise(img, n2f.params(seed=0, fixed_steps=10, downsample=downsample, exact=exact))
    ref, _ = oracle.denoise(img, oracle.Params(seed=0, fixed_steps=10, downsample=downsample,
                                               exact=bool(exact)))
    d = synth.psnr(out, clean) - synth.psnr(ref, clean)
    assert abs(d) <= PSNR_TOL and np.max(np.abs(out - ref)) <= MAXABS_TOL, (d,)


def test_exact_with_zero_clean_plane_is_the_method(n2f):
    # A zero clean image removes nothing: the Exact job trains on the method's own targets.
    _, x = _img(24, 20, 22)
    p = dict(seed=3, fixed_steps=6)
    plain = n2f.denoise(x, n2f.params(**p))
    ex = n2f.denoise(np.stack([x, np.zeros_like(x)]), n2f.params(exact=1, **p))
    assert np.array_equal(plain, ex)


def test_ablation_errors(n2f):
    x = np.zeros((8, 8), np.float32)
    with n2f.Context() as ctx:
        for kw in (dict(downsample=2), dict(exact=2)):
            with pytest.raises(n2f.N2FError) as e:
                ctx.submit(x, n2f.params(**kw))
            assert e.value.code == n2f.N2F_EINVAL
        with pytest.raises(n2f.N2FError) as e:
            ctx.submit_u16(np.zeros((8, 8), np.uint16), n2f.params(exact=1))
        assert e.value.code == n2f.N2F_EINVAL
