"""Multi-channel input (Fig. 2a caption: the network input may be multi-channel, its output is
always one channel, and an RGB image is denoised one channel per network), through the C ABI
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import MAXABS_TOL, PSNR_TOL, REL_STEP, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


def _rgb(h, w, seed):
    from paper_2108_10209_gb300 import synth
    clean = np.stack([synth.blobs(h, w, seed=seed + 10 * c) for c in range(3)])
    noisy = clean + synth.rng(seed + 1).normal(0, 0.1, clean.shape)
    return clean, noisy.astype(np.float32)


def test_initial_weights_bit_identical(n2f):
    x = np.zeros((3, 8, 8), np.float32)
    tr = n2f.Trainer(x, n2f.params(seed=9, channels=3))
    assert np.array_equal(tr.export(n2f.N2F_X_THETA), oracle.init_params(seed=9, channels=3))


@pytest.mark.parametrize("engine", [1, 2])
def test_first_layer_and_target_step_parity(n2f, engine):
    # One step per pair on the GPU's own inputs: every input plane of the pair is the
    # checkerboard sub-image of that channel, the first layer's forward and weight gradient over
    # three planes, and the loss gradient against the predicted plane of the paired sub-image.
    _, x = _rgb(32, 32, 3)
    t = 2
    tr = n2f.Trainer(x, n2f.params(seed=1, channels=3, target_channel=t, engine=engine))
    subs = [oracle.checker(x[c].astype(np.float64)) for c in range(3)]
    ow = oracle.WIDTHS_PLIT
    for pair in (0, 3, 1, 2):
        theta = tr.export(n2f.N2F_X_THETA)
        tr.step(pair)
        h, w = (32, 16) if pair < 2 else (16, 32)
        inp = tr.export(n2f.N2F_X_PAIR, pair).reshape(3, h, w)
        for c in range(3):
            assert np.array_equal(inp[c], subs[c][pair])
        parts = oracle.unpack(ow, theta, 3)
        a1 = tr.export(n2f.N2F_X_ACT, 1).reshape(ow[0], h, w)
        assert rel_err(a1, oracle.conv3x3_fwd(inp, parts[0][0], parts[0][1])) < REL_STEP
        act8 = tr.export(n2f.N2F_X_ACT, 8).reshape(ow[7], h, w)
        z = oracle.head_fwd(act8, parts[8][0], parts[8][1][0])
        _, dz_ref = oracle.loss(z, subs[t][pair ^ 1], 0)
        assert rel_err(tr.export(n2f.N2F_X_DZ).reshape(h, w), dz_ref) < REL_STEP
        d1 = tr.export(n2f.N2F_X_DELTA, 1).reshape(ow[0], h, w)
        dw, db = oracle.conv3x3_wgrad(d1, inp)
        n1 = ow[0] * 3 * 9
        grad = tr.export(n2f.N2F_X_GRAD)
        assert rel_err(grad[:n1], dw) < REL_STEP and rel_err(grad[n1:n1 + ow[0]], db) < REL_STEP


@pytest.mark.parametrize("precision", [0, 1])
def test_fixed_steps_per_channel(n2f, precision):
    # Each output channel of an RGB image after the fixed 10-step run against the oracle's run
    # of that channel's network; denoise_channels equals the three jobs run one by one.
    from paper_2108_10209_gb300 import synth
    clean, x = _rgb(32, 32, 7)
    p = n2f.params(seed=0, fixed_steps=10, precision=precision)
    both = n2f.denoise_channels(x, p)
    for t in range(3):
        q = n2f.params(seed=0, fixed_steps=10, precision=precision, channels=3, target_channel=t)
        out = n2f.denoise(x, q)
        assert np.array_equal(out, both[t])
        ref, _ = oracle.denoise(x, oracle.Params(seed=0, fixed_steps=10, channels=3, target=t))
        d = synth.psnr(out, clean[t]) - synth.psnr(ref, clean[t])
        m = np.max(np.abs(out - ref))
        if precision == 0:
            assert abs(d) <= PSNR_TOL and m <= MAXABS_TOL, (t, d, m)
        else:
            assert abs(d) <= 0.5 and m <= 5e-2, (t, d, m)


def test_channel_errors(n2f):
    x = np.zeros((3, 8, 8), np.float32)
    with n2f.Context() as ctx:
        for kw in (dict(channels=5), dict(channels=3, target_channel=3),
                   dict(channels=-1), dict(channels=1, target_channel=1)):
            with pytest.raises(n2f.N2FError) as e:
                ctx.submit(x, n2f.params(**kw))
            assert e.value.code == n2f.N2F_EINVAL
        with pytest.raises(n2f.N2FError) as e:
            ctx.submit_u16(np.zeros((8, 8), np.uint16), n2f.params(channels=3))
        assert e.value.code == n2f.N2F_EINVAL
