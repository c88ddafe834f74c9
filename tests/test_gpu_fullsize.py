"""Parity at the benchmark's full size: a 512x512 cell image (the plain float32 workload), the
library's own launch configuration for that size, outputs sampled where the FP64 oracle can
compute them one by one. Each sampled value is computed by an oracle function on the GPU's own
inputs of that kernel (a 3x3 crop around an output pixel, a one-channel pixel sum, the whole
parameter vector for Adam), so both sides take the same ReLU decisions."""
import numpy as np
import pytest

import oracle
from gpu_util import REL_STEP, layer_slices, rel_err

pytestmark = pytest.mark.gpu

S = 512
LAYERS = (2, 5, 8)  # one 32-, one 64-/128- and one 256-channel layer
NS = 48             # sampled outputs per check


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


@pytest.fixture(scope="module")
def case():
    from paper_2108_10209_gb300 import synth
    clean, noisy = synth.image_cells(S, S, sigma=25 / 255, seed=101)
    return noisy.astype(np.float32)


def _crop(a, y, x):
    """(C, 3, 3) neighbourhood of pixel (y, x) of a (C, h, w) map, zeros outside it."""
    c, h, w = a.shape
    out = np.zeros((c, 3, 3))
    for dy in range(3):
        for dx in range(3):
            yy, xx = y + dy - 1, x + dx - 1
            if 0 <= yy < h and 0 <= xx < w:
                out[:, dy, dx] = a[:, yy, xx]
    return out


def _pixels(r, h, w, n):
    # include the corners and edges (zero padding) besides random interior pixels
    fixed = [(0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1), (0, w // 2), (h // 2, 0)]
    return fixed + [(int(r.integers(0, h)), int(r.integers(0, w))) for _ in range(n - len(fixed))]


def test_training_step_sampled(n2f, case):
    ow = oracle.WIDTHS_PLIT
    sl = layer_slices(ow)
    tr = n2f.Trainer(case, n2f.params(seed=0))
    subs = oracle.checker(case.astype(np.float64))
    r = np.random.default_rng(7)
    for pair in (0, 2):  # both sub-image shapes (512x256, 256x512)
        theta = tr.export(n2f.N2F_X_THETA)
        m0, v0 = tr.export(n2f.N2F_X_ADAM_M), tr.export(n2f.N2F_X_ADAM_V)
        tr.step(pair)
        h, w = (S, S // 2) if pair < 2 else (S // 2, S)
        inp = tr.export(n2f.N2F_X_PAIR, pair).reshape(1, h, w)
        assert np.array_equal(inp[0], subs[pair])  # the gather, bit-exact at full size
        parts = oracle.unpack(ow, theta)
        grad = tr.export(n2f.N2F_X_GRAD)
        act = {l: tr.export(n2f.N2F_X_ACT, l).reshape(ow[l - 1], h, w)
               for l in sorted({l for L in LAYERS for l in (L - 1, L)} - {0})}
        dlt = {l: tr.export(n2f.N2F_X_DELTA, l).reshape(ow[l - 1], h, w)
               for l in sorted({l for L in LAYERS for l in (L - 1, L)})}
        px = _pixels(r, h, w, NS)
        for L in LAYERS:
            W, b = parts[L - 1]
            prev = act[L - 1]
            # forward: one output pixel per crop, every output channel
            got = np.stack([act[L][:, y, x] for y, x in px])
            ref = np.stack([oracle.conv3x3_fwd(_crop(prev, y, x), W, b)[:, 1, 1] for y, x in px])
            assert rel_err(got, ref) < REL_STEP, ("forward", pair, L)
            # dgrad with the ReLU mask of the layer's input
            got = np.stack([dlt[L - 1][:, y, x] for y, x in px])
            ref = np.stack([oracle.conv3x3_dgrad(_crop(dlt[L], y, x), W)[:, 1, 1] *
                            (prev[:, y, x] > 0) for y, x in px])
            assert rel_err(got, ref) < REL_STEP, ("dgrad", pair, L)
            # weight and bias gradients: pixel sums over the whole sub-image, sampled (o, c)
            gw = grad[sl[L - 1][0]].reshape(W.shape)
            gb = grad[sl[L - 1][1]]
            oc = [(int(r.integers(0, W.shape[0])), int(r.integers(0, W.shape[1]))) for _ in range(8)]
            got_w, ref_w, got_b, ref_b = [], [], [], []
            for o, c in oc:
                dw, db = oracle.conv3x3_wgrad(dlt[L][o:o + 1], prev[c:c + 1])
                got_w.append(gw[o, c]); ref_w.append(dw[0, 0])
                got_b.append(gb[o]); ref_b.append(db[0])
            assert rel_err(got_w, ref_w) < REL_STEP, ("wgrad", pair, L)
            assert rel_err(got_b, ref_b) < REL_STEP, ("bias grad", pair, L)
        # head: logits, loss gradient, delta_8 at the sampled pixels
        a8 = act[8]
        z = np.array([oracle.head_fwd(a8[:, y:y + 1, x:x + 1], parts[8][0], parts[8][1][0])[0, 0]
                      for y, x in px])
        tgt = np.array([subs[pair ^ 1][y, x] for y, x in px])
        _, dz_ref = oracle.loss(z, tgt, 0)
        dz = tr.export(n2f.N2F_X_DZ).reshape(h, w)
        got = np.array([dz[y, x] for y, x in px]) * (h * w)
        assert rel_err(got, dz_ref * len(px)) < REL_STEP, ("dz", pair)
        # Adam over the whole parameter vector
        th, m, v = theta.copy(), m0.copy(), v0.copy()
        oracle.adam(th, grad, m, v, t=pair // 2 + 1)
        assert rel_err(tr.export(n2f.N2F_X_THETA), th) < 1e-6, ("adam", pair)


def test_validation_sampled(n2f, case):
    # The full-image validation forward after one step, at interior pixels (the 8 layers see
    # 17 x 17 pixels, so the oracle's forward on that crop gives the exact output there).
    tr = n2f.Trainer(case, n2f.params(seed=3))
    tr.step(0)
    tr.validate()
    theta = tr.export(n2f.N2F_X_THETA)
    V = tr.export(n2f.N2F_X_VAL).reshape(S, S)
    r = np.random.default_rng(11)
    got, ref = [], []
    for _ in range(24):
        y, x = int(r.integers(8, S - 8)), int(r.integers(8, S - 8))
        crop = case[y - 8:y + 9, x - 8:x + 9].astype(np.float64)
        v, _ = oracle.net_forward(oracle.WIDTHS_PLIT, theta, crop)
        got.append(V[y, x]); ref.append(v[8, 8])
    assert rel_err(got, ref) < REL_STEP
