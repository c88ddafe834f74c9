"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test names the passage of the paper (or the textbook / library definition) it pins.
The float64 torch checks use torch only as an independent implementation of the textbook
operation (conv2d, autograd, BCE-with-logits, Adam); the oracle never imports torch.
"""
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")
GOLD = os.path.join(os.path.dirname(__file__), "golden")
TINY = (3, 4, 4, 5, 5, 6, 6, 4)


def _rng(s):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- weight initialisation ----

def test_splitmix64_reference_sequence():
    # First outputs of SplitMix64 seeded with 0, as printed by the published reference
    # implementation (Vigna's splitmix64.c, next() called three times).
    assert oracle.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64_at(0, 2) == 0x06C45D188009454F


def test_param_count_matches_architecture_text():
    # Methods: 1->32, 32->32, 32->64, 64->64, 64->128, 128->128, 128->256, 256->256 (3x3 with
    # bias), then 1x1 256->1 with bias.
    n = 0
    cin = 1
    for c in oracle.WIDTHS_PLIT:
        n += c * cin * 9 + c
        cin = c
    assert n + 257 == 1_171_937 == oracle.param_count(oracle.WIDTHS_PLIT)
    assert oracle.param_count(oracle.WIDTHS_W64) == 259_201


def test_init_is_float32_uniform_within_fan_in_bound():
    th = oracle.init_params(oracle.WIDTHS_PLIT, seed=7)
    assert np.array_equal(th, th.astype(np.float32).astype(np.float64))
    parts = oracle.unpack(oracle.WIDTHS_PLIT, th)
    cin = 1
    for l, (w, b) in enumerate(parts):
        fan = cin * 9 if l < 8 else cin
        bound = 1.0 / math.sqrt(fan)
        allv = np.concatenate([w.ravel(), b.ravel()])
        assert np.all(np.abs(allv) <= bound * (1 + 1e-7))
        if allv.size > 5000:  # U(-b, b): mean 0, variance b^2/3
            assert abs(allv.mean()) < 0.02 * bound
            assert abs(allv.var() / (bound * bound / 3) - 1) < 0.02
        if l < 8:
            cin = w.shape[0]
    assert not np.array_equal(th, oracle.init_params(oracle.WIDTHS_PLIT, seed=8))
    assert np.array_equal(th, oracle.init_params(oracle.WIDTHS_PLIT, seed=7))
    # element k of the flat vector is draw k of the generator
    u = (oracle.splitmix64_at(7, 0) >> 11) * 2.0 ** -53
    assert th[0] == float(np.float32((2 * u - 1) / 3.0))


# ---------------------------------------------------------------- checkerboard downsampling --

def _load_golden_checker():
    out = {}
    for line in open(os.path.join(GOLD, "checker_4x4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, rows = line.split(":")
        out[name.strip()] = np.array([[float(v) for v in r.split(",")] for r in rows.split("|")])
    return out


def test_checker_hand_example():
    g = _load_golden_checker()
    x = np.arange(16.0).reshape(4, 4)
    got = dict(zip(("up_e", "up_o", "lf_e", "lf_o"), oracle.checker(x)))
    for k in g:
        assert np.array_equal(got[k], g[k]), k
        assert got[k].sum() == 60


@pytest.mark.parametrize("H,W", [(2, 2), (4, 6), (6, 8), (7, 9), (5, 4), (2, 130)])
def test_checker_partition_parity_adjacency(H, W):
    # Theoretical Background: even = pixels with i+j even, odd = i+j odd, compressed into
    # m x n/2 images whose (i,j) entries are adjacent pixels of the original image.
    x = np.arange(H * W, dtype=np.float64).reshape(H, W)
    up_e, up_o, lf_e, lf_o = oracle.checker(x)
    assert up_e.shape == (H, W // 2) and lf_e.shape == (H // 2, W)
    Wc, Hc = 2 * (W // 2), 2 * (H // 2)
    ii, jj = np.divmod(np.arange(H * W), W)
    for img, par, rows, cols in ((up_e, 0, H, Wc), (up_o, 1, H, Wc), (lf_e, 0, Hc, W),
                                 (lf_o, 1, Hc, W)):
        want = {k for k in range(H * W) if ii[k] < rows and jj[k] < cols and (ii[k] + jj[k]) % 2 == par}
        got = set(img.astype(int).ravel().tolist())
        assert got == want and len(got) == img.size
    # up: same row, neighbouring column; left: same column, neighbouring row
    ue, uo = up_e.astype(int), up_o.astype(int)
    assert np.all(ue // W == uo // W) and np.all(np.abs(ue % W - uo % W) == 1)
    le, lo = lf_e.astype(int), lf_o.astype(int)
    assert np.all(le % W == lo % W) and np.all(np.abs(le // W - lo // W) == 1)
    # order-preserving compaction: source columns (rows) increase along each row (column)
    assert np.all(np.diff(ue % W, axis=1) > 0) and np.all(np.diff(uo % W, axis=1) > 0)
    assert np.all(np.diff(le // W, axis=0) > 0) and np.all(np.diff(lo // W, axis=0) > 0)


def test_checker_transpose_identity():
    x = _rng(3).normal(size=(6, 10))
    up_e, up_o, lf_e, lf_o = oracle.checker(x)
    t_e, t_o, _, _ = oracle.checker(x.T.copy())
    assert np.array_equal(lf_e, t_e.T) and np.array_equal(lf_o, t_o.T)


# ---------------------------------------------------------------- convolution ---------------

def test_conv_fwd_matches_torch_float64():
    r = _rng(1)
    x = r.normal(size=(3, 7, 9)); w = r.normal(size=(5, 3, 3, 3)); b = r.normal(size=5)
    for relu in (False, True):
        got = oracle.conv3x3_fwd(x, w, b, relu)
        ref = F.conv2d(torch.tensor(x)[None], torch.tensor(w), torch.tensor(b), padding=1)[0]
        if relu:
            ref = ref.clamp_min(0)
        np.testing.assert_allclose(got, ref.numpy(), rtol=1e-13, atol=1e-13)


def test_conv_delta_kernels_pin_padding_and_direction():
    r = _rng(2)
    x = r.normal(size=(1, 5, 6))
    for ky in range(3):
        for kx in range(3):
            w = np.zeros((1, 1, 3, 3)); w[0, 0, ky, kx] = 1.0
            got = oracle.conv3x3_fwd(x, w, np.zeros(1), relu=False)[0]
            want = np.zeros((5, 6))
            dy, dx = ky - 1, kx - 1  # out(y,x) = in(y+dy, x+dx), zero outside
            for y in range(5):
                for xx in range(6):
                    if 0 <= y + dy < 5 and 0 <= xx + dx < 6:
                        want[y, xx] = x[0, y + dy, xx + dx]
            assert np.array_equal(got, want)


def test_conv_center_tap_is_matrix_product():
    r = _rng(4)
    x = r.normal(size=(4, 3, 5)); w = np.zeros((6, 4, 3, 3)); w[:, :, 1, 1] = r.normal(size=(6, 4))
    b = r.normal(size=6)
    got = oracle.conv3x3_fwd(x, w, b, relu=False)
    want = np.einsum("oc,chw->ohw", w[:, :, 1, 1], x) + b[:, None, None]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_conv_dgrad_wgrad_match_autograd_and_adjoint():
    r = _rng(5)
    x = r.normal(size=(3, 6, 7)); w = r.normal(size=(4, 3, 3, 3)); g = r.normal(size=(4, 6, 7))
    xt = torch.tensor(x, requires_grad=True); wt = torch.tensor(w, requires_grad=True)
    bt = torch.zeros(4, dtype=torch.float64, requires_grad=True)
    out = F.conv2d(xt[None], wt, bt, padding=1)[0]
    (out * torch.tensor(g)).sum().backward()
    din = oracle.conv3x3_dgrad(g, w)
    dw, db = oracle.conv3x3_wgrad(g, x)
    np.testing.assert_allclose(din, xt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dw, wt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-12, atol=1e-12)
    # adjoint identities (no library): <conv(x), g> = <x, dgrad(g)> = <w, wgrad(g, x)>
    y = oracle.conv3x3_fwd(x, w, np.zeros(4), relu=False)
    lhs = float((y * g).sum())
    assert abs(lhs - float((x * din).sum())) < 1e-10 * (1 + abs(lhs))
    assert abs(lhs - float((w * dw).sum())) < 1e-10 * (1 + abs(lhs))


# ---------------------------------------------------------------- loss ---------------------

def test_bce_closed_forms():
    z = np.zeros(10); y = _rng(6).uniform(-0.2, 1.2, 10)
    L, dz = oracle.loss(z, y, 0)
    assert abs(L - math.log(2.0)) < 1e-15            # softplus(0) = log 2, y*0 = 0
    np.testing.assert_allclose(dz, (0.5 - y) / 10, rtol=0, atol=1e-17)
    assert oracle.sigmoid(0.0) == 0.5
    assert abs(oracle.sigmoid(-800.0)) < 1e-300 and oracle.sigmoid(800.0) == 1.0


def test_bce_clamp_bounds_the_loss_for_unclipped_targets():
    # Targets outside [0, 1] (the noisy images are not clipped): with the log terms clamped at
    # -100 the loss is bounded and its gradient vanishes once the clamp is active.
    # z = 150, y = 1.2: log s ~ -e^-150, log(1-s) = -150 -> -100:  L = 0.2 * (-100) = -20
    L, dz = oracle.loss(np.array([150.0]), np.array([1.2]), 0)
    assert abs(L - (-20.0)) < 1e-12 and abs(dz[0]) < 1e-60
    # z = -150, y = -0.3: log s = -150 -> -100, log(1-s) ~ -e^-150:  L = 0.3 * (-100) = -30
    L, dz = oracle.loss(np.array([-150.0]), np.array([-0.3]), 0)
    assert abs(L - (-30.0)) < 1e-12 and 0 < dz[0] < 1e-60
    # just inside the clamps the gradient is (s - y)
    L, dz = oracle.loss(np.array([99.0]), np.array([1.2]), 0)
    assert abs(dz[0] - (oracle.sigmoid(99.0) - 1.2)) < 1e-15


@pytest.mark.parametrize("kind", [0, 1])
def test_loss_matches_torch(kind):
    r = _rng(7)
    z = r.normal(scale=2, size=(5, 6)); y = r.uniform(-0.3, 1.3, size=(5, 6))
    zt = torch.tensor(z, requires_grad=True)
    if kind == 0:
        Lt = F.binary_cross_entropy_with_logits(zt, torch.tensor(y))
    else:
        Lt = F.mse_loss(torch.sigmoid(zt), torch.tensor(y))
    Lt.backward()
    L, dz = oracle.loss(z, y, kind)
    assert abs(L - Lt.item()) < 1e-13
    np.testing.assert_allclose(dz, zt.grad.numpy(), rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- Adam ---------------------

def test_adam_first_step_closed_form():
    r = _rng(8)
    th = r.normal(size=50); g = r.normal(size=50); th0 = th.copy()
    m = np.zeros(50); v = np.zeros(50)
    oracle.adam(th, g, m, v, 1)
    # t = 1: m_hat = g, v_hat = g^2  ->  theta_1 = theta_0 - lr g / (|g| + eps)
    np.testing.assert_allclose(th, th0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_adam_matches_torch_over_steps():
    r = _rng(9)
    th = r.normal(size=40)
    p = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(40); v = np.zeros(40)
    for t in range(1, 8):
        g = r.normal(size=40) * (10.0 ** r.uniform(-3, 1))
        p.grad = torch.tensor(g.copy()); opt.step()
        oracle.adam(th, g, m, v, t)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- whole network ------------

def _torch_net(widths, theta):
    parts = [(torch.tensor(w.copy(), requires_grad=True), torch.tensor(b.copy(), requires_grad=True))
             for w, b in oracle.unpack(widths, theta)]

    def fwd(img, keep=None):
        a = torch.tensor(img)[None, None]
        for l in range(8):
            pre = F.conv2d(a, parts[l][0], parts[l][1], padding=1)
            if keep is not None:
                pre.retain_grad(); keep.append(pre)
            a = torch.relu(pre)
        wh, bh = parts[8]
        return (F.conv2d(a, wh.reshape(1, -1, 1, 1), bh))[0, 0]
    return parts, fwd


def test_training_step_matches_torch_float64():
    # Steps of the Methods' training scheme (BCE between target and output, Adam lr 1e-3),
    # replayed with a float64 torch model and torch's Adam kept across the steps.
    r = _rng(10)
    x = r.uniform(0, 1, size=(9, 8))
    p = oracle.Params(widths=TINY, seed=3)
    job = oracle.Job(x, p)
    parts, fwd = _torch_net(TINY, job.get(oracle.THETA))
    params = [t for wb in parts for t in wb]
    opt = torch.optim.Adam(params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for pair in (0, 2, 1, 3, 0):
        inp = job.get(oracle.PAIR_IN, pair); tgt = job.get(oracle.PAIR_TGT, pair)
        h, w = (9, 4) if pair < 2 else (4, 8)
        keep = []
        opt.zero_grad()
        z = fwd(inp.reshape(h, w), keep)
        L = F.binary_cross_entropy_with_logits(z, torch.tensor(tgt.reshape(h, w)))
        L.backward()
        loss = job.step(pair)
        assert abs(loss - L.item()) < 1e-12
        g = np.concatenate([t.grad.numpy().ravel() for t in params])
        np.testing.assert_allclose(job.get(oracle.GRAD), g, rtol=1e-9, atol=1e-14)
        for l in range(8):
            np.testing.assert_allclose(job.get(oracle.DELTA, l + 1), keep[l].grad.numpy().ravel(),
                                       rtol=1e-9, atol=1e-15)
            np.testing.assert_allclose(job.get(oracle.ACT, l + 1),
                                       torch.relu(keep[l]).detach().numpy().ravel(), rtol=1e-12,
                                       atol=1e-14)
        opt.step()
        th = np.concatenate([t.detach().numpy().ravel() for t in params])
        np.testing.assert_allclose(job.get(oracle.THETA), th, rtol=1e-11, atol=1e-13)
    assert job.info()["t"] == 5


def test_gradients_match_finite_differences():
    r = _rng(11)
    x = r.uniform(0, 1, size=(6, 6))
    widths = (2, 3, 3, 2, 3, 2, 2, 3)
    p = oracle.Params(widths=widths, seed=5)
    job = oracle.Job(x, p)
    th = job.get(oracle.THETA)
    inp = job.get(oracle.PAIR_IN, 0).reshape(6, 3); tgt = job.get(oracle.PAIR_TGT, 0).reshape(6, 3)
    job.step(0)
    g = job.get(oracle.GRAD)

    def L(t):
        _, z = oracle.net_forward(widths, t, inp)
        return oracle.loss(z, tgt, 0)[0]

    idx = r.choice(th.size, 60, replace=False)
    checked = 0
    for i in idx:
        hh = 1e-6 * max(1.0, abs(th[i]))
        tp = th.copy(); tp[i] += hh
        tm = th.copy(); tm[i] -= hh
        fd = (L(tp) - L(tm)) / (2 * hh)
        if abs(fd - g[i]) > 1e-6 * max(1e-3, abs(g[i])):
            # a ReLU kink inside [-h, h] is the only admissible cause
            tp2 = th.copy(); tp2[i] += hh / 10; tm2 = th.copy(); tm2[i] -= hh / 10
            fd2 = (L(tp2) - L(tm2)) / (2 * hh / 10)
            assert abs(fd2 - fd) > 1e-6 * max(1e-3, abs(fd)), (i, fd, g[i])
            continue
        checked += 1
    assert checked >= 50


def test_zero_steps_is_one_forward_pass():
    # Zero training steps: the output is the untrained network applied to the full image.
    r = _rng(12)
    x = r.uniform(0, 1, size=(8, 10))
    p = oracle.Params(widths=TINY, seed=9, fixed_steps=0)
    out, _ = oracle.denoise(x, p)
    parts, fwd = _torch_net(TINY, oracle.init_params(TINY, 9))
    want = torch.sigmoid(fwd(x)).detach().numpy()
    np.testing.assert_allclose(out, want, rtol=1e-13, atol=1e-15)


def test_fixed_steps_cycle_pairs_in_table_order():
    r = _rng(13)
    x = r.uniform(0, 1, size=(6, 8))
    p = oracle.Params(widths=TINY, seed=2, fixed_steps=6)
    out, info = oracle.denoise(x, p)
    j = oracle.Job(x, oracle.Params(widths=TINY, seed=2))
    for k in range(6):
        j.step(k % 4)
    _, v = j.validate()
    assert np.array_equal(out, v) and info["t"] == 6
    # table: (x_even -> x_odd), (x_odd -> x_even), (x'_even -> x'_odd), (x'_odd -> x'_even)
    up_e, up_o, lf_e, lf_o = oracle.checker(x)
    for k, (a, b) in enumerate(((up_e, up_o), (up_o, up_e), (lf_e, lf_o), (lf_o, lf_e))):
        assert np.array_equal(j.get(oracle.PAIR_IN, k), a.ravel())
        assert np.array_equal(j.get(oracle.PAIR_TGT, k), b.ravel())


# ---------------------------------------------------------------- stopping rule ------------

def test_stop_rule_scripted_sequences():
    # Methods: stop once 100 epochs pass without improving the best validation score.
    s = oracle.StopRule(100)
    seq = [5.0, 4.0, 3.0, 2.0, 1.0] + [1.0] * 100   # ties are not improvements
    for e, v in enumerate(seq, 1):
        s.update(v)
        assert s.stopped == (e == 105)
    s = oracle.StopRule(100)
    for e in range(1, 400):
        v = 10.0 - (min(e, 150) // 50)              # improves at epochs 1, 50, 100 and 150 only
        s.update(v)
        if s.stopped:
            break
    assert e == 250 and s.best == 7.0
    s = oracle.StopRule(100)
    for e in range(1, 400):
        s.update(1e9 if e == 1 else 2e9)            # the first epoch always sets the best
        if s.stopped:
            break
    assert e == 101
    s = oracle.StopRule(100, incl_best=True)
    for e in range(1, 200):
        s.update(1.0)
        if s.stopped:
            break
    assert e == 100


def test_output_is_mean_of_last_patience_validations():
    r = _rng(14)
    x = r.uniform(0, 1, size=(6, 6))
    P = 3
    p = oracle.Params(widths=(2,) * 8, seed=4, patience=P, lr=3e-2)
    out, info = oracle.denoise(x, p)
    # replay epoch by epoch, collecting every validation output
    j = oracle.Job(x, p)
    rule = oracle.StopRule(P)
    outs = []
    while not rule.stopped:
        for k in range(4):
            j.step(k)
        s, v = j.validate()
        rule.update(s)
        outs.append(v)
    assert info["epoch"] == rule.epoch and info["stopped"]
    np.testing.assert_allclose(out, np.mean(outs[-P:], axis=0), rtol=1e-13, atol=1e-15)


def _replay(x, p, epochs):
    """Validation scores and outputs of the first `epochs` epochs, stepped by hand."""
    j = oracle.Job(x, p)
    scores, outs = [], []
    for _ in range(epochs):
        for k in range(4):
            j.step(k)
        sc, v = j.validate()
        scores.append(sc)
        outs.append(v)
    return scores, outs


def test_window_including_the_best_epoch():
    # incl_best: the averaging window is the best epoch and the patience - 1 epochs after it;
    # the output is still the mean of the last `patience` validations when the rule fires
    r = _rng(21)
    x = r.uniform(0, 1, size=(6, 6))
    P = 3
    p = oracle.Params(widths=(2,) * 8, seed=4, patience=P, lr=3e-2, incl_best=True)
    out, info = oracle.denoise(x, p)
    assert info["stopped"]
    scores, outs = _replay(x, p, info["epoch"])
    best = int(np.argmin(scores))  # strict improvement: the first of equal minima
    assert best == info["epoch"] - P
    np.testing.assert_allclose(out, np.mean(outs[best:], axis=0), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("cap", [1, 2, 3, 5, 8])
def test_epoch_cap_averages_the_window_so_far(cap):
    # a cap reached before the rule fires: the mean of the validations after the best epoch,
    # or the best epoch's own output when none came after it (the first epoch always sets the
    # best, so a cap of one takes that branch)
    r = _rng(22)
    x = r.uniform(0, 1, size=(6, 6))
    p = oracle.Params(widths=(2,) * 8, seed=4, patience=100, lr=3e-2, max_epochs=cap)
    out, info = oracle.denoise(x, p)
    assert info["epoch"] == cap and not info["stopped"]
    scores, outs = _replay(x, p, cap)
    best = min(range(cap), key=lambda e: (scores[e], e))
    assert (best + 1 < cap) == (cap == 8)  # both branches are exercised on this image
    expect = np.mean(outs[best + 1:], axis=0) if best + 1 < cap else outs[best]
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-15)


def test_max_projection():
    # The projection of a Z-stack (Methods, fluorescence microscopy) against numpy's max along
    # Z, plus its defining properties: never below a slice, equal to some slice at every pixel,
    # the identity on a one-slice stack, and invariant under reordering the slices.
    r = _rng(15)
    vol = r.normal(size=(5, 7, 9))
    out = oracle.max_project(vol)
    assert np.array_equal(out, vol.max(axis=0))
    assert np.all(out[None] >= vol)
    assert np.all(np.any(vol == out[None], axis=0))
    assert np.array_equal(oracle.max_project(vol[:1]), vol[0])
    assert np.array_equal(oracle.max_project(vol[::-1]), out)


def test_stack_is_slices_denoised_independently():
    # Each slice of a stack is denoised as its own image: the stack result equals the per-slice
    # results, and the projection is their maximum.
    r = _rng(16)
    vol = r.uniform(0, 1, size=(3, 6, 6))
    p = oracle.Params(widths=(2,) * 8, seed=2, fixed_steps=3)
    outs, proj = oracle.denoise_stack(vol, p)
    for z in range(3):
        ref, _ = oracle.denoise(vol[z], p)
        assert np.array_equal(outs[z], ref)
    assert np.array_equal(proj, outs.max(axis=0))


def _torch_net_c(widths, theta, c0):
    parts = [(torch.tensor(w.copy(), requires_grad=True), torch.tensor(b.copy(), requires_grad=True))
             for w, b in oracle.unpack(widths, theta, c0)]

    def fwd(img):
        a = torch.tensor(img)[None]
        for l in range(8):
            a = torch.relu(F.conv2d(a, parts[l][0], parts[l][1], padding=1))
        wh, bh = parts[8]
        return (F.conv2d(a, wh.reshape(1, -1, 1, 1), bh))[0, 0]
    return parts, fwd


def test_multichannel_step_matches_torch_float64():
    # Fig. 2a caption: a multi-channel input, one predicted channel per network. Each pair's
    # input is all channels of one sub-image and its target the predicted channel of the paired
    # sub-image; replayed with a float64 torch model whose first convolution has three inputs.
    r = _rng(17)
    x = r.uniform(0, 1, size=(3, 9, 8))
    p = oracle.Params(widths=TINY, seed=5, channels=3, target=1)
    job = oracle.Job(x, p)
    assert job.np == oracle.param_count(TINY, 3) == oracle.param_count(TINY) + TINY[0] * 2 * 9
    parts, fwd = _torch_net_c(TINY, job.get(oracle.THETA), 3)
    params = [t for wb in parts for t in wb]
    opt = torch.optim.Adam(params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    subs = [oracle.checker(x[c]) for c in range(3)]
    for pair in (0, 3, 1, 2):
        h, w = (9, 4) if pair < 2 else (4, 8)
        inp = job.get(oracle.PAIR_IN, pair).reshape(3, h, w)
        tgt = job.get(oracle.PAIR_TGT, pair).reshape(h, w)
        for c in range(3):
            assert np.array_equal(inp[c], subs[c][pair])
        assert np.array_equal(tgt, subs[1][pair ^ 1])
        opt.zero_grad()
        z = fwd(inp)
        L = F.binary_cross_entropy_with_logits(z, torch.tensor(tgt))
        L.backward()
        loss = job.step(pair)
        assert abs(loss - L.item()) < 1e-12
        g = np.concatenate([t.grad.numpy().ravel() for t in params])
        np.testing.assert_allclose(job.get(oracle.GRAD), g, rtol=1e-9, atol=1e-14)
        opt.step()
        th = np.concatenate([t.detach().numpy().ravel() for t in params])
        np.testing.assert_allclose(job.get(oracle.THETA), th, rtol=1e-12, atol=1e-15)
    # validation: the predicted channel of the noisy image is the reference
    s, v = job.validate()
    v_ref, _ = oracle.net_forward(TINY, job.get(oracle.THETA), x)
    np.testing.assert_array_equal(v, v_ref)
    assert abs(s - np.mean((v_ref - x[1]) ** 2)) < 1e-15


def test_multichannel_reduces_to_one_channel():
    # With the extra input channels identically zero, the three-channel network computes what
    # the one-channel network with the first layer's channel-0 weights computes, and the
    # gradient of the zero channels' first-layer weights vanishes.
    r = _rng(18)
    x1 = r.uniform(0, 1, size=(8, 8))
    x3 = np.stack([x1, np.zeros_like(x1), np.zeros_like(x1)])
    th3 = oracle.init_params(TINY, seed=6, channels=3)
    parts3 = oracle.unpack(TINY, th3, 3)
    th1 = np.concatenate([parts3[0][0][:, :1].ravel(), parts3[0][1]] +
                         [np.concatenate([w.ravel(), b.ravel()]) for w, b in parts3[1:]])
    v3, z3 = oracle.net_forward(TINY, th3, x3)
    v1, z1 = oracle.net_forward(TINY, th1, x1)
    np.testing.assert_array_equal(z3, z1)
    job = oracle.Job(x3, oracle.Params(widths=TINY, seed=6, channels=3, target=0))
    job.step(0)
    gw1 = oracle.unpack(TINY, job.get(oracle.GRAD), 3)[0][0]
    assert np.all(gw1[:, 1:] == 0.0) and np.any(gw1[:, 0] != 0.0)


# ---------------------------------------------------------------- ablations (Quad, Exact) --

def _load_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, rows = line.split(":")
        out[k.strip()] = np.array([[float(v) for v in r.split(",")] for r in rows.split("|")])
    return out


def test_quad_hand_example():
    g = _load_golden("quad_4x4.txt")
    got = dict(zip(("tl", "tr", "bl", "br"), oracle.quad(np.arange(16.0).reshape(4, 4))))
    for k in g:
        assert np.array_equal(got[k], g[k]), k
    assert sum(v.sum() for v in got.values()) == 120


@pytest.mark.parametrize("H,W", [(2, 2), (4, 6), (7, 9), (5, 4), (2, 130)])
def test_quad_partition_and_slices(H, W):
    # The four images are the strided slices of the even crop and partition its pixels.
    x = np.arange(H * W, dtype=np.float64).reshape(H, W)
    tl, tr, bl, br = oracle.quad(x)
    crop = x[: H // 2 * 2, : W // 2 * 2]
    assert np.array_equal(tl, crop[0::2, 0::2]) and np.array_equal(tr, crop[0::2, 1::2])
    assert np.array_equal(bl, crop[1::2, 0::2]) and np.array_equal(br, crop[1::2, 1::2])
    vals = np.sort(np.concatenate([a.ravel() for a in (tl, tr, bl, br)]))
    assert np.array_equal(vals, np.sort(crop.ravel()))


def test_quad_pairs_go_round_the_block():
    # The reading taken for Quad's training pairs: TL->TR, TR->BR, BR->BL, BL->TL (every image
    # once as input and once as target, each pair of horizontally or vertically adjacent
    # pixels); one step against the float64 torch model on each pair.
    r = _rng(19)
    x = r.uniform(0, 1, size=(8, 10))
    tl, tr, bl, br = oracle.quad(x)
    want = [(tl, tr), (tr, br), (br, bl), (bl, tl)]
    job = oracle.Job(x, oracle.Params(widths=TINY, seed=2, downsample=1))
    parts, fwd = _torch_net(TINY, job.get(oracle.THETA))
    params = [t for wb in parts for t in wb]
    opt = torch.optim.Adam(params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for pair in range(4):
        inp = job.get(oracle.PAIR_IN, pair).reshape(4, 5)
        tgt = job.get(oracle.PAIR_TGT, pair).reshape(4, 5)
        assert np.array_equal(inp, want[pair][0]) and np.array_equal(tgt, want[pair][1])
        opt.zero_grad()
        L = F.binary_cross_entropy_with_logits(fwd(inp), torch.tensor(tgt))
        L.backward()
        assert abs(job.step(pair) - L.item()) < 1e-12
        g = np.concatenate([t.grad.numpy().ravel() for t in params])
        np.testing.assert_allclose(job.get(oracle.GRAD), g, rtol=1e-9, atol=1e-14)
        opt.step()


@pytest.mark.parametrize("downsample", [0, 1])
def test_exact_targets(downsample):
    # Ablation Study, Exact: the target x_tgt minus the signal difference s_tgt - s_in, taken
    # from the clean image downsampled the same way. A zero or constant clean image leaves the
    # targets unchanged; otherwise they equal the difference computed here from the sub-images.
    r = _rng(20)
    x = r.uniform(0, 1, size=(8, 8))
    s = r.uniform(0, 1, size=(8, 8))
    split = oracle.checker if downsample == 0 else (lambda a: (lambda q: (q[0], q[1], q[3], q[2]))(oracle.quad(a)))
    order = [1, 0, 3, 2] if downsample == 0 else [1, 2, 3, 0]
    base = oracle.Job(x, oracle.Params(widths=TINY, downsample=downsample))
    for clean in (np.zeros_like(x), np.full_like(x, 0.375)):
        j = oracle.Job(np.stack([x, clean]), oracle.Params(widths=TINY, downsample=downsample,
                                                            exact=True))
        for k in range(4):
            assert np.array_equal(j.get(oracle.PAIR_TGT, k), base.get(oracle.PAIR_TGT, k))
            assert np.array_equal(j.get(oracle.PAIR_IN, k), base.get(oracle.PAIR_IN, k))
    j = oracle.Job(np.stack([x, s]), oracle.Params(widths=TINY, downsample=downsample, exact=True))
    xs, ss = split(x), split(s)
    for k in range(4):
        g = order[k]
        np.testing.assert_array_equal(j.get(oracle.PAIR_TGT, k), (xs[g] - (ss[g] - ss[k])).ravel())


def test_stop_rule_golden_is_the_oracle_run():
    """tests/golden/stop_rule_plit_48.npz (written by make_stop_rule_golden.py from the oracle
    alone) is self-consistent and still the oracle's run: the image is the seeded generator's,
    the stopping rule replayed on the stored scores fires at the stored stop epoch, the output
    is the window sum over the patience, and the oracle recomputes the first two epochs' scores
    bit for bit."""
    from paper_2108_10209_gb300 import synth
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "stop_rule_plit_48.npz"))
    clean, noisy = synth.image_cells(48, 48, sigma=25.0 / 255.0, seed=int(g["image_seed"]))
    assert np.array_equal(noisy, g["noisy"]) and np.array_equal(clean, g["clean"])
    scores, P = g["scores"], int(g["patience"])
    rule = oracle.StopRule(patience=P)
    fired = []
    for s in scores:
        rule.update(float(s))
        fired.append(rule.stopped)
    assert fired[-1] and not any(fired[:-1]) and len(scores) == int(g["stop_epoch"])
    assert int(g["best_epoch"]) == int(np.argmin(scores)) + 1 == len(scores) - P
    assert rule.best == float(g["best"])
    assert np.array_equal(g["out"], g["window_sum"] / P)
    job = oracle.Job(g["noisy"], oracle.Params(widths=oracle.WIDTHS_PLIT,
                                               seed=int(g["init_seed"]), patience=P))
    assert [job.epoch(), job.epoch()] == list(scores[:2])
