"""The allocation-free weight-gradient entry point against the allocating one.

n2f_conv3x3_wgrad_noalloc serves callers that cannot allocate device memory when they need a
weight gradient (device memory reserved in full by another allocator, or loops that must not
block on cudaMalloc): its partial-sum workspace is a fixed device array inside the library.
Two calls in a row must each match n2f_conv3x3_wgrad (the array keeps the previous call's
contents, so the second call also checks nothing stale leaks through). This file is collected
last and passes alone in a fresh process or after the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# float32: the pixel sums may be split differently (a smaller workspace means fewer splits),
# so the two results agree to float32 summation-order differences; bf16 inputs, same.
REL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f
    torch.cuda.set_device(0)
    return n2f, torch


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("engine", [1, 2])
def test_noalloc_wgrad_matches_allocating_entry_point(env, precision, engine):
    n2f, torch = env
    cases = [(256, 256, 24, 200), (32, 64, 17, 130)]
    for call, (cin, cout, H, W) in enumerate(cases * 2):  # two calls in a row per shape
        g = torch.Generator(device="cpu").manual_seed(1000 * call + cin + cout)
        x = torch.relu(torch.randn((cin, H, W), generator=g)).cuda()
        d = torch.randn((cout, H, W), generator=g).cuda()
        xc, dc = n2f.pack_cg(x, precision), n2f.pack_cg(d, precision)
        ref_w, ref_b = n2f.conv3x3_wgrad(dc, xc, cin, cout, H, W, precision=precision,
                                         engine=engine)
        dw = torch.full((cout, cin, 3, 3), float("nan"), device="cuda")
        db = torch.full((cout,), float("nan"), device="cuda")
        n2f.conv3x3_wgrad_noalloc(dc, xc, cin, cout, H, W, dw, db, precision=precision,
                                  engine=engine)
        torch.cuda.synchronize()
        assert torch.isfinite(dw).all() and torch.isfinite(db).all()
        assert _rel(dw, ref_w) < REL, (call, cin, cout)
        assert _rel(db, ref_b) < REL, (call, cin, cout)


def test_noalloc_rejects_layers_beyond_the_workspace(env):
    n2f, torch = env
    big = 1024  # one split needs 9 * 1024 * 1024 floats: more than the 4 Mi-float array
    t = torch.zeros(big * 2 * 2, dtype=torch.float32, device="cuda")
    dw = torch.zeros((big, big, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.zeros((big,), dtype=torch.float32, device="cuda")
    with pytest.raises(n2f.N2FError) as e:
        n2f.conv3x3_wgrad_noalloc(t, t, big, big, 2, 2, dw, db, engine=n2f.N2F_ENGINE_SIMT)
    assert e.value.code == n2f.N2F_ETOOBIG
