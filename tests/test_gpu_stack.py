"""Z-stacks (Methods, fluorescence microscopy: slices denoised as independent images, then max
projected along Z): the projection kernel bit-exact against torch's max, and a small stack
through the job API against the oracle's per-slice runs."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


@pytest.mark.parametrize("Z,H,W", [(1, 8, 8), (5, 37, 41), (7, 64, 64), (41, 96, 128)])
def test_max_project_exact(n2f, Z, H, W):
    # 37 x 41 is not a multiple of 4 pixels (scalar path); the others take 16-byte accesses.
    import torch
    g = torch.Generator(device="cpu").manual_seed(Z * 1000 + H)
    vol = torch.randn((Z, H, W), generator=g).cuda()
    out = n2f.max_project(vol)
    torch.cuda.synchronize()
    assert torch.equal(out, vol.max(dim=0).values)


def test_max_project_errors(n2f):
    import torch
    vol = torch.zeros((2, 4, 4), device="cuda")
    out = torch.zeros((4, 4), device="cuda")
    for Z, H, W in ((0, 4, 4), (2, 0, 4), (2, 4, 0)):
        rc = n2f.lib().n2f_max_project(n2f._ptr(vol), Z, H, W, n2f._ptr(out), None)
        assert rc == n2f.N2F_EINVAL


def test_stack_against_oracle(n2f):
    # Three slices of a live-cell-like volume, a fixed number of steps each: every slice within
    # the fixed-run bar of the oracle's run of that slice; the projection equal to the maximum of
    # the GPU's own slices exactly and within the same bar of the oracle's projection; each
    # slice identical to the same image denoised alone.
    from paper_2108_10209_gb300 import synth
    clean, noisy = synth.volume_cells(3, 32, 32, seed=5)
    p_gpu = n2f.params(seed=0, fixed_steps=10)
    slices, proj = n2f.denoise_stack(noisy.astype(np.float32), p_gpu)
    s = slices.cpu().numpy().astype(np.float64)
    pr = proj.cpu().numpy().astype(np.float64)
    assert np.array_equal(pr, s.max(axis=0))
    ref_s, ref_p = oracle.denoise_stack(noisy, oracle.Params(seed=0, fixed_steps=10))
    for z in range(3):
        d = synth.psnr(s[z], clean[z]) - synth.psnr(ref_s[z], clean[z])
        assert abs(d) <= 0.05 and np.max(np.abs(s[z] - ref_s[z])) <= 2e-3, (z, d)
        alone = n2f.denoise(noisy[z].astype(np.float32), p_gpu)
        assert np.array_equal(alone, slices[z].cpu().numpy())
    assert np.max(np.abs(pr - ref_p)) <= 2e-3
