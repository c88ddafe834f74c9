"""The two precision forms against the FP64 oracle, per image, on both noise models of the
workloads (Gaussian and Poisson-Gaussian, photon peak 30, read noise 0.02): PSNR delta and
max-abs pixel error after the same fixed number of steps from the same initial weights."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

STEPS = 8


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


def _images():
    from paper_2108_10209_gb300 import synth
    return [("gauss25", synth.image_cells(128, 128, sigma=25 / 255, seed=11)),
            ("poisson-gauss", synth.image_cells_pg(128, 128, peak=30.0, read=0.02, seed=12))]


def test_forms_against_the_oracle(n2f):
    from paper_2108_10209_gb300 import synth
    rows = []
    for name, (clean, noisy) in _images():
        ref, _ = oracle.denoise(noisy, oracle.Params(seed=0, fixed_steps=STEPS))
        for prec in (n2f.N2F_FP32, n2f.N2F_BF16):
            out = n2f.denoise(noisy, n2f.params(seed=0, fixed_steps=STEPS, precision=prec))
            dpsnr = synth.psnr(out, clean) - synth.psnr(ref, clean)
            maxabs = float(np.max(np.abs(out - ref)))
            rows.append((name, "fp32" if prec == n2f.N2F_FP32 else "bf16", dpsnr, maxabs))
            if prec == n2f.N2F_FP32:
                assert abs(dpsnr) <= 0.05 and maxabs <= 2e-3, rows[-1]
            else:
                assert abs(dpsnr) <= 0.5 and maxabs <= 5e-2, rows[-1]
    for r in rows:
        print(f"{r[0]:14s} {r[1]}: dPSNR vs FP64 oracle {r[2]:+.4f} dB, max-abs {r[3]:.2e}")
