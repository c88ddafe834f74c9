"""Helpers shared by the GPU tests (comparison metrics and small conversions)."""
import numpy as np

# Tolerances of the float32 form against the FP64 oracle:
#   single-step activations and gradients: max|gpu - oracle| <= 1e-4 * max|oracle| per tensor
#   after a fixed-step run: |PSNR difference| <= 0.05 dB and max-abs pixel error <= 2e-3
REL_STEP = 1e-4
PSNR_TOL = 0.05
MAXABS_TOL = 2e-3


def rel_err(got, ref):
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(got))) if got.size else 0.0
    return float(np.max(np.abs(got - ref))) / scale


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_slices(widths):
    """[(w_slice, b_slice)] * 8 + [(head_w, head_b)] into the flat parameter vector."""
    out, off, cin = [], 0, 1
    for c in widths:
        n = c * cin * 9
        out.append((slice(off, off + n), slice(off + n, off + n + c)))
        off += n + c
        cin = c
    out.append((slice(off, off + cin), slice(off + cin, off + cin + 1)))
    return out
