"""Pins the tcgen05 operand conventions the tensor-core convolutions rely on.

A single 128 x N tile D = A B^T is computed through n2f_umma_gemm from shared-memory images
built here in the no-swizzle canonical layouts: K-major (8 rows x 16 bytes per core matrix,
K-adjacent core matrices `lbo` bytes apart, 8-row groups `sbo` apart) and MN-major (8 K-rows x
16 bytes of consecutive M/N elements per core matrix, K-adjacent `lbo`, M/N-adjacent `sbo`).
Operands are small integers, exact in bf16 and TF32 and in an FP32 sum, so D must be exact.
Every case keeps the footprint of either stride reading inside the kernel's fixed 200 KB of
shared memory (A in the first 100 KB, B in the second)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f
    torch.cuda.set_device(0)
    return n2f, torch


def _bits(vals, tf32):
    if tf32:
        return vals.astype(np.float32).view(np.uint8).reshape(*vals.shape, 4)
    f = vals.astype(np.float32).view(np.uint32)
    return (f >> 16).astype(np.uint16).view(np.uint8).reshape(*vals.shape, 2)


def kmajor_image(M, rows, K, lbo, sbo, tf32):
    """M[rows][K] -> K-major image: byte (r//8)*sbo + (k//T)*lbo + (r%8)*16 + (k%T)*es."""
    es = 4 if tf32 else 2
    T = 16 // es
    size = (rows // 8 - 1) * sbo + (K // T - 1) * lbo + 128
    img = np.zeros(size, np.uint8)
    b = _bits(M, tf32)
    for r in range(rows):
        for k in range(K):
            off = (r // 8) * sbo + (k // T) * lbo + (r % 8) * 16 + (k % T) * es
            img[off:off + es] = b[r, k]
    return img


def mnmajor_image(M, rows, K, lbo, sbo, tf32):
    """M[rows][K] -> MN-major image: byte (r//T)*sbo + (k//8)*lbo + (k%8)*16 + (r%T)*es."""
    es = 4 if tf32 else 2
    T = 16 // es
    size = (rows // T - 1) * sbo + (K // 8 - 1) * lbo + 128
    img = np.zeros(size, np.uint8)
    b = _bits(M, tf32)
    for r in range(rows):
        for k in range(K):
            off = (r // T) * sbo + (k // 8) * lbo + (k % 8) * 16 + (r % T) * es
            img[off:off + es] = b[r, k]
    return img


CASES = [
    # (name, tf32, N, K, a_mn, b_mn, a_lbo, a_sbo, b_lbo, b_sbo)  (lbo/sbo None = dense)
    ("bf16 K-major dense", 0, 64, 64, 0, 0, None, None, None, None),
    ("bf16 K-major padded", 0, 128, 32, 0, 0, 128 * 16 + 64, 128, 16 * 256 + 32, 256),
    ("tf32 K-major dense", 1, 128, 32, 0, 0, None, None, None, None),
    ("bf16 K-major N=32", 0, 32, 48, 0, 0, None, None, None, None),
    ("bf16 MN-major", 0, 256, 64, 1, 1, None, None, None, None),
    ("tf32 K-major padded", 1, 64, 32, 0, 0, 128 * 16 + 48, 128, 8 * 256 + 16, 256),
    ("bf16 MN-major padded", 0, 128, 32, 1, 1, 160, 4 * 160 + 32, 144, 4 * 160 + 32),
]
# TF32 operands would have to be K-major: an MN-major TF32 image in the same convention did not
# give the product on the GB300. The float32 form therefore multiplies fp16 parts, which the
# weight gradient reads MN-major like the bf16 form's operands.


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_umma_tile_layouts(env, case):
    n2f, torch = env
    name, tf32, N, K, a_mn, b_mn, a_lbo, a_sbo, b_lbo, b_sbo = case
    r = np.random.default_rng(N * 7 + K)
    A = r.integers(-4, 5, size=(128, K)).astype(np.float64)
    B = r.integers(-4, 5, size=(N, K)).astype(np.float64)
    T = 4 if tf32 else 8
    kstep = 8 if tf32 else 16

    def build(Mx, rows, mn, lbo, sbo):
        if mn:
            lbo = 128 if lbo is None else lbo        # K-adjacent core matrices (8 rows of 16 B)
            sbo = K * 16 if sbo is None else sbo     # M/N-adjacent: one [K][16 B] column block
            return mnmajor_image(Mx, rows, K, lbo, sbo, tf32), lbo, sbo, (kstep // 8) * lbo
        lbo = rows * 16 if lbo is None else lbo      # one 16-byte K slab of all rows
        sbo = 128 if sbo is None else sbo
        return kmajor_image(Mx, rows, K, lbo, sbo, tf32), lbo, sbo, (kstep // T) * lbo

    ia, al, as_, ak = build(A, 128, a_mn, a_lbo, a_sbo)
    ib, bl, bs, bk = build(B, N, b_mn, b_lbo, b_sbo)
    pad = lambda img: np.concatenate([img, np.zeros((-img.size) % 16, np.uint8)])
    ta = torch.tensor(pad(ia), device="cuda")
    tb = torch.tensor(pad(ib), device="cuda")
    D = n2f.umma_gemm(ta, al, as_, ak, tb, bl, bs, bk, N, K, tf32=bool(tf32), a_mn=a_mn,
                      b_mn=b_mn).cpu().numpy().astype(np.float64)
    want = A @ B.T
    bad = np.argwhere(D != want)
    assert bad.size == 0, f"{name}: {len(bad)} mismatches, first {bad[:4].tolist()}"
