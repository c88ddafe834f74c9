"""Argument checks of the Python binding that run before any C call (CPU only).

Two entry points take device buffers whose size the library cannot see: the allocation-free
weight gradient writes dw and db in place, and n2f_submit_device copies planes * H * W floats
from the image pointer. The binding must reject tensors that do not fit before calling them."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def n2f():
    import __graft_entry__ as g
    g.build_library()
    from paper_2108_10209_gb300 import n2f as mod
    return mod


def _noalloc(n2f, dw, db, dout=None, inp=None, cin=32, cout=64, H=4, W=5, precision=0):
    es = 2 if precision == 1 else 4
    dout = dout if dout is not None else torch.zeros(cout * H * W * es, dtype=torch.uint8)
    inp = inp if inp is not None else torch.zeros(cin * H * W * es, dtype=torch.uint8)
    n2f.conv3x3_wgrad_noalloc(dout, inp, cin, cout, H, W, dw, db, precision=precision)


def test_noalloc_rejects_outputs_that_do_not_fit(n2f):
    cin, cout = 32, 64
    good_w = torch.zeros((cout, cin, 3, 3))
    good_b = torch.zeros((cout,))
    cases = [
        (dict(dw=good_w.double(), db=good_b), "dw: dtype"),
        (dict(dw=good_w.bfloat16(), db=good_b), "dw: dtype"),
        (dict(dw=torch.zeros((cout, cin, 3, 2)), db=good_b), "dw: shape"),
        (dict(dw=torch.zeros((cin, cout, 3, 3)), db=good_b), "dw: shape"),
        (dict(dw=torch.zeros((cin, cout, 3, 3)).transpose(0, 1), db=good_b), "dw: must be contiguous"),
        (dict(dw=good_w, db=torch.zeros((cout + 1,))), "db: shape"),
        (dict(dw=good_w, db=good_b.half()), "db: dtype"),
        (dict(dw=good_w, db=good_b), "dw: on cpu"),  # right size and type, wrong device
    ]
    for kw, msg in cases:
        with pytest.raises(ValueError, match=msg):
            _noalloc(n2f, kw["dw"], kw["db"], cin=cin, cout=cout)


def test_noalloc_rejects_inputs_smaller_than_their_maps(n2f):
    cin, cout, H, W = 32, 64, 4, 5
    w, b = torch.zeros((cout, cin, 3, 3)), torch.zeros((cout,))
    with pytest.raises(ValueError, match="dout_cg: .* bytes"):
        _noalloc(n2f, w, b, dout=torch.zeros(cout * H * W - 1), cin=cin, cout=cout, H=H, W=W)
    with pytest.raises(ValueError, match="in_cg: .* bytes"):
        # bf16 maps take 2 bytes per element: a map sized for bf16 is too small for float32
        _noalloc(n2f, w, b, inp=torch.zeros(cin * H * W * 2, dtype=torch.uint8), cin=cin,
                 cout=cout, H=H, W=W)


def test_submit_device_image_must_match_planes(n2f):
    chk = n2f._check_device_image
    p1 = n2f.params()
    p3 = n2f.params(channels=3)
    pex = n2f.params(exact=1)
    assert n2f.image_planes(None) == 1 and n2f.image_planes(p1) == 1
    assert n2f.image_planes(p3) == 3 and n2f.image_planes(pex) == 2
    cases = [
        (torch.zeros((8, 8), dtype=torch.float64), p1, "dtype"),
        (torch.zeros((8, 8), dtype=torch.float16), p1, "dtype"),
        (torch.zeros((8,)), p1, "shape"),
        (torch.zeros((8, 8)), p3, "64 elements, 192 required"),   # one plane for three channels
        (torch.zeros((8, 8)), pex, "64 elements, 128 required"),  # Exact: the clean plane missing
        (torch.zeros((4, 8, 8)), p3, "256 elements, 192 required"),
        (torch.zeros((8, 16))[:, ::2], p1, "contiguous"),
        (torch.zeros((3, 8, 8)), p3, "on cpu"),  # right size, wrong device
        (torch.zeros((8, 8)), None, "on cpu"),
    ]
    for t, p, msg in cases:
        with pytest.raises(ValueError, match=msg):
            chk(t, p, 0)
