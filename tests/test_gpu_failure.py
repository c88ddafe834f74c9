"""Failure detection without a GPU fault: a kernel waits on a barrier that nothing completes,
with the bounded wait of the tensor-core kernels; the wait must give up after its limit, the
kernel report the time-out through its error word, and the context stay usable."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


@pytest.mark.parametrize("limit_ms", [50, 300])
def test_bounded_wait_times_out_and_the_context_survives(n2f, limit_ms):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = n2f.wait_probe(limit_ms)
    dt = (time.perf_counter() - t0) * 1e3
    assert rc == n2f.N2F_ETIMEDOUT
    assert limit_ms <= dt < limit_ms + 2000
    # the context still runs work: the gather of a small image, checked against numpy
    x = np.arange(64, dtype=np.float32).reshape(8, 8)
    ue, uo, le, lo = [t.cpu().numpy() for t in n2f.checker_gather(torch.tensor(x, device="cuda"))]
    assert np.array_equal(ue[0], x[0, 0::2]) and np.array_equal(uo[0], x[0, 1::2])
    assert np.array_equal(ue[1], x[1, 1::2]) and np.array_equal(uo[1], x[1, 0::2])


def test_limit_out_of_range_is_rejected(n2f):
    assert n2f.wait_probe(0) == n2f.N2F_EINVAL
    assert n2f.wait_probe(20000) == n2f.N2F_EINVAL
