"""Lockstep groups (n2f_config.group_size): jobs of identical parameters share one stream and
one epoch graph, the tensor-core forward and dgrad of each layer run as one persistent
launch over all members' tiles. Every tile is computed exactly as when the job runs alone, so
a member's result, stop epoch and step count equal its solo run bit for bit."""
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


def _img(h, w, seed):
    from paper_2108_10209_gb300 import synth
    clean = synth.blobs(h, w, seed=seed)
    return (clean + synth.rng(seed + 1).normal(0, 0.1, (h, w))).astype(np.float32)


def _run(n2f, imgs, p, **ctx_kw):
    with n2f.Context(**ctx_kw) as ctx:
        ids = [ctx.submit(x, p) for x in imgs]
        out = []
        for x, j in zip(imgs, ids):
            assert ctx.wait(j) == 0
            st = ctx.poll(j)
            assert st.state == n2f.N2F_DONE
            out.append((ctx.result(j, x.shape), st.epoch, st.steps))
        return out, ctx.stats()


@pytest.mark.parametrize("precision,widths", [(0, 0), (1, 0), (1, 1)])
def test_group_members_equal_solo_runs(n2f, precision, widths):
    # groups form among jobs of the same size: two groups of two here, plus one job alone
    imgs = [_img(40, 36, 1), _img(64, 64, 2), _img(40, 36, 3), _img(64, 64, 4), _img(33, 47, 5)]
    p = n2f.params(seed=5, patience=4, precision=precision, widths=widths)
    solo, st_solo = _run(n2f, imgs, p)
    grp, st = _run(n2f, imgs, p, group_size=8)
    for (a, ea, sa), (b, eb, sb) in zip(solo, grp):
        assert ea == eb and sa == sb
        assert np.array_equal(a, b)
    # the grouped forward / dgrad launches replace the members' own. A group keeps stepping
    # (its stopped members' kernels return at once) until its last member stops, so the counts
    # are compared where every member stops at the same epoch: the epoch cap
    pc = n2f.params(seed=5, patience=100, max_epochs=5, precision=precision, widths=widths)
    _, st_solo = _run(n2f, imgs, pc)
    _, st = _run(n2f, imgs, pc, group_size=8)
    assert st["kernel_launches"] < st_solo["kernel_launches"]


def test_groups_split_by_parameters(n2f):
    # Jobs with different parameters, and fixed-step jobs, run outside the group; all results
    # equal their solo runs.
    imgs = [_img(32, 32, 11), _img(32, 48, 12), _img(32, 32, 13)]
    ps = [n2f.params(seed=1, patience=3), n2f.params(seed=1, patience=3, precision=1),
          n2f.params(seed=1, fixed_steps=6)]
    with n2f.Context(group_size=4) as ctx:
        ids = [ctx.submit(x, p) for x, p in zip(imgs, ps)]
        got = []
        for x, j in zip(imgs, ids):
            assert ctx.wait(j) == 0
            got.append(ctx.result(j, x.shape))
    for x, p, g in zip(imgs, ps, got):
        assert np.array_equal(n2f.denoise(x, p), g)
