"""Overlapped validation (n2f_params.overlap = 1) gives the in-line schedule's results exactly.

With overlap a job validates each epoch's weights on a second stream, from a snapshot taken at
the epoch boundary, while the next epoch trains; the epoch that ran beside the validation that
stopped the job is discarded. Nothing about the method changes (Methods, validation paragraph:
a full-image validation after every epoch, stop after 100 epochs without improvement, output
the average of the last 100 validation outputs), so every observable of a job must equal the
in-line run's bit for bit: the result, the stop epoch, the step count, the scores, the loss of
the last step and the per-epoch history. The in-line runs are themselves checked against the
oracle by the stop-rule and parity tests."""
import numpy as np
import pytest

from paper_2108_10209_gb300 import n2f, synth

pytestmark = pytest.mark.gpu


def _image(h, w, seed, sigma=25):
    return synth.image_cells(h, w, sigma=sigma / 255.0, seed=seed)[1].astype(np.float32)


def _run(imgs, prm, use_graphs=True, lookahead=0, profile_kernel=0, group_size=0):
    """Submits every image at once; returns per image (result, status dict, history)."""
    out = []
    with n2f.Context(use_graphs=use_graphs, lookahead=lookahead, profile_kernel=profile_kernel,
                     group_size=group_size) as ctx:
        ids = [ctx.submit(x, prm) for x in imgs]
        for j, x in zip(ids, imgs):
            assert ctx.wait(j, 600000) == n2f.N2F_OK
            st = ctx.poll(j)
            assert st.state == n2f.N2F_DONE, st.as_dict()
            hist, first = ctx.history(j)
            out.append((ctx.result(j, x.shape), st.as_dict(), hist, first))
    return out


def _same(a, b):
    for (ra, sa, ha, fa), (rb, sb, hb, fb) in zip(a, b):
        assert np.array_equal(ra, rb)
        for k in ("epoch", "steps", "since", "stopped", "best_mse", "last_mse", "last_loss", "H",
                  "W"):
            assert sa[k] == sb[k], (k, sa[k], sb[k])
        assert fa == fb and np.array_equal(ha, hb)


@pytest.mark.parametrize("precision", [n2f.N2F_FP32, n2f.N2F_BF16])
def test_overlap_matches_in_line_under_the_stopping_rule(precision):
    # literal widths, patience 100: the rule fires on its own (about 150-250 epochs here)
    imgs = [_image(48, 64, seed=11)]
    base = dict(seed=5, precision=precision)
    inline = _run(imgs, n2f.params(**base))
    over = _run(imgs, n2f.params(**base, overlap=1))
    assert inline[0][1]["stopped"] == 1 and inline[0][1]["steps"] == 4 * inline[0][1]["epoch"]
    _same(inline, over)


def test_overlap_matches_in_line_without_graphs_and_at_the_epoch_cap():
    # stopped by max_epochs, kernels launched one by one, three epochs enqueued ahead
    imgs = [_image(40, 56, seed=12)]
    base = dict(seed=6, max_epochs=7)
    inline = _run(imgs, n2f.params(**base), use_graphs=False, lookahead=3)
    over = _run(imgs, n2f.params(**base, overlap=1), use_graphs=False, lookahead=3)
    assert inline[0][1]["epoch"] == 7 and inline[0][1]["stopped"] == 2
    _same(inline, over)


def test_overlap_with_several_jobs_in_flight_and_odd_sizes():
    # jobs of different sizes share the device; each equals its in-line run, also when the conv
    # launches are timed (event-record nodes on both streams of the epoch graph)
    imgs = [_image(33, 47, seed=13), _image(64, 40, seed=14, sigma=50), _image(50, 50, seed=15)]
    base = dict(seed=7, patience=20, widths=n2f.N2F_WIDTHS_W64)
    inline = _run(imgs, n2f.params(**base))
    _same(inline, _run(imgs, n2f.params(**base, overlap=1)))
    _same(inline, _run(imgs, n2f.params(**base, overlap=1), profile_kernel=n2f.N2F_K_CONV))


def test_overlap_is_ignored_by_fixed_step_jobs():
    imgs = [_image(32, 48, seed=16)]
    base = dict(seed=8, fixed_steps=9)
    _same(_run(imgs, n2f.params(**base)), _run(imgs, n2f.params(**base, overlap=1)))


def test_overlap_jobs_in_a_lockstep_group():
    # jobs that ask for overlap and join a lockstep group validate in line with their group; the
    # numbers are the same, so each result equals its solo overlapped run
    imgs = [_image(40, 48, seed=17), _image(40, 48, seed=18, sigma=50)]
    p = n2f.params(seed=9, patience=10, widths=n2f.N2F_WIDTHS_W64, overlap=1)
    _same(_run(imgs, p), _run(imgs, p, group_size=4))
