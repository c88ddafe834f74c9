"""The stopping rule end to end against the FP64 oracle (Methods, validation paragraph: validate on
the full image after every epoch, stop once 100 epochs pass without a better score, output the
average of the last 100 validation outputs).

A free-running float32 job cannot follow the FP64 oracle's trajectory through a whole run: the
training is chaotic. Measured on the 32x32 blob image with eight 64-channel layers, the float32
CUDA-core engine's validation score is within 2e-8 of the oracle's after one epoch, 4e-5 after
ten, 2e-2 after thirty, and the run stops at epoch 144 where the oracle stops at 152 (the
tensor-core float32 form: 167). So the whole run is compared epoch by epoch from the oracle's own
state ("forced"): before every epoch the GPU trainer is loaded with the oracle's weights, Adam
moments and step count, best score, epoch and since counters, running output sum and best output
(rounded to float32), runs one epoch with its own kernels, and must then agree with the oracle's
epoch:
  - the FP64 validation scores within SCORE_REL's bars (relative difference: median, 90th
    percentile and largest over the run);
  - the decision (new best or not) and the since / stopped counters identical, except where the
    best so far lies between the GPU's and the oracle's score (a near tie: either decision is
    correct for that score);
  - the validation output V and the running sum S within V_MAXABS's bars;
  - at the oracle's stop epoch the rule fires on the GPU too, and the output (the window mean)
    is within the fixed-run bar: max-abs 2e-3 and 0.05 dB PSNR.
The free-running job is checked for what is unique to it: its history ring holds its own scores,
the oracle's stopping rule replayed on them fires where the GPU's fired, the first epoch (before
the trajectories separate) matches the oracle's golden run, and the final quality lies within
the oracle's own spread over initial seeds.
"""
import os

import numpy as np
import pytest

import oracle
from gpu_util import MAXABS_TOL, PSNR_TOL

pytestmark = pytest.mark.gpu

# One epoch (four Adam steps and a full-image forward) from the oracle's state rounded to float32.
# The one-epoch difference is heavy-tailed: most epochs agree closely, but the state is
# occasionally sensitive (late in the run, as the network starts to fit the noise) and four steps
# then amplify rounding differences. Measured (24x24 literal widths and 32x32 constant 64, about
# 130-150 epochs each): float32 scores median 2e-6 to 6e-6, 90th percentile up to 3e-5, largest
# 1e-3 (CUDA-core engine: median 3e-8, largest 7e-5); V max-abs 90th percentile up to 1.1e-4,
# largest 3.6e-3; bf16 scores median 5e-4, largest 5.5e-2, V largest 0.18. The bars below sit a
# few times above those figures: bars on the median and the 90th percentile hold the bulk of the
# epochs tight, the largest-value bars bound the sensitive ones.
SCORE_REL = {0: dict(median=2e-5, p90=1e-4, max=3e-3), 1: dict(median=2e-3, p90=1e-2, max=0.15)}
V_MAXABS = {0: dict(p90=5e-4, max=1e-2), 1: dict(p90=3e-2, max=0.5)}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "stop_rule_plit_48.npz")


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


def _psnr(a, ref):
    from paper_2108_10209_gb300 import synth
    return synth.psnr(a, ref)


def forced_run(n2f, noisy, ow, widths, engine, precision=0, patience=100, incl_best=False):
    """Runs the oracle freely to its stop and the GPU trainer one epoch at a time from the
    oracle's state; returns the per-epoch records and both outputs."""
    job = oracle.Job(noisy, oracle.Params(widths=ow, seed=0, patience=patience,
                                          incl_best=incl_best))
    tr = n2f.Trainer(noisy, n2f.params(seed=0, widths=widths, engine=engine, precision=precision,
                                       patience=patience, incl_best=int(incl_best)))
    rec = []
    while True:
        info = job.info()
        for what_g, what_o in ((n2f.N2F_X_THETA, oracle.THETA), (n2f.N2F_X_ADAM_M, oracle.ADAM_M),
                               (n2f.N2F_X_ADAM_V, oracle.ADAM_V), (n2f.N2F_X_SUM, oracle.SUM),
                               (n2f.N2F_X_VBEST, oracle.VBEST)):
            tr.import_(what_g, job.get(what_o))
        tr.set_progress(info["t"], info["epoch"], info["since"], info["best"])
        s_before = job.get(oracle.SUM)
        score_o = job.epoch()
        after = job.info()
        tr.epoch()
        st = tr.status()
        new_o = after["since"] == 0 and after["best"] == score_o
        v_o = job.get(oracle.VBEST) if new_o else job.get(oracle.SUM) - s_before
        best_prev = info["best"]
        # the decisions may differ only where the best so far lies between the two scores
        flip_ok = np.isfinite(best_prev) and min(score_o, st.last_mse) <= best_prev <= max(
            score_o, st.last_mse)
        rec.append(dict(
            epoch=after["epoch"], score_o=score_o, score_g=st.last_mse, tie=bool(flip_ok),
            same=(st.since == after["since"] and st.epoch == after["epoch"]
                  and bool(st.stopped) == after["stopped"]),
            v_err=float(np.max(np.abs(tr.export(n2f.N2F_X_VAL) - v_o))),
            s_err=float(np.max(np.abs(tr.export(n2f.N2F_X_SUM) - job.get(oracle.SUM)))),
            gpu_stopped=st.stopped))
        if after["stopped"]:
            break
    tr.finish()
    out_g = tr.export(n2f.N2F_X_OUT).reshape(noisy.shape)
    out_o = job.run()  # the rule has fired: the window's mean, no further epoch
    hist = tr.export(n2f.N2F_X_HIST)
    return rec, out_g, out_o, hist


def check_forced(rec, out_g, out_o, hist, clean, precision, patience):
    sb, vb = SCORE_REL[precision], V_MAXABS[precision]
    rel = np.array([abs(r["score_g"] - r["score_o"]) / r["score_o"] for r in rec])
    ties = [r["epoch"] for r in rec if r["tie"]]
    v_err = np.array([r["v_err"] for r in rec])
    # S differs by the whole window where a near tie flipped the decision (reset or add)
    s_err = np.array([r["s_err"] for r in rec if not r["tie"]])
    dpsnr = _psnr(out_g, clean) - _psnr(out_o, clean)
    maxabs = float(np.max(np.abs(out_g - out_o)))
    print(f"{len(rec)} epochs: score rel median {np.median(rel):.1e} p90 "
          f"{np.percentile(rel, 90):.1e} max {rel.max():.1e}; V max-abs p90 "
          f"{np.percentile(v_err, 90):.1e} max {v_err.max():.1e}; S max-abs {s_err.max():.1e}; "
          f"near ties at {ties}; output dPSNR {dpsnr:+.6f} dB, max-abs {maxabs:.1e}")
    assert np.median(rel) <= sb["median"] and np.percentile(rel, 90) <= sb["p90"]
    assert rel.max() <= sb["max"]
    assert np.percentile(v_err, 90) <= vb["p90"] and v_err.max() <= vb["max"]
    # S = the oracle's sum so far + this epoch's V (or V, or 0, at a new best)
    assert s_err.max() <= vb["max"]
    # identical decisions and counters wherever the best did not fall between the two scores
    for r in rec:
        if not r["tie"]:
            assert r["same"], r
    assert len(ties) <= max(2, len(rec) // 20)
    # the rule fired at the oracle's stop epoch on the GPU too
    assert rec[-1]["gpu_stopped"] == 1 or rec[-1]["tie"]
    assert len(rec) >= patience + 1
    if precision == 0:
        assert maxabs <= MAXABS_TOL and abs(dpsnr) <= PSNR_TOL
    else:
        assert maxabs <= 5e-2 and abs(dpsnr) <= 0.5
    # the device history ring holds the GPU's own score of every epoch, in order
    assert hist.size == len(rec)
    assert np.array_equal(hist, np.array([r["score_g"] for r in rec]))


def test_forced_run_literal_widths(n2f):
    """Literal widths (32 ... 256), patience 100, the production float32 form (tensor cores),
    on a 24x24 cell image (sub-images 24x12 and 12x24: partial tiles)."""
    from paper_2108_10209_gb300 import synth
    clean, noisy = synth.image_cells(24, 24, seed=5)
    rec, out_g, out_o, hist = forced_run(n2f, noisy, oracle.WIDTHS_PLIT, n2f.N2F_WIDTHS_PLIT,
                                         n2f.N2F_ENGINE_TC)
    check_forced(rec, out_g, out_o, hist, clean, 0, 100)


@pytest.mark.parametrize("engine", [1, 2])
def test_forced_run_w64(n2f, engine):
    """Eight 64-channel layers, patience 100, CUDA-core and tensor-core engines, on the 32x32
    blob image of the fixed-step case."""
    from paper_2108_10209_gb300 import synth
    clean, noisy = synth.image_small(seed=0)
    rec, out_g, out_o, hist = forced_run(n2f, noisy, oracle.WIDTHS_W64, n2f.N2F_WIDTHS_W64, engine)
    check_forced(rec, out_g, out_o, hist, clean, 0, 100)


def test_forced_run_bf16(n2f):
    """The bf16 form, literal widths, patience 100, at its own per-epoch bars."""
    from paper_2108_10209_gb300 import synth
    clean, noisy = synth.image_cells(24, 24, seed=5)
    rec, out_g, out_o, hist = forced_run(n2f, noisy, oracle.WIDTHS_PLIT, n2f.N2F_WIDTHS_PLIT,
                                         n2f.N2F_ENGINE_TC, precision=n2f.N2F_BF16)
    check_forced(rec, out_g, out_o, hist, clean, 1, 100)


@pytest.mark.parametrize("incl_best", [False, True])
def test_forced_run_short_patience_both_windows(n2f, incl_best):
    """Both readings of the averaging window (the epochs after the best, or with it) on a
    16x16 image with patience 6."""
    from paper_2108_10209_gb300 import synth
    clean = synth.blobs(16, 16, seed=3)
    noisy = (clean + synth.rng(4).normal(0, 0.1, clean.shape)).astype(np.float32).astype(np.float64)
    rec, out_g, out_o, hist = forced_run(n2f, noisy, oracle.WIDTHS_W64, n2f.N2F_WIDTHS_W64,
                                         n2f.N2F_ENGINE_AUTO, patience=6, incl_best=incl_best)
    check_forced(rec, out_g, out_o, hist, clean, 0, 6)


def test_free_run_against_the_oracle_golden(n2f):
    """A free-running job through the job API on the 48x48 golden image (literal widths,
    patience 100): its validation history, its own decisions, its first epoch against the
    oracle's, and its output quality against the oracle's own spread over initial seeds."""
    g = np.load(GOLDEN)
    noisy, clean = g["noisy"], g["clean"]
    p = n2f.params(seed=int(g["init_seed"]), patience=int(g["patience"]))
    with n2f.Context() as ctx:
        j = ctx.submit(noisy.astype(np.float32), p)
        assert ctx.wait(j, 600000) == n2f.N2F_OK
        st = ctx.poll(j)
        assert st.state == n2f.N2F_DONE and st.stopped == 1
        hist, first = ctx.history(j)
        out = ctx.result(j, noisy.shape).astype(np.float64)
    # one score per epoch, from the first
    assert first == 1 and hist.size == st.epoch and np.all(np.isfinite(hist))
    # the oracle's stopping rule replayed on the GPU's own scores takes the GPU's decisions
    rule = oracle.StopRule(patience=int(g["patience"]))
    fired = []
    for s in hist:
        rule.update(s)
        fired.append(rule.stopped)
    assert fired[-1] and not any(fired[:-1])
    assert rule.best == st.best_mse and int(np.argmin(hist)) + 1 == st.epoch - int(g["patience"])
    assert st.last_mse == hist[-1]
    # epoch 1 starts from bit-identical weights: its score is within the one-epoch bar
    assert abs(hist[0] - g["scores"][0]) <= SCORE_REL[0]["max"] * g["scores"][0]
    # the run's quality: a free run's trajectory is one sample of the method's run-to-run
    # variation (a late new best prolongs a run into overfitting: stops from 150 to 256 epochs
    # have been seen on this image), so its PSNR is held to the oracle's own spread over
    # initial seeds (the golden run and three more, each FP64 to its stop): within that range
    # widened by its width on each side
    orc = np.concatenate([[_psnr(g["out"], clean)], g["spread_psnr"]])
    p_gpu, p_noisy = _psnr(out, clean), _psnr(noisy, clean)
    print(f"free run: GPU stop {st.epoch} (oracle {int(g['stop_epoch'])}, other seeds "
          f"{list(g['spread_stop_epochs'])}), PSNR GPU {p_gpu:.3f}, oracle seeds "
          f"{np.round(orc, 3).tolist()}, noisy {p_noisy:.3f} dB; first-epoch score rel "
          f"{abs(hist[0] - g['scores'][0]) / g['scores'][0]:.2e}")
    width = orc.max() - orc.min()
    assert orc.min() - width <= p_gpu <= orc.max() + width
    assert p_gpu > p_noisy + 3.0
