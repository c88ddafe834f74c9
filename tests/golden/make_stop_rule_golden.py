"""Writes ``stop_rule_plit_48.npz``: the FP64 oracle's whole stopping-rule run on one small cell
image, for the GPU tests to compare against.

Calls nothing but ``oracle`` (the FP64 restatement of the method) and the seeded input
generator. The run is the method as the Methods section states it: the literal channel widths
(32, 32, 64, 64, 128, 128, 256, 256), BCE, Adam with lr 0.001, four steps per epoch in the
table's pair order, full-image validation after every epoch, stop once 100 epochs pass without
a better validation score, output the average of the last 100 validation outputs.

Stored: the noisy and clean images, every epoch's validation score, the stop epoch, the best
epoch and score, the running output sum at the stop and the output, the oracle's thread count
and the CPU seconds the run took; and, as the method's own run-to-run spread on this image, the
stop epochs and output PSNRs of the same run from SPREAD_SEEDS further initial seeds. Run from
the repository root:

    python tests/golden/make_stop_rule_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2108_10209_gb300 import synth  # noqa: E402  (input generation only)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "stop_rule_plit_48.npz")
SIZE, IMAGE_SEED, INIT_SEED, PATIENCE = 48, 7, 0, 100
SPREAD_SEEDS = (1, 2, 3)


def main():
    clean, noisy = synth.image_cells(SIZE, SIZE, sigma=25.0 / 255.0, seed=IMAGE_SEED)
    job = oracle.Job(noisy, oracle.Params(widths=oracle.WIDTHS_PLIT, seed=INIT_SEED,
                                          patience=PATIENCE))
    t0 = time.time()
    scores = []
    while not job.info()["stopped"]:
        scores.append(job.epoch())
    secs = time.time() - t0
    info = job.info()
    out = job.run()  # the rule has fired: the output is the window's mean, no more epochs
    window = job.get(oracle.SUM).reshape(SIZE, SIZE)
    scores = np.array(scores)
    best_epoch = int(np.argmin(scores)) + 1
    assert info["epoch"] == best_epoch + PATIENCE and info["best"] == scores.min()
    spread_epochs, spread_psnr = [], []
    for seed in SPREAD_SEEDS:
        o, inf = oracle.denoise(noisy, oracle.Params(widths=oracle.WIDTHS_PLIT, seed=seed,
                                                     patience=PATIENCE))
        spread_epochs.append(inf["epoch"])
        spread_psnr.append(synth.psnr(o, clean))
    np.savez_compressed(
        OUT, noisy=noisy, clean=clean, scores=scores, stop_epoch=info["epoch"],
        best_epoch=best_epoch, best=info["best"], window_sum=window, out=out, patience=PATIENCE,
        init_seed=INIT_SEED, image_seed=IMAGE_SEED, steps=info["t"], threads=oracle.threads(),
        cpu_seconds=secs, spread_seeds=np.array(SPREAD_SEEDS),
        spread_stop_epochs=np.array(spread_epochs), spread_psnr=np.array(spread_psnr))
    print(f"stop epoch {info['epoch']} (best {best_epoch}, score {info['best']:.9g}), "
          f"{secs:.1f} s on {oracle.threads()} threads; PSNR {synth.psnr(out, clean):.3f} dB, "
          f"other seeds {spread_epochs} epochs, {[round(v, 3) for v in spread_psnr]} dB -> {OUT}")


if __name__ == "__main__":
    main()
