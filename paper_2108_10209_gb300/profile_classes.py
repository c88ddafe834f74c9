"""Live GPU time per kernel class over one image's whole run (build the library first).

    python -m paper_2108_10209_gb300.profile_classes [--precision 0|1] [--widths 0|1] [--size N]

One synthetic cell image (Gaussian noise, sigma 25/255) is denoised with the stopping rule once
per kernel class, each time in a fresh context whose `profile_kernel` is that class: the library
then brackets every launch of the class with CUDA events on the job's stream (event-record nodes
of the captured epoch graph) and reports their summed time, launch count and algorithmic FLOP.
A first run tunes the launch configurations, as bench.py's default run does. Prints one JSON
object: per class its time (ms), its share of the job's compute time, its launches and, for the
tensor-core classes, the achieved FP32-equivalent (float32 form) or bf16 TFLOP/s."""
import argparse
import json

import numpy as np

from . import n2f, synth

CLASSES = {1: "forward", 2: "dgrad", 3: "wgrad", 4: "first layer", 5: "head", 6: "adam"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", type=int, default=0, help="0 float32, 1 bf16")
    ap.add_argument("--widths", type=int, default=0, help="0 literal widths, 1 constant 64")
    ap.add_argument("--size", type=int, default=512)
    args = ap.parse_args()
    _, noisy = synth.image_cells(args.size, args.size, sigma=25 / 255, seed=1)
    x = noisy.astype(np.float32)
    p = n2f.params(seed=0, precision=args.precision, widths=args.widths)
    with n2f.Context(autotune=True) as ctx:  # loads the kernels and tunes the launches
        n2f.denoise(x, p, ctx)
    out, compute_ms, epochs = {}, None, None
    for k, name in CLASSES.items():
        with n2f.Context(profile_kernel=k, autotune=True) as ctx:
            j = ctx.submit(x, p)
            ctx.wait(j)
            st = ctx.poll(j)
            ctx.result(j, x.shape)
            s = ctx.stats()
        if compute_ms is None:
            compute_ms, epochs = st.compute_ms, st.epoch
        ms = s["prof_ms"]
        out[name] = {"ms": round(ms, 1), "share_pct": round(100 * ms / st.compute_ms, 1),
                     "launches": s["prof_launches"],
                     "tflops": round(s["prof_flops"] / (ms / 1e3) / 1e12, 1) if ms else 0.0}
    print(json.dumps({"precision": args.precision, "widths": args.widths, "size": args.size,
                      "epochs": epochs, "compute_ms": round(compute_ms, 1), "classes": out},
                     indent=1))


if __name__ == "__main__":
    main()
