#!/usr/bin/env python
"""Throughput benchmark of the Noise2Fast per-image path: denoised images/s and per-image
latency (p50/p99), one JSON line on rank 0.

A step is one image taken through the whole path (upload, checkerboard gather, training on the
four pairs until the stopping rule fires, full-image validation each epoch, output averaging,
result). Default workload: 512x512 synthetic ellipse "cells" with Gaussian noise sigma 25/255 and
50/255 alternating, float32 plain form, the literal-width network, one image at a time.

  value   images/s from device time with the input resident: per image, CUDA events on the
          job's stream from "input uploaded" to "result ready"; summed over the K images, max
          over ranks.
  e2e     the same images through the public C ABI with host buffers (n2f_submit / n2f_result):
          host wall time from submit to result, including the pinned-staging copy, H2D and D2H.
  roofline  the profiled kernel class, timed per launch with CUDA events on its stream.
  cpu_baseline  the FP64 oracle on the host cores over a bounded sample (one epoch on a 128x128
          crop), extrapolated to the whole image at the shortest run the stopping rule allows.

--impl reference times the oracle the same way (no GPU work) and prints the same kind of line.
Multi-GPU (torchrun): images are sharded across ranks, no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "denoised images/s (p50/p99 latency per image)"
UNIT = "images/s"
WIDTH_NAMES = {0: "32-32-64-64-128-128-256-256", 1: "64x8"}
CLASS_NAMES = {1: "conv3x3_fwd", 2: "conv3x3_dgrad", 3: "conv3x3_wgrad", 4: "conv1_fwd",
               5: "head", 6: "adam", 7: "k_conv_tc (forward + dgrad)"}
MIN_EPOCHS = 101  # shortest run the stopping rule allows: one best epoch + 100 without gain


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def image_for(step: int, rank: int, size: int):
    from paper_2108_10209_gb300 import synth
    sigma = (25.0 if step % 2 == 0 else 50.0) / 255.0
    return synth.image_cells(size, size, sigma=sigma, seed=1_000_000 + rank * 10_000 + step)


# ---------------------------------------------------------------------------- clocks ---------

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        clk = sorted(r[0] for r in rows)
        return {"sm_mhz": clk[len(clk) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- CPU oracle -----

def host_cores() -> int:
    """Cores this process may run on (its affinity set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_threads() -> int:
    """Threads the oracle's parallel loops actually use."""
    import oracle
    return oracle.threads()


def oracle_epoch_seconds(noisy, widths: int, crop: int = 128):
    """Wall time of one oracle epoch (4 steps + validation) on the top-left crop x crop."""
    os.environ.setdefault("OMP_NUM_THREADS", str(host_cores()))
    import oracle
    ow = oracle.WIDTHS_PLIT if widths == 0 else oracle.WIDTHS_W64
    job = oracle.Job(noisy[:crop, :crop], oracle.Params(widths=ow, seed=0))
    t0 = time.perf_counter()
    job.epoch()
    return time.perf_counter() - t0


def oracle_whole_run(widths: int, side: int = 24):
    """One whole stopping-rule run (patience 100) of the FP64 oracle on a side x side cell
    image, timed on the host cores: the measured counterpart of the extrapolation."""
    os.environ.setdefault("OMP_NUM_THREADS", str(host_cores()))
    import oracle
    from paper_2108_10209_gb300 import synth
    ow = oracle.WIDTHS_PLIT if widths == 0 else oracle.WIDTHS_W64
    _, noisy = synth.image_cells(side, side, seed=5)
    t0 = time.perf_counter()
    _, info = oracle.denoise(noisy, oracle.Params(widths=ow, seed=0))
    secs = time.perf_counter() - t0
    return {"image": [side, side], "epochs": info["epoch"], "seconds": secs,
            "images_per_s": 1.0 / secs,
            "us_per_pixel_epoch": secs / (info["epoch"] * side * side) * 1e6}


def cpu_baseline(noisy, size: int, widths: int, crop: int = 128, reps: int = 1,
                 whole_run: bool = True):
    ts = [oracle_epoch_seconds(noisy, widths, crop) for _ in range(reps)]
    t = min(ts)
    scale = (size * size) / float(crop * crop)
    ips = 1.0 / (MIN_EPOCHS * scale * t)
    out = {"value": ips, "unit": UNIT, "cores": oracle_threads(),
           "kind": "oracle",
           "sample": (f"one epoch (4 training steps + validation) of the FP64 oracle on a "
                      f"{crop}x{crop} crop: {t:.2f} s; scaled by pixel count x{scale:.0f} to the "
                      f"{size}x{size} image and by {MIN_EPOCHS} epochs, the shortest run the "
                      f"stopping rule allows (real runs are longer, so this overstates the "
                      f"oracle)")}
    if whole_run:
        out["whole_run_measured"] = oracle_whole_run(widths)
    return out


# ---------------------------------------------------------------------------- peaks ----------

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# the sources of the conv kernel whose DRAM traffic profiles/traffic.json records
CONV_SOURCES = ("conv_tc.cu", "tc_common.cuh", "f16_split.cuh", "tc_ptx.cuh", "tc_layout.cuh",
                "cg_util.cuh")


def kernel_source_hash(files=CONV_SOURCES):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2108_10209_gb300", "csrc")
    for f in files:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(kclass: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if its kernels are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        recs = json.load(open(path))
    except Exception:
        return None
    r = recs.get(f"{kclass}|{workload}")
    if not r or r.get("source_hash") != kernel_source_hash():
        return None
    return r.get("dram_bytes_per_launch")


def roofline(stats, kclass: int, precision: int, engine_tc: bool, workload: str):
    pk, src = peaks()
    n = stats["prof_launches"]
    if not n or stats["prof_ms"] <= 0:
        return None
    avg_s = stats["prof_ms"] / n / 1e3
    flops = stats["prof_flops"] / n
    bytes_ = stats["prof_bytes"] / n
    name = CLASS_NAMES.get(kclass, str(kclass))
    if kclass in (1, 2, 3, 7) and engine_tc:
        if precision == 1:
            peak, note = pk["bf16_tflops_sustained"], f"bf16 dense sustained, {src}"
        else:
            peak = pk["bf16_tflops_sustained"] / 3.0
            note = ("float32 as two scaled fp16 parts, three fp16 products at the bf16 dense "
                    f"rate: bf16 sustained / 3, {src}")
        rl = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s"}
    elif kclass in (1, 2, 3, 7):
        clk = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * clk * 1e6 / 1e12
        note = f"FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x {clk:.0f} MHz (unit counts x max clock)"
        rl = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s"}
    else:
        peak, note = pk["hbm_gbs"], f"HBM copy bandwidth, {src}"
        rl = {"bound": "hbm", "achieved": bytes_ / avg_s / 1e9, "peak": peak, "unit": "GB/s"}
    rl["frac"] = rl["achieved"] / rl["peak"]
    tr = traffic_record(name, workload)
    rl["traffic"] = tr
    rl.update({"kernel": name, "launches": n, "avg_launch_us": avg_s * 1e6,
               "algorithmic_per_launch": flops if rl["unit"] == "TFLOP/s" else bytes_,
               "peak_source": note})
    return rl


# ---------------------------------------------------------------------------- our arm -------

def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f

    size = args.size
    p = n2f.params(seed=0, precision=args.precision, widths=args.widths, engine=args.engine,
                   overlap=args.overlap)
    work = [image_for(i, rank, size) for i in range(args.warmup + args.steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    # the launches of every --profile-every-th epoch are timed for the roofline: timing every
    # launch of a step puts two event records around each one and costs the step several percent
    ctx = n2f.Context(device=local, max_slots=1, profile_kernel=args.profile_kernel,
                      autotune=bool(args.autotune), profile_every=args.profile_every)
    for i in range(args.warmup):
        j = ctx.submit(work[i][1].astype(np.float32), p)
        ctx.wait(j)
        ctx.result(j, (size, size))
    clocks = ClockSampler(local)
    st0 = ctx.stats()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    comp_ms, wall_ms, epochs, outs = [], [], [], []
    for i in range(args.warmup, args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        x = work[i][1].astype(np.float32)
        t0 = time.perf_counter()
        j = ctx.submit(x, p)
        ctx.wait(j)
        st = ctx.poll(j)
        out = ctx.result(j, x.shape)
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        comp_ms.append(st.compute_ms)
        epochs.append(st.epoch)
        assert st.state == n2f.N2F_DONE, st.as_dict()
        assert np.isfinite(out).all()
        outs.append(out)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    st1 = ctx.stats()
    overlap = None
    if not args.overlap:
        # the same images again, each epoch's validation beside the next epoch's training
        po = n2f.params(seed=0, precision=args.precision, widths=args.widths, engine=args.engine,
                        overlap=1)
        o_ms, same = [], True
        for k, i in enumerate(range(args.warmup, args.warmup + args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            x = work[i][1].astype(np.float32)
            j = ctx.submit(x, po)
            ctx.wait(j)
            st = ctx.poll(j)
            out = ctx.result(j, x.shape)
            assert st.state == n2f.N2F_DONE, st.as_dict()
            o_ms.append(st.compute_ms)
            same = same and st.epoch == epochs[k] and bool(np.array_equal(out, outs[k]))
        from paper_2108_10209_gb300 import dispatch
        o_dev_s, o_img = dispatch.aggregate(sum(o_ms) / 1e3, args.steps)
        overlap = {"value": o_img / o_dev_s, "unit": UNIT,
                   "epochs_per_s_mpx": sum(epochs) * size * size / 1e6 / (sum(o_ms) / 1e3),
                   "results_identical": same,
                   "note": "n2f_params.overlap = 1: each epoch's validation on a second stream "
                           "beside the next epoch's training (weights snapshot at the boundary); "
                           "same images, same stop epochs"}
    ctx.close()
    from paper_2108_10209_gb300 import dispatch
    tot_dev_s, n_img = dispatch.aggregate(sum(comp_ms) / 1e3, args.steps)
    tot_wall_s, _ = dispatch.aggregate(sum(wall_ms) / 1e3, args.steps)
    if rank != 0:
        return None
    stats = {k: st1[k] - st0[k] if isinstance(st1[k], (int, float)) else st1[k] for k in st1}
    workload = f"{size}x{size} cells fp{'32' if args.precision == 0 else 'bf16'} " \
               f"{WIDTH_NAMES[args.widths]} plain"
    rl = roofline(stats, args.profile_kernel, args.precision, args.engine != 1, workload)
    if rl is not None:
        rl["sample"] = (f"the class's launches in every {args.profile_every}th epoch of the timed "
                        "images (epochs 0, k, 2k, ...), CUDA events on the launching stream")
    q = sorted(comp_ms)
    line = {
        "metric": METRIC, "value": n_img / tot_dev_s, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_dev_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == 0 else "bf16 (f32 accumulate)",
        "data": "synthetic (ellipse cells + Gaussian noise, seeded)",
        "config": {"workload": f"{size}x{size} grayscale, Gaussian sigma 25/255 and 50/255 "
                               f"alternating, stopping rule (patience 100), one image at a time",
                   "image": [size, size], "widths": WIDTH_NAMES[args.widths],
                   "precision": "fp32" if args.precision == 0 else "bf16",
                   "engine": {0: "auto", 1: "simt", 2: "tcgen05"}[args.engine],
                   "jobs_in_flight": 1, "parallelism": f"images sharded over {ws} GPU(s)",
                   "l2": "256 MB buffer written between timed images; per-image working set "
                         "~0.8 GB is larger than L2"},
        "latency_ms": {"p50": q[len(q) // 2], "p99": q[min(len(q) - 1, int(0.99 * len(q)))],
                       "per_image": [round(v, 2) for v in comp_ms]},
        "epochs_per_image": epochs,
        "epochs_per_s_mpx": sum(epochs) * size * size / 1e6 / (sum(comp_ms) / 1e3),
        "e2e": {"value": n_img / tot_wall_s, "unit": UNIT,
                "h2d_bytes_per_step": size * size * 4, "d2h_bytes_per_step": size * size * 4},
        "gpu_launches": int(stats["kernel_launches"]),
        "roofline": rl,
        "clocks": clk,
        "paper_context": "under 45 s per 512x512 image on an RTX 5000 mobile GPU (Contribution "
                         "and Significance); other hardware and data, context only",
    }
    from paper_2108_10209_gb300 import synth
    line["psnr_db"] = [round(synth.psnr(o, work[args.warmup + k][0]), 3)
                       for k, o in enumerate(outs)]
    line["mpx_per_s"] = args.steps * size * size / 1e6 / tot_dev_s
    if overlap is not None:
        line["overlap_validation"] = overlap
    if args.compare_batch > 0 and args.precision == 0:
        line["bf16_batched"] = c3_batched(n2f, args.widths, args.c3_jobs)
        line["bf16_vs_fp32"] = bf16_vs_fp32(
            n2f, work[args.warmup:args.warmup + args.steps], outs, epochs, args.widths,
            args.compare_batch)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(work[args.warmup][1], size, args.widths)
    return line


# ---------------------------------------------------------------------------- batched / serving

def run_jobs(ctx, n2f, jobs, p_of, submit_times=None, u16=False):
    """Submits jobs (list of noisy float32 arrays, or uint16 arrays with u16=True, submitted
    through n2f_submit_u16), optionally at host times (seconds from start), waits for all,
    returns per-job dicts and the host/device makespans."""
    t0 = time.perf_counter()
    ids = []
    results = [None] * len(jobs)
    next_i = 0
    while next_i < len(jobs):
        if submit_times is not None:
            wait = submit_times[next_i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.002))
                continue
        x = jobs[next_i]
        ids.append(ctx.submit_u16(x, p_of(next_i)) if u16 else ctx.submit(x, p_of(next_i)))
        next_i += 1
    for i, j in enumerate(ids):
        ctx.wait(j)
        st = ctx.poll(j)
        out = ctx.result(j, jobs[i].shape)
        assert st.state == n2f.N2F_DONE, st.as_dict()
        results[i] = dict(out=out, latency_ms=st.latency_ms, compute_ms=st.compute_ms,
                          device_ms=st.device_ms, t0=st.t_start_ms, t1=st.t_done_ms,
                          epoch=st.epoch, H=st.H, W=st.W)
    host_s = time.perf_counter() - t0
    dev_s = (max(r["t1"] for r in results) - min(r["t0"] for r in results)) / 1e3
    return results, host_s, dev_s


def pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(q * len(v)))]


def c3_batched(n2f, widths, n_jobs):
    """The batching form's workload: n_jobs independent jobs, sizes uniform over 256x256,
    512x512, 768x512 and 1024x768, sigma U[15, 50]/255, each with its own weights and the
    stopping rule, all submitted at once in the bf16 form (one stream and one epoch graph per
    job, autotuned launches). value: jobs / device makespan (first upload to last result)."""
    from paper_2108_10209_gb300 import synth
    jobs = synth.batch_jobs(n_jobs)
    imgs = [synth.image_cells(j["h"], j["w"], sigma=j["sigma"], seed=j["seed"]) for j in jobs]
    p = n2f.params(seed=0, precision=1, widths=widths)
    with n2f.Context(max_slots=n_jobs, autotune=True) as ctx:
        # warm-up: one job of every size (tunes each conv shape once, outside the timed region)
        seen = {}
        for j, im in zip(jobs, imgs):
            seen.setdefault((j["h"], j["w"]), im[1].astype("float32"))
        run_jobs(ctx, n2f, list(seen.values()), lambda _: n2f.params(seed=0, precision=1,
                                                                     widths=widths,
                                                                     fixed_steps=4))
        st0 = ctx.stats()
        res, host_s, dev_s = run_jobs(ctx, n2f, [im[1].astype("float32") for im in imgs],
                                      lambda _: p)
        st1 = ctx.stats()
    lat = [r["latency_ms"] for r in res]
    mpx = sum(r["H"] * r["W"] for r in res) / 1e6
    return {"value": len(res) / dev_s, "unit": UNIT, "precision": "bf16",
            "workload": f"{n_jobs} jobs, sizes uniform over 256x256, 512x512, 768x512, 1024x768, "
                        "sigma U[15,50]/255, stopping rule, all in flight",
            "jobs": len(res), "jobs_in_flight": n_jobs, "megapixels": round(mpx, 3),
            "mpx_per_s": mpx / dev_s,
            "e2e": {"value": len(res) / host_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(mpx * 4e6), "d2h_bytes_per_step": int(mpx * 4e6)},
            "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "max": max(lat)},
            "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
            "epochs": [r["epoch"] for r in res],
            "psnr_db": [round(synth.psnr(r["out"], imgs[k][0]), 3) for k, r in enumerate(res)]}


def bf16_vs_fp32(n2f, noisy_clean, fp32_outs, fp32_epochs, widths, batch):
    """The plain form's images again in the bf16 form (submitted together): PSNR per image
    against the float32 plain output, from free runs (each form stops where its own rule
    fires) and at the float32 run's stop epoch (the bf16 job capped there, its patience raised
    so that only the cap ends it: its output is then the mean of its validation outputs since
    its own best epoch, or that epoch's output)."""
    from paper_2108_10209_gb300 import synth
    imgs = [nc[1].astype("float32") for nc in noisy_clean]
    p_free = n2f.params(seed=0, precision=1, widths=widths)
    with n2f.Context(max_slots=batch, autotune=True) as ctx:
        free, host_s, dev_s = run_jobs(ctx, n2f, imgs, lambda _: p_free)
        forced, _, _ = run_jobs(ctx, n2f, imgs, lambda k: n2f.params(
            seed=0, precision=1, widths=widths, max_epochs=fp32_epochs[k],
            patience=fp32_epochs[k] + 1))
    ref = [synth.psnr(o, nc[0]) for o, nc in zip(fp32_outs, noisy_clean)]
    d_free = [synth.psnr(r["out"], nc[0]) - p for r, nc, p in zip(free, noisy_clean, ref)]
    d_forced = [synth.psnr(r["out"], nc[0]) - p for r, nc, p in zip(forced, noisy_clean, ref)]
    return {"images": len(imgs), "jobs_in_flight": batch,
            "value_free_runs": len(free) / dev_s, "unit": UNIT,
            "psnr_bf16_minus_fp32_db": [round(d, 4) for d in d_free],
            "epochs_bf16": [r["epoch"] for r in free], "epochs_fp32": list(fp32_epochs),
            "psnr_bf16_minus_fp32_at_fp32_stop_epoch_db": [round(d, 4) for d in d_forced],
            "max_abs_delta_db": {"free": max(abs(d) for d in d_free),
                                 "at_fp32_stop_epoch": max(abs(d) for d in d_forced)},
            "mean_delta_db": {"free": sum(d_free) / len(d_free),
                              "at_fp32_stop_epoch": sum(d_forced) / len(d_forced)}}


def run_batched(args, n2f):
    """64 independent jobs, sizes uniform over {256^2, 512^2, 768x512, 1024x768}, sigma
    U[15, 50]/255, all submitted at once; stopping rule each."""
    from paper_2108_10209_gb300 import synth
    jobs = synth.batch_jobs(args.jobs)
    if args.side:  # every job args.side x args.side instead of the size mix
        for j in jobs:
            j["h"] = j["w"] = args.side
    imgs = [synth.image_cells(j["h"], j["w"], sigma=j["sigma"], seed=j["seed"]) for j in jobs]
    p = n2f.params(seed=0, precision=args.precision, widths=args.widths, engine=args.engine)
    with n2f.Context(max_slots=args.jobs, group_size=args.group,
                     autotune=bool(args.autotune)) as ctx:
        warm = synth.image_cells(256, 256, seed=7)
        run_jobs(ctx, n2f, [warm[1].astype("float32")], lambda _: p)
        st0 = ctx.stats()
        res, host_s, dev_s = run_jobs(ctx, n2f, [im[1].astype("float32") for im in imgs],
                                      lambda _: p)
        st1 = ctx.stats()
    lat = [r["latency_ms"] for r in res]
    mpx = sum(r["H"] * r["W"] for r in res) / 1e6
    return {
        "metric": METRIC, "value": len(res) / dev_s, "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": dev_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (f32 accumulate)" if args.precision else "f32",
        "data": "synthetic (ellipse cells + Gaussian noise, seeded)",
        "config": {"workload": (f"{args.jobs} jobs of {args.side}x{args.side}" if args.side else
                                f"{args.jobs} jobs, sizes uniform over 256x256, 512x512, "
                                "768x512, 1024x768") +
                               ", sigma U[15,50]/255, stopping rule, all in flight",
                   "widths": WIDTH_NAMES[args.widths],
                   "precision": "bf16" if args.precision else "fp32", "jobs_in_flight": args.jobs,
                   "grouping": (f"lockstep groups of up to {args.group}: one grouped tensor-core "
                                "launch per conv phase, one epoch graph per group")
                   if args.group > 1 else "one stream and one epoch graph per job"},
        "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99)},
        "megapixels": mpx, "mpx_per_s": mpx / dev_s,
        "e2e": {"value": len(res) / host_s, "unit": UNIT,
                "h2d_bytes_per_step": int(mpx * 4e6), "d2h_bytes_per_step": int(mpx * 4e6)},
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "epochs": [r["epoch"] for r in res],
    }


def run_serving(args, n2f):
    """Poisson arrivals of 16-bit images (n2f_submit_u16: normalised on the device as
    value / 65535), square sides log-uniform in [256, max_side], Gaussian (sigma U[10, 50]/255)
    or Poisson-Gaussian (photon peak U(10, 100)) noise, admitted against the HBM budget as slots
    and memory free up. For every rate in --rates a stream of --jobs requests (the first
    --jobs of one seeded 1000-request stream, arrival times rescaled to the rate); latency =
    submit to DONE (host clock). Reported per rate: delivered images/s (completed / time from
    the first arrival to the last result) and p50 / p99 latency."""
    import numpy as np
    from paper_2108_10209_gb300 import synth
    rates = [float(r) for r in args.rates.split(",")]
    full = synth.serving_stream(1000, rate=1.0, smin=256, smax=args.max_side)
    base = full[:args.jobs]
    # the two largest images of the whole 1000-request stream join the shorter stream (at a
    # third and two thirds of it), so that every rate admits the largest sides
    big = sorted(full[args.jobs:], key=lambda r: -r["side"])[:2]
    for k, r in enumerate(big):
        base.insert((k + 1) * len(base) // 3, dict(r))
    t_unit = [r["t"] for r in full[:len(base)]]  # arrival times at 1 request/s
    imgs = [synth.to_u16(synth.make_serving_image(r)[0]) for r in base]
    clean = [synth.make_serving_image(r)[1] for r in base]
    p = n2f.params(seed=0, precision=args.precision, widths=args.widths, engine=args.engine)
    rows = []
    budget = int(args.budget_gb * (1 << 30))
    with n2f.Context(max_slots=args.slots, autotune=bool(args.autotune),
                     hbm_budget_bytes=budget) as ctx:
        warm = synth.to_u16(synth.image_cells(256, 256, seed=7)[1])
        run_jobs(ctx, n2f, [warm], lambda _: n2f.params(seed=0, precision=args.precision,
                                                        widths=args.widths, fixed_steps=4),
                 u16=True)
        for rate in rates:
            res, host_s, dev_s = run_jobs(ctx, n2f, imgs, lambda _: p,
                                          submit_times=[t / rate for t in t_unit], u16=True)
            lat = [r["latency_ms"] for r in res]
            rows.append({
                "rate_per_s": rate, "completed": len(res), "images_per_s": len(res) / host_s,
                "device_images_per_s": len(res) / dev_s,
                "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "max": max(lat)},
                "mpx": sum(r["H"] * r["W"] for r in res) / 1e6,
                "psnr_db_mean": float(np.mean([synth.psnr(r["out"], c)
                                               for r, c in zip(res, clean)]))})
            print(json.dumps({"rate": rate, **{k: v for k, v in rows[-1].items()
                                               if k != "rate_per_s"}}), file=sys.stderr,
                  flush=True)
    sides = [r["side"] for r in base]
    best = max(rows, key=lambda r: r["images_per_s"])
    return {
        "metric": METRIC, "value": best["images_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": len(rates), "warmup": 1, "ms_per_step": 1e3 / best["images_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (f32 accumulate)" if args.precision else "f32",
        "data": "synthetic (ellipse cells, Gaussian or Poisson-Gaussian, 16-bit)",
        "config": {"workload": f"{len(base)} requests per rate (the first {args.jobs} of a "
                               "seeded 1000-request stream and its two largest), Poisson "
                               "arrivals at "
                               f"{args.rates} /s, square sides log-uniform 256..{args.max_side}, "
                               "16-bit input, stopping rule",
                   "slots": args.slots, "hbm_budget_gb": args.budget_gb,
                   "widths": WIDTH_NAMES[args.widths],
                   "sides": {"min": min(sides), "max": max(sides),
                             "n_2048": sum(1 for x in sides if x >= 2000)}},
        "per_rate": rows,
    }


def run_zstack(args, n2f):
    """A live-cell-like Z-stack (Methods, fluorescence microscopy: 1024x1024 slices, Z = 20 um at
    0.5 um, denoised slice by slice and max projected): Poisson-Gaussian noise, every slice its
    own job, all in flight, the denoised slices gathered on the device and max projected there.
    Timed from the first submission to the projection back on the host."""
    import numpy as np
    import torch
    from paper_2108_10209_gb300 import synth
    Z, S = args.z, args.stack_side
    clean, noisy = synth.volume_cells(Z, S, S, seed=5_000_000)
    noisy32 = noisy.astype(np.float32)
    p = n2f.params(seed=0, precision=args.precision, widths=args.widths, engine=args.engine)
    with n2f.Context(max_slots=Z, group_size=args.group, autotune=bool(args.autotune)) as ctx:
        warm = synth.image_cells(256, 256, seed=7)[1].astype(np.float32)
        n2f.denoise(warm, p, ctx)
        st0 = ctx.stats()
        slices = torch.empty((Z, S, S), dtype=torch.float32, device="cuda")
        t0 = time.perf_counter()
        ids = [ctx.submit(noisy32[z], p) for z in range(Z)]
        sts = []
        for z, j in enumerate(ids):
            ctx.wait(j)
            sts.append(ctx.poll(j))
            assert sts[-1].state == n2f.N2F_DONE, sts[-1].as_dict()
            ctx.result_device(j, slices[z])
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        proj = n2f.max_project(slices)
        ev1.record()
        proj_host = proj.cpu().numpy()
        host_s = time.perf_counter() - t0
        st1 = ctx.stats()
    proj_ms = ev0.elapsed_time(ev1)
    dev_s = (max(s.t_done_ms for s in sts) - min(s.t_start_ms for s in sts) + proj_ms) / 1e3
    lat = [s.latency_ms for s in sts]
    ref = clean.max(axis=0)
    return {
        "metric": METRIC, "value": Z / dev_s, "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": dev_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (f32 accumulate)" if args.precision else "f32",
        "data": "synthetic (ellipsoid cells, Poisson-Gaussian per slice, seeded)",
        "config": {"workload": f"Z-stack of {Z} slices of {S}x{S}, Poisson-Gaussian (peak 30, "
                               "read 0.02), stopping rule per slice, all slices in flight, "
                               "max projection on the device",
                   "widths": WIDTH_NAMES[args.widths],
                   "precision": "bf16" if args.precision else "fp32"},
        "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "max": max(lat)},
        "projection_ms": proj_ms,
        "psnr_projection_db": {"noisy": synth.psnr(noisy.max(axis=0), ref),
                               "denoised": synth.psnr(proj_host.astype(np.float64), ref)},
        "e2e": {"value": Z / host_s, "unit": UNIT, "h2d_bytes_per_step": Z * S * S * 4,
                "d2h_bytes_per_step": S * S * 4},
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "epochs": [s.epoch for s in sts],
    }


def run_variants(args, n2f):
    """The Ablation Study's comparison on synthetic data (Table 1's Normal / Quad / Exact
    columns; the U-net column is out of scope) plus an RGB image denoised one channel per
    network (Fig. 2a caption). Every variant runs the same images (512x512 ellipse cells,
    Gaussian sigma 25/255 and 50/255) under the stopping rule; reported: images/s and PSNR."""
    import numpy as np
    from paper_2108_10209_gb300 import synth
    S = args.size
    imgs = [synth.image_cells(S, S, sigma=sg / 255.0, seed=6_000_000 + i)
            for i, sg in enumerate((25, 50))]
    base = dict(seed=0, precision=args.precision, widths=args.widths, engine=args.engine)
    rows = {}
    with n2f.Context() as ctx:
        n2f.denoise(synth.image_cells(256, 256, seed=7)[1].astype(np.float32), n2f.params(**base),
                    ctx)
        for name, kw, extra in (("normal", {}, False), ("quad", {"downsample": 1}, False),
                                ("exact", {"exact": 1}, True)):
            t0 = time.perf_counter()
            ps = []
            for clean, noisy in imgs:
                img = noisy.astype(np.float32)
                if extra:
                    img = np.stack([img, clean.astype(np.float32)])
                out = n2f.denoise(img, n2f.params(**base, **kw), ctx)
                ps.append(synth.psnr(out.astype(np.float64), clean))
            dt = time.perf_counter() - t0
            rows[name] = {"images_per_s": len(imgs) / dt, "psnr_db": ps}
        # RGB: three channels of independent cell images, one network per output channel
        cl = np.stack([synth.ellipses(S, S, seed=6_100_000 + c) for c in range(3)])
        no = (cl + synth.rng(6_200_000).normal(0, 25 / 255.0, cl.shape)).astype(np.float32)
        t0 = time.perf_counter()
        out = n2f.denoise_channels(no, n2f.params(**base), ctx)
        dt = time.perf_counter() - t0
        rows["rgb"] = {"images_per_s": 1.0 / dt,
                       "psnr_db": [synth.psnr(out[c].astype(np.float64), cl[c]) for c in range(3)],
                       "noisy_psnr_db": [synth.psnr(no[c].astype(np.float64), cl[c])
                                         for c in range(3)]}
    return {
        "metric": METRIC, "value": rows["normal"]["images_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": len(imgs), "warmup": 1, "ms_per_step": 1e3 / rows["normal"]["images_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (f32 accumulate)" if args.precision else "f32",
        "data": "synthetic (ellipse cells + Gaussian noise, seeded)",
        "config": {"workload": f"{S}x{S} cells, sigma 25/255 and 50/255: the method, Quad and "
                               "Exact ablations, and an RGB image (three networks)",
                   "widths": WIDTH_NAMES[args.widths],
                   "precision": "bf16" if args.precision else "fp32"},
        "variants": rows,
    }


# ---------------------------------------------------------------------------- reference arm -

def run_reference(args, ws, rank):
    if rank != 0:
        return None
    size = args.size
    work = [image_for(i, 0, size) for i in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        oracle_epoch_seconds(work[i][1], args.widths)
    ts = [oracle_epoch_seconds(work[i][1], args.widths)
          for i in range(args.warmup, args.warmup + args.steps)]
    scale = (size * size) / (128.0 * 128.0)
    per_img = [MIN_EPOCHS * scale * t for t in ts]
    value = len(per_img) / sum(per_img)
    cores = oracle_threads()
    sample = (f"each step: one epoch of the FP64 oracle on a 128x128 crop, scaled by pixel "
              f"count x{scale:.0f} and by {MIN_EPOCHS} epochs (the shortest stopping-rule run)")
    q = sorted(per_img)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(per_img) * 1e3 / len(per_img), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{size}x{size} grayscale, Gaussian sigma 25/255 and 50/255 "
                               f"alternating, stopping rule", "image": [size, size],
                   "widths": WIDTH_NAMES[args.widths]},
        "latency_ms": {"p50": q[len(q) // 2] * 1e3, "p99": q[-1] * 1e3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--precision", type=int, default=0, help="0 fp32, 1 bf16")
    ap.add_argument("--widths", type=int, default=0, help="0 literal widths, 1 constant 64")
    ap.add_argument("--engine", type=int, default=0, help="0 auto, 1 simt, 2 tcgen05")
    ap.add_argument("--profile-kernel", type=int, default=7,
                    help="kernel class timed for the roofline (7 conv forward+dgrad, 1 forward, "
                         "2 dgrad, 3 wgrad)")
    ap.add_argument("--overlap", type=int, default=0,
                    help="plain form: 1 validates each epoch beside the next epoch's training "
                         "(n2f_params.overlap; results identical), 0 in line (the default: "
                         "the roofline's per-launch times are then the kernels' own); with 0 the "
                         "timed images are also run once with 1 and reported beside")
    ap.add_argument("--profile-every", type=int, default=8,
                    help="plain form: time the profiled class's launches in every k-th epoch "
                         "(n2f_config.profile_every)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="plain",
                    choices=["plain", "batched", "serving", "zstack", "variants"])
    ap.add_argument("--compare-batch", type=int, default=16,
                    help="plain form: also run the timed images in the bf16 form, this many in "
                         "flight, and the batching form's job mix (0 = off)")
    ap.add_argument("--c3-jobs", type=int, default=64,
                    help="plain form: jobs of the batching form's size mix run in bf16")
    ap.add_argument("--jobs", type=int, default=64, help="batched / serving: number of images")
    ap.add_argument("--rates", default="1,2,5,10,20,50,100,200",
                    help="serving: arrival rates per second, one stream each")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: HBM admission budget")
    ap.add_argument("--slots", type=int, default=64, help="serving: jobs resident at once")
    ap.add_argument("--max-side", type=int, default=2048, help="serving: largest image side")
    ap.add_argument("--z", type=int, default=41, help="zstack: slices")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: tune each conv shape's launch choices (stages, CTAs per SM) once, "
                         "during warm-up; results are unchanged by them")
    ap.add_argument("--side", type=int, default=0,
                    help="batched: every job side x side instead of the size mix")
    ap.add_argument("--group", type=int, default=0,
                    help="batched / zstack: lockstep group size (n2f_config.group_size), 0 = off")
    ap.add_argument("--stack-side", type=int, default=1024, help="zstack: slice side")
    args = ap.parse_args()
    os.environ.setdefault("OMP_NUM_THREADS", str(host_cores()))
    ws, rank, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
    else:
        if ws > 1:
            import torch
            torch.cuda.set_device(local)
            torch.distributed.init_process_group("nccl")
        if args.form == "plain":
            line = run_ours(args, ws, rank, local)
        else:
            import torch
            torch.cuda.set_device(local)
            import __graft_entry__ as g
            g.build()
            from paper_2108_10209_gb300 import n2f
            run = {"batched": run_batched, "serving": run_serving, "zstack": run_zstack,
                   "variants": run_variants}[args.form]
            line = run(args, n2f)
            if rank != 0:
                line = None
        if ws > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
