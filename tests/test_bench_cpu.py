"""bench.py's host logic on the CPU: the reference arm's JSON line (the FP64 oracle timed on the
host cores) and the roofline arithmetic of our arm's line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "images/s" and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["steps"] == 1
    cb = d["cpu_baseline"]
    # cores: the threads the oracle's parallel loops used, as the oracle itself reports them
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_conv_roofline_uses_the_form_ceiling(precision):
    # 10 launches of 48.7 GFLOP in 1.0 ms: 487 TFLOP/s achieved
    stats = {"prof_launches": 10, "prof_ms": 1.0, "prof_flops": 10 * 48.7e9, "prof_bytes": 0.0}
    rl = bench.roofline(stats, 7, precision, True, "none")
    pk, _ = bench.peaks()
    ceiling = pk["bf16_tflops_sustained"] / (3.0 if precision == 0 else 1.0)
    assert rl["bound"] == "tensor" and rl["unit"] == "TFLOP/s"
    assert rl["achieved"] == pytest.approx(487.0)
    assert rl["peak"] == pytest.approx(ceiling)
    assert rl["frac"] == pytest.approx(487.0 / ceiling)
    assert rl["traffic"] is None  # no record for this workload name


def test_memory_bound_roofline_is_against_hbm():
    stats = {"prof_launches": 4, "prof_ms": 2.0, "prof_flops": 0.0, "prof_bytes": 4 * 1e9}
    rl = bench.roofline(stats, 5, 0, True, "none")  # the head: 1 GB per launch in 0.5 ms
    pk, _ = bench.peaks()
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert rl["achieved"] == pytest.approx(2000.0)
    assert rl["frac"] == pytest.approx(2000.0 / pk["hbm_gbs"])


def test_traffic_record_is_keyed_on_the_conv_sources():
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, r in recs.items():
        kclass, workload = key.split("|", 1)
        expected = r["dram_bytes_per_launch"] if r["source_hash"] == bench.kernel_source_hash() \
            else None
        assert bench.traffic_record(kclass, workload) == expected


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_samples_give_median_max_and_active_reasons(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits rows of ClockSampler.FIELDS
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1995, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2032, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbled line",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    f = tmp_path / "clocks.csv"
    f.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = _DoneProc(), str(f)
    clk = cs.stop()
    assert clk["samples"] == 3 and clk["sm_mhz"] == 2032.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]
    assert not f.exists()


def test_clock_samples_report_a_thermal_slowdown(tmp_path):
    f = tmp_path / "clocks.csv"
    f.write_text("0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = _DoneProc(), str(f)
    assert cs.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_missing_sampler_is_reported():
    cs = bench.ClockSampler(0)
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    # two ranks on one node: rank 0 times the oracle and prints; rank 1 exits 0 without work
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    env = dict(os.environ, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps",
                        "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_cpu_baseline_scales_one_crop_epoch_to_a_whole_run(monkeypatch):
    # one epoch on a 128x128 crop taking t seconds stands for (512/128)^2 = 16 times the pixels
    # and MIN_EPOCHS = 101 epochs (one best epoch + 100 without improvement)
    monkeypatch.setattr(bench, "oracle_epoch_seconds", lambda noisy, widths, crop=128: 0.5)
    monkeypatch.setattr(bench, "oracle_whole_run", lambda widths: {"seconds": 1.0})
    cb = bench.cpu_baseline(None, 512, 0)
    assert cb["whole_run_measured"] == {"seconds": 1.0}
    assert bench.MIN_EPOCHS == 101
    assert cb["value"] == pytest.approx(1.0 / (101 * 16 * 0.5))
    assert cb["unit"] == "images/s" and cb["kind"] == "oracle" and cb["cores"] >= 1
    assert "128x128" in cb["sample"]


def test_oracle_whole_run_is_a_stopping_rule_run():
    # a whole run on a tiny image: the rule fires after at least 101 epochs, and the rate per
    # pixel-epoch follows from the measured seconds
    w = bench.oracle_whole_run(1, side=8)
    assert w["image"] == [8, 8] and w["epochs"] >= bench.MIN_EPOCHS and w["seconds"] > 0
    assert w["us_per_pixel_epoch"] == pytest.approx(w["seconds"] / (w["epochs"] * 64) * 1e6)
