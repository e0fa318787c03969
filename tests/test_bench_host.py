"""Host-side pieces of bench.py that need no GPU: the clock record keeps only
the nvidia-smi samples taken inside the timed region and reports the
throttle reasons seen there; the reference arm (the oracle on the host cores)
prints one line of the bench contract."""
import datetime
import json
import os
import socket
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(t, sm, reason_cap="Not Active", reason_hw="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, 2070, 900.0, 0x0, {reason_hw}, Not Active, Not Active, {reason_cap}"


def test_clock_samples_outside_the_timed_region_are_ignored():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 1000.0, 1000.5
    c.lines = [_line(999.0, 345), _line(1000.1, 2070), _line(1000.3, 2055, reason_cap="Active"),
               _line(1001.5, 600, reason_hw="Active")]
    s = c.summary()
    assert s["samples"] == 2
    assert s["sm_mhz"] == (2070 + 2055) / 2 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]  # the idle sample's hw_slowdown is outside


def test_clock_summary_without_samples_in_the_region_says_so():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 1000.0, 1000.01
    c.lines = [_line(990.0, 2070)]
    s = c.summary()
    assert s["samples"] == 0 and "note" in s


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["unit"] == "points/s" and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("at_scale")


def test_reference_arm_under_torchrun_prints_from_rank_zero_only():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_cpu_baseline_reports_all_cores_and_one_thread():
    import numpy as np
    import oracle
    from paper_2303_14102_gb300 import synth
    w = synth.workload_at_scale(N=30_000)
    cores = oracle.num_threads()
    cb = bench.cpu_oracle_sample(w.X.numpy(), w.labels.numpy(), w.K, target_s=0.5)
    assert cb["kind"] == "oracle" and cb["cores"] == cores and cb["value"] > 0
    one = cb["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == "points/s"
    assert oracle.num_threads() == cores  # the thread count is put back
    ref = oracle.linear(w.X.numpy().astype(np.float64), w.labels.numpy(), w.K)
    assert abs(cb["S_sample"] - ref["S"]) < 1e-12


def test_traffic_record_is_used_only_for_unchanged_sources(tmp_path, monkeypatch):
    import torch
    rec = json.load(open(bench.TRAFFIC_RECORD))
    entry = rec["k_score_tc"]
    assert set(entry) >= {"D", "K", "rows", "dram_bytes", "sources", "sha256", "profile"}
    assert os.path.exists(os.path.join(ROOT, entry["profile"]))
    t, why = bench.measured_traffic("k_score_tc (pass 2, tcgen05)", 10_000_000, 64, 100, torch.float32)
    if bench.source_digest(entry["sources"]) == entry["sha256"]:
        assert t == entry["dram_bytes"] / entry["rows"] * 10_000_000 and "ncu" in why
    else:
        assert t is None and "changed" in why
    # a record whose sources no longer hash the same is not used
    bad = dict(rec, k_score_tc=dict(entry, sha256="0" * 64))
    p = tmp_path / "rec.json"
    p.write_text(json.dumps(bad))
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(p))
    t, why = bench.measured_traffic("k_score_tc (pass 2, tcgen05)", 10_000_000, 64, 100, torch.float32)
    assert t is None and "changed" in why
    # nor one of another shape
    t, why = bench.measured_traffic("k_score_tc (pass 2, tcgen05)", 10_000_000, 32, 100, torch.float32)
    assert t is None
