"""Benchmark of the linear-complexity Silhouette on one GB300 (or N replicas).

Headline workload (one step = one pass of the whole forward hot path:
sil_aggregate + sil_score = pass 1, finalisation, pass 2, s_i and S):
  at_scale: N = 10,000,000 points, D = 64, K = 100 clusters, FP32 Gaussian
  blobs (centres U[-5,5]^D, sigma 1, truncated rank-Zipf(1.1) sizes, shuffled),
  squared Euclidean distance.
Metric: points/s (whole job).  Beside it, per pass: achieved HBM GB/s and the
roofline of the dominant kernel, the same step through host buffers (e2e),
the FP64 oracle's linear form on the host cores (cpu_baseline), and variant
lines (cosine, BF16 storage, fwd+bwd ms, batched labelings, the 1e8-point
precision workload) measured in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU runs (torchrun) are replicas: every rank scores its own copy of the
workload with no data-path collective ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Silhouette points/s & HBM GB/s, FP32 vs BF16 at |ΔS|≤1e-4; fwd+bwd ms"
WORKLOAD = {"workload": "at_scale Gaussian blobs, sq-Euclidean", "N": 10_000_000, "D": 64, "K": 100,
            "sizes": "rank-Zipf(1.1)", "storage": "fp32"}


def bench_config(N, D, world):
    """The `config` object of both arms' lines (the same workload)."""
    return dict(WORKLOAD, N=N, parallelism="replicas" if world > 1 else "single",
                l2=f"inputs ({N * (4 * D + 4) / 1e9:.2f} GB) larger than L2 (129 MB); no flush")


def oracle_full(X64, labels, K, metric, S_gpu):
    """|S_gpu - S| with S the FP64 oracle's linear form over every row."""
    import oracle
    ref = oracle.linear(X64, labels, K, metric)
    return {"dS_vs_oracle": abs(S_gpu - ref["S"]), "oracle_S": ref["S"], "rows": int(X64.shape[0]),
            "kind": "FP64 linear form over all rows"}


def oracle_sampled(X_dev, labels_dev, K, metric, s_gpu, S_gpu, col_scale=None, rows=20_000, seed=2030):
    """Error against the FP64 oracle where its linear form over every row would take minutes:
    FP64 aggregates of all rows, then the oracle's s_i of `rows` seeded rows against the GPU's.
    S_gpu is the mean of the GPU's s_i, so its distance from the oracle's full-N S is the mean of
    the per-row differences, which the paired sample estimates (bound = |mean| + 5 standard errors)."""
    import numpy as np
    import torch
    import oracle
    N, D = X_dev.shape

    def deq(t):
        x = t.detach().cpu().to(torch.float64)
        if col_scale is not None:
            x = x * col_scale.detach().cpu().to(torch.float64)[None, :]
        return x.numpy()

    count = np.zeros(K, np.int64)
    s1 = np.zeros((K, D), np.float64)
    s2 = np.zeros(K, np.float64)
    step = 4_000_000
    for lo in range(0, N, step):
        hi = min(N, lo + step)
        part = oracle.aggregate(deq(X_dev[lo:hi]), labels_dev[lo:hi].cpu().numpy(), K, metric)
        count += part[0]
        s1 += part[1]
        s2 += part[2]
    idx = np.sort(np.random.default_rng(seed).choice(N, min(rows, N), replace=False))
    it = torch.as_tensor(idx, device=X_dev.device)
    sub = oracle.linear(deq(X_dev[it]), labels_dev[it].cpu().numpy(), K, metric, agg=(count, s1, s2),
                        idx=np.arange(idx.shape[0]))
    diff = s_gpu[it].detach().cpu().double().numpy() - sub["s"]
    se = float(np.std(diff)) / np.sqrt(diff.size)
    return {"dS_vs_oracle": abs(float(np.mean(diff))) + 5 * se, "max_abs_ds_i": float(np.abs(diff).max()),
            "mean_ds_i": float(np.mean(diff)), "se_mean_ds_i": se,
            "S_minus_mean_s_i": abs(S_gpu - float(s_gpu.double().mean())), "rows": int(N),
            "rows_scored_by_oracle": int(idx.size),
            "kind": "bound |mean| + 5 SE of paired per-row differences (FP64 aggregates of all rows)"}


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "dram_traffic_at_scale.json")


def source_digest(paths):
    """sha256 over the named source files (repository-relative), in order."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kname, N, D, K, dtype):
    """DRAM bytes (read + write) of one launch of the dominant kernel, from the
    committed ncu capture of the same kernel on this recipe, scaled by rows --
    only while the kernel's sources are byte-identical to those captured."""
    import torch
    if not os.path.exists(TRAFFIC_RECORD):
        return None, "no ncu capture recorded"
    rec = json.load(open(TRAFFIC_RECORD)).get(kname.split(" ")[0])
    if rec is None or (D, K) != (rec["D"], rec["K"]) or dtype != torch.float32:
        return None, "no ncu capture of this kernel on this recipe"
    if source_digest(rec["sources"]) != rec["sha256"]:
        return None, "kernel sources changed since the ncu capture"
    return rec["dram_bytes"] / rec["rows"] * N, (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                                 f"launch at N = {rec['rows']}, scaled by rows ({rec['profile']})")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi samples (every 100 ms, time-stamped); summary() keeps those
    taken inside the timed region [t0, t1] (wall clock)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # nvidia-smi is sampling before the timed region starts
        except (FileNotFoundError, OSError):
            self.proc = None
        self.t0 = self.t1 = None
        return self

    def mark(self, start: bool):
        """Wall-clock bounds of the timed region."""
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, window=None):
        """Samples inside the timed region, or inside window = (t0, t1)."""
        import datetime
        rows = []
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = rows
        t0, t1 = window if window is not None else (self.t0, self.t1)
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {n for r in inside for n, v in zip(names, r[3]) if v.lower() == "active"}
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "no nvidia-smi sample fell inside the timed region"}
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside),
                "window": "timed region only" if window is None else "given window"}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_sample(X_host, labels_host, K, metric="sqeuclidean", target_s=12.0):
    """Time the FP64 oracle's linear form (aggregate + score) on a row sample."""
    import numpy as np
    import oracle
    M = min(200_000, X_host.shape[0])
    while True:
        Xs = X_host[:M].astype(np.float64)
        ls = labels_host[:M]
        t0 = time.perf_counter()
        r = oracle.linear(Xs, ls, K, metric)
        dt = time.perf_counter() - t0
        if dt * 3 > target_s or M >= X_host.shape[0]:
            break
        M = min(X_host.shape[0], int(M * max(2.0, target_s / max(dt, 1e-3) * 0.8)))
    cores = oracle.num_threads()
    # the same on one thread, beside the paper's single-thread timings
    m1 = min(M, 200_000)
    X1, l1 = X_host[:m1].astype(np.float64), labels_host[:m1]
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.linear(X1, l1, K, metric)
        d1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"value": M / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"first {M} rows of the workload as a dataset of their own: FP64 aggregates "
                      f"(Eq. 6/8) + linear scoring (Eq. 11) of every sampled point, {dt:.2f} s",
            "S_sample": r["S"],
            "single_thread": {"value": m1 / d1, "unit": "points/s", "cores": 1,
                              "sample": f"first {m1} rows, the same oracle on one thread, {d1:.2f} s"}}


def run_reference(args):
    """--impl reference: the FP64 oracle (linear form) on the host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2303_14102_gb300 import synth
    M = 300_000
    w = synth.workload_at_scale(device="cpu", N=M)  # same recipe and seed, first-M sample
    X = w.X.double().numpy()
    lab = w.labels.numpy()
    for _ in range(args.warmup):
        oracle.linear(X[:20000], lab[:20000], w.K)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.linear(X, lab, w.K)
    dt = time.perf_counter() - t0
    v = M * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(WORKLOAD["N"], WORKLOAD["D"], world),
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"each step scores the first {M} points of the at_scale recipe as a "
                                       f"dataset of their own: FP64 aggregates + linear scoring on the host "
                                       f"cores; points/s is rows scored / time"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def timed(fn, steps, stream):
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def num_sms_of(dev):
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def variant_lines(dev, steps, budget_s, pk_sustained, pk_sm_mhz):
    """Secondary measurements, each bounded in time."""
    import numpy as np
    import torch
    from paper_2303_14102_gb300 import sil, synth
    from paper_2303_14102_gb300.autograd import silhouette_loss
    out = {}
    t_start = time.time()

    def left():
        return budget_s - (time.time() - t_start)

    # precision workload (N=1e8, D=128, K=1000, centres at radius 1e3): the
    # same blobs stored in BF16, FP8-E4M3 with column scales, and FP32
    if left() > 0:
        w = synth.workload_precision(device=dev)
        lab, K = w.labels, w.K
        N = lab.shape[0]
        forms = {"bf16": (synth.to_bf16(w.X), None)}
        q, cs = synth.to_fp8_e4m3(w.X)
        forms["fp8_e4m3"] = (q, cs)
        forms["fp32"] = (w.X, None)
        del w
        torch.cuda.empty_cache()
        stream = torch.cuda.current_stream()
        res = {}
        for name, (Xs, sc) in forms.items():
            if left() <= 0:
                break
            st = sil.new_status(dev)
            agg = sil.aggregate(Xs, lab, K, col_scale=sc, status=st)
            sil.score(Xs, lab, K, agg, col_scale=sc, status=st)
            n = max(1, min(steps, 3))
            t1 = timed(lambda: sil.aggregate(Xs, lab, K, col_scale=sc, out=agg, status=st), n, stream) / n
            t2 = timed(lambda: sil.score(Xs, lab, K, agg, col_scale=sc, status=st), n, stream) / n
            r = sil.score(Xs, lab, K, agg, col_scale=sc, want_s=True, status=st)
            torch.cuda.synchronize()
            sil.check_status(st, "precision " + name)
            check = oracle_sampled(Xs, lab, K, "sqeuclidean", r.s, float(r.S.item()), col_scale=sc)
            plan = sil.tensor_plan(Xs.dtype, Xs.shape[1], K)
            entry = {"points_per_s": N / (t1 + t2), "ms": (t1 + t2) * 1e3, "pass1_ms": t1 * 1e3,
                     "pass2_ms": t2 * 1e3, "S": float(r.S.item()), "dS_vs_oracle": check["dS_vs_oracle"],
                     "oracle_check": check,
                     "pass1_hbm_gbs": Xs.numel() * Xs.element_size() / t1 / 1e9 + N * 4 / t1 / 1e9,
                     "pass2_useful_tflops": 2.0 * N * K * Xs.shape[1] / t2 / 1e12}
            if plan is not None:
                bk, nb = plan
                mmas = 3 if Xs.dtype == torch.float32 else 2  # BF16 hi/lo products per k-step
                mma_flops = 2.0 * N * bk * nb * 128 * mmas
                entry.update({"tensor_plan": {"block_k": bk, "blocks": nb, "mma_per_kstep": mmas},
                              "pass2_mma_tflops": mma_flops / t2 / 1e12,
                              "pass2_tensor_frac_of_measured_bf16": mma_flops / t2 / 1e12
                              / pk_sustained})
            res[name] = entry
            del r
        if "fp32" in res:
            for name in ("bf16", "fp8_e4m3"):
                if name in res:
                    res[name]["dS_vs_fp32_storage"] = abs(res[name]["S"] - res["fp32"]["S"])
        out["precision"] = dict(res, N=N, D=128, K=K)
        del forms, q, cs, lab
        torch.cuda.empty_cache()
    # fwd+bwd on the differentiation workload (N=1e6, D=256, K=1000 unit-normalised)
    if left() > 0:
        w = synth.workload_grad(device=dev)
        X, lab = w.X, w.labels
        for metric in ("sqeuclidean", "cosine"):
            def step():
                Xg = X.detach().requires_grad_(True)
                S = silhouette_loss(Xg, lab, w.K, metric)
                S.backward()
            step()
            n = max(1, min(steps, 3))
            s = timed(step, n, torch.cuda.current_stream())
            # the backward alone (dS/dX from the saved a_i, b_i, k*_i, the call
            # autograd's backward makes), 10 calls back to back: two reads of X
            # and one write of dX are its algorithmic bytes
            agg = sil.aggregate(X, lab, w.K, metric)
            rs = sil.score(X, lab, w.K, agg, metric, save=True)
            dX = torch.empty_like(X)
            sil.score_backward(X, lab, w.K, agg, metric, saved=rs.saved, out=dX)
            tb = timed(lambda: sil.score_backward(X, lab, w.K, agg, metric, saved=rs.saved, out=dX), 10,
                       torch.cuda.current_stream()) / 10
            del agg, rs, dX
            nbytes = 3.0 * X.shape[0] * X.shape[1] * 4
            rf = sil.silhouette(X, lab, w.K, metric, want_s=True)  # the forward's kernels, with s_i kept
            check = oracle_sampled(X, lab, w.K, metric, rf.s, float(rf.S.item()))
            out[f"fwd_bwd_grad_{metric}"] = {"ms": s / n * 1e3, "bwd_ms": tb * 1e3, "bwd_hbm_gbs": nbytes / tb / 1e9,
                                             "N": 1_000_000, "D": 256, "K": 1000,
                                             "dS_vs_oracle": check["dS_vs_oracle"], "oracle_check": check}
        del X, lab, w
        torch.cuda.empty_cache()
    # the exact (non-squared) Euclidean Silhouette by the quadratic method on
    # the at_scale recipe at 20,000 points (the size the oracle's brute force
    # checks in seconds); bound by the FP32 pipe: 3 D flop per pair (difference,
    # square, sum) plus a square root
    if left() > 0:
        import oracle
        w = synth.workload_at_scale(device=dev, N=20_000)
        X, lab, K = w.X, w.labels, w.K
        N, D = X.shape
        fn = lambda: sil.score_euclidean(X, lab, K)  # noqa: E731
        r = sil.score_euclidean(X, lab, K, want_s=True)
        n = max(3, min(steps, 20))
        fn()
        s = timed(fn, n, torch.cuda.current_stream()) / n
        ref = oracle.bruteforce(X.cpu().double().numpy(), lab.cpu().numpy(), K, "euclidean")
        Se = float(r.S.item())
        flops = 3.0 * D * N * N
        peak = num_sms_of(dev) * 128 * 2 * pk_sm_mhz * 1e6 / 1e12
        out["euclidean_exact_bruteforce"] = {
            "ms": s * 1e3, "points_per_s": N / s, "pairs_per_s": N * N / s, "N": N, "D": D, "K": K, "S": Se,
            "dS_vs_oracle": abs(Se - ref["S"]),
            "max_abs_ds_i_vs_oracle": float(np.abs(r.s.cpu().double().numpy() - ref["s"]).max()),
            "roofline": {"bound": "alu", "achieved": flops / s / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / s / 1e12 / peak,
                         "peak_source": "derived: SMs x 128 FP32 lanes x 2 flop x max SM clock",
                         "algorithmic": "3 D flop per ordered pair (N^2 pairs)"}}
        del X, lab, w
        torch.cuda.empty_cache()
    # batched labelings (N=2e6, D=32, B=256, k ~ U{2..512}): pass 1 and the
    # finalisation per labeling, then every labeling's pass 2 in ONE
    # tensor-core launch (+ the combine of the two-block labelings and the B
    # means), all captured once in a CUDA graph, one graph launch per step
    if left() > 0:
        X, labs, ks = synth.workload_batched(device=dev)
        # the one launch's plan (CTAs per labeling block, A buffers) picked by
        # measurement before timing
        t0 = time.perf_counter()
        tuned = sil.autotune_batched(X, labs, ks)
        t_tune = time.perf_counter() - t0
        one_launch = sil.serves_one_launch(X, labs, ks)
        # the same batch as one launch sequence per labeling (for comparison)
        import os as _os
        _os.environ["SIL_BATCH_PER_LABELING"] = "1"
        sil.score_batched(X, labs, ks)
        s_per = timed(lambda: sil.score_batched(X, labs, ks), 1, torch.cuda.current_stream())
        del _os.environ["SIL_BATCH_PER_LABELING"]
        sil.score_batched(X, labs, ks)
        s_loop = timed(lambda: sil.score_batched(X, labs, ks), 1, torch.cuda.current_stream())
        g = sil.BatchedGraph(X, labs, ks)
        g.run()
        s = timed(g.run, max(1, min(steps, 3)), torch.cuda.current_stream()) / max(1, min(steps, 3))
        S_all = g.run().cpu().numpy()
        import numpy as np
        import oracle
        X64 = X.cpu().double().numpy()
        order = np.argsort(ks)
        picks = sorted({0, int(order[len(ks) // 2]), len(ks) - 1})
        dS = {int(b): abs(float(S_all[b]) - oracle.linear(X64, labs[b].cpu().numpy(), ks[b])["S"]) for b in picks}
        del X64
        out["batched"] = {"labelings_per_s": len(ks) / s, "point_labelings_per_s": len(ks) * X.shape[0] / s,
                          "dS_vs_oracle": max(dS.values()),
                          "oracle_check": {"labelings": {str(b): {"k": ks[b], "dS": v} for b, v in dS.items()},
                                           "kind": "FP64 linear form over all rows of the first, median-k "
                                                   "and last labelings"},
                          "ms": s * 1e3, "ms_without_graph": s_loop * 1e3,
                          "ms_per_labeling_launches_without_graph": s_per * 1e3, "N": X.shape[0], "D": 32,
                          "B": len(ks), "sum_k": int(sum(ks)),
                          "launch": ("pass 1 per labeling; every labeling's pass 2 in one tensor-core launch; "
                                     "one CUDA graph per step") if one_launch else "one CUDA graph per step",
                          "autotune": {"plan": tuned.get("one_launch") if one_launch else None,
                                       "seconds": t_tune}}
        del X, labs, g
        torch.cuda.empty_cache()
    return out


def run_case(args):
    """One small case of a secondary workload, untimed, for profiler captures:
    the same recipe and seed as the full workload at args.n points."""
    import torch
    from paper_2303_14102_gb300 import sil, synth
    from paper_2303_14102_gb300.autograd import silhouette_loss
    dev = torch.device("cuda", 0)
    if args.case.startswith("precision"):
        w = synth.workload_precision(device=dev, N=args.n)
        cs = None
        if args.case == "precision_bf16":
            X = synth.to_bf16(w.X)
        else:
            X, cs = synth.to_fp8_e4m3(w.X)
        st = sil.new_status(dev)
        agg = sil.aggregate(X, w.labels, w.K, col_scale=cs, status=st)
        for _ in range(3):
            r = sil.score(X, w.labels, w.K, agg, col_scale=cs, status=st)
        torch.cuda.synchronize()
        sil.check_status(st, args.case)
        print(json.dumps({"case": args.case, "N": args.n, "S": float(r.S)}))
    elif args.case == "grad":
        w = synth.workload_grad(device=dev, N=args.n)
        for _ in range(2):
            Xg = w.X.detach().requires_grad_(True)
            S = silhouette_loss(Xg, w.labels, w.K, "sqeuclidean")
            S.backward()
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "N": args.n, "S": float(S.detach())}))
    else:
        X, labs, ks = synth.workload_batched(device=dev, B=args.batch)
        sil.autotune_batched(X, labs, ks)  # as the timed bench does
        for _ in range(2):
            S = sil.score_batched(X, labs, ks)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "B": args.batch, "ks": ks, "S": S.tolist()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variants", type=int, default=1, help="also measure the variant lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=10_000_000,
                    help="points of the at_scale workload (smaller only for profiling captures)")
    ap.add_argument("--case", default=None, choices=["precision_bf16", "precision_fp8", "grad", "batched"],
                    help="run one untimed small case of another workload (for profiler captures) and exit")
    ap.add_argument("--batch", type=int, default=2, help="labelings of the batched case")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case is not None:
        return run_case(args)

    import numpy as np
    import torch
    from paper_2303_14102_gb300 import sil, synth

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sil.load()
    pk = peaks()
    w = synth.workload_at_scale(device=dev, N=args.n)
    X, lab, K = w.X, w.labels, w.K
    N, D = X.shape
    stream = torch.cuda.current_stream(dev)
    status = sil.new_status(dev)

    # one step: pass 1 + pass 2 (sq-Euclidean), events between the two calls
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    agg_buf = (torch.zeros(K, dtype=torch.int64, device=dev), torch.zeros(K, D, dtype=torch.float64, device=dev),
               torch.zeros(K, dtype=torch.float64, device=dev))

    def step(record=None):
        if record is not None:
            ev[0].record(stream)
        agg = sil.aggregate(X, lab, K, out=agg_buf, status=status)
        if record is not None:
            ev[1].record(stream)
        r = sil.score(X, lab, K, agg, status=status)
        if record is not None:
            ev[2].record(stream)
            torch.cuda.synchronize()
            record.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sil.check_status(status, "bench warm-up")

    barrier(world)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk.mark(True)
        e0.record(stream)
        for _ in range(args.steps):
            r = step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
        barrier(world)
        t = e0.elapsed_time(e1) / 1e3
        # per-pass split (same launches, events between the two calls), over
        # at least half a second of steps so that the split is steady
        split = []
        ts0 = time.time()
        for _ in range(max(args.steps, int(0.5 / max(t / args.steps, 1e-6)) + 1)):
            step(record=split)
        ts1 = time.time()
    clocks = clk.summary()
    # the same steps run for the per-pass split right after the timed region,
    # for at least half a second: many more samples of the clocks under this load
    clocks["split_window"] = dict(clk.summary((ts0, ts1)), seconds=round(ts1 - ts0, 3),
                                  window="the per-pass timing right after the timed region")
    t = max_over_ranks(t, world)
    S_val = float(r.S.item())
    sil.check_status(status, "bench")
    value = N * args.steps * world / t
    ms_pass1 = statistics.mean(s[0] for s in split)
    ms_pass2 = statistics.mean(s[1] for s in split)

    # roofline of the dominant kernel (the longer pass); both passes read X and
    # the labels once, so both are HBM-bound at this K (2K flop per 4 bytes of
    # X on the tensor cores is far below the tensor ridge)
    bytes_pass1 = N * D * 4 + N * 4          # one read of X and labels
    bytes_pass2 = N * D * 4 + N * 4          # one read of X and labels
    flops_pass2 = 2.0 * N * K * D            # the K dot products per point
    plan = sil.tensor_plan(X.dtype, D, K)
    p2_kernel = "k_score_tc (pass 2, tcgen05)" if plan is not None else "k_score_simt (pass 2)"
    if ms_pass2 >= ms_pass1:
        kname, kbytes, kms = p2_kernel, bytes_pass2, ms_pass2
    else:
        kname, kbytes, kms = "k_gather_reduce_tma (pass 1)", bytes_pass1, ms_pass1
    achieved = kbytes / (kms / 1e3) / 1e9
    traffic, traffic_source = measured_traffic(kname, N, D, K, X.dtype)
    roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "traffic_source": traffic_source,
            "peak_source": f"{pk['source']} copy bandwidth (burst)",
            "algorithmic": f"N*(4D+4) = {kbytes:.3e} B per launch",
            "timing": "CUDA events around the pass on the launching stream, mean over steps "
                      "(pass 1 includes its small reference-point and finalisation launches)"}
    pass_info = {"pass1_ms": ms_pass1, "pass1_hbm_gbs": bytes_pass1 / (ms_pass1 / 1e3) / 1e9,
                 "pass2_ms": ms_pass2, "pass2_hbm_gbs": bytes_pass2 / (ms_pass2 / 1e3) / 1e9,
                 "pass2_tflops": flops_pass2 / (ms_pass2 / 1e3) / 1e12}

    # end to end through the public API from pinned host buffers: every step
    # copies its inputs host -> device (pinned, on a copy stream, into one of
    # two device buffers so that the copy of step s+1 overlaps the scoring of
    # step s), scores them with sil.silhouette and reads S back to the host
    Xh = X.cpu().pin_memory()
    lh = lab.cpu().pin_memory()
    Xd = [torch.empty_like(X) for _ in range(2)]
    ld = [torch.empty_like(lab) for _ in range(2)]
    S_host = torch.empty(2, dtype=torch.float64).pin_memory()
    copy_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    for ev_ in consumed:
        ev_.record(stream)

    def e2e_step(sidx):
        b = sidx % 2
        copy_stream.wait_event(consumed[b])
        with torch.cuda.stream(copy_stream):
            Xd[b].copy_(Xh, non_blocking=True)
            ld[b].copy_(lh, non_blocking=True)
            copied[b].record(copy_stream)
        stream.wait_event(copied[b])
        res = sil.silhouette(Xd[b], ld[b], K, status=status)
        S_host[b].copy_(res.S, non_blocking=True)
        consumed[b].record(stream)

    for sidx in range(2):
        e2e_step(sidx)
    torch.cuda.synchronize()
    counter = iter(range(10 ** 9))
    te = timed(lambda: e2e_step(next(counter)), args.steps, stream)
    te = max_over_ranks(te, world)
    e2e = {"value": N * args.steps * world / te, "unit": "points/s",
           "h2d_bytes_per_step": int(Xh.numel() * 4 + lh.numel() * 4), "d2h_bytes_per_step": 8,
           "pipelining": "host-to-device copy of step s+1 overlaps the scoring of step s (two device buffers)"}
    del Xd, ld
    variants = {}
    if args.variants and rank == 0:
        # same workload: cosine, the approximate Euclidean form (square roots of
        # the mean squared distances in Eq. 2), and BF16 storage
        X64 = X.cpu().double().numpy()
        lab_h = lab.cpu().numpy()
        head_check = oracle_full(X64, lab_h, K, "sqeuclidean", S_val)
        for name, metric in (("cosine_fp32", "cosine"), ("euclidean_rms_fp32", "euclidean_rms")):
            fn = lambda: sil.silhouette(X, lab, K, metric, status=status)  # noqa: E731
            rv = fn()
            s = timed(fn, args.steps, stream)
            Sv = float(rv.S.item())
            chk = oracle_full(X64, lab_h, K, metric, Sv)
            variants[name] = {"points_per_s": N * args.steps / s, "ms": s / args.steps * 1e3, "S": Sv,
                              "dS_vs_oracle": chk["dS_vs_oracle"], "oracle_check": chk}
        # the small workload (N 1e4, D 8, K 5, both passes of one call): launch
        # latency, not bytes, bounds it -- microseconds per API call, and per
        # replay of the same call captured in a CUDA graph
        wsm = synth.workload_small(device=dev)
        fn = lambda: sil.silhouette(wsm.X, wsm.labels, wsm.K, status=status)  # noqa: E731
        rsm = fn()
        t_call = timed(fn, 200, stream) / 200
        graph_info = {}
        try:
            side = torch.cuda.Stream(dev)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                for _ in range(3):
                    fn()
            stream.wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                rg = fn()
            graph.replay()
            torch.cuda.synchronize()
            graph_info = {"us_per_graph_replay": timed(graph.replay, 200, stream) / 200 * 1e6,
                          "S_graph": float(rg.S.item())}
            del graph, rg
        except Exception as exc:  # the direct calls above stand on their own
            graph_info = {"graph": f"not captured: {type(exc).__name__}: {exc}"[:200]}
        S_sm = float(rsm.S.item())
        chk = oracle_full(wsm.X.cpu().double().numpy(), wsm.labels.cpu().numpy(), wsm.K, "sqeuclidean", S_sm)
        variants["small_sqeuclidean"] = dict({"us_per_call": t_call * 1e6, "points_per_s": wsm.X.shape[0] / t_call,
                                              "S": S_sm, "dS_vs_oracle": chk["dS_vs_oracle"], "oracle_check": chk,
                                              "N": wsm.X.shape[0], "D": wsm.X.shape[1], "K": wsm.K}, **graph_info)
        del wsm
        # pass 2 on the CUDA cores (FP32 FFMA against Z in shared memory), the
        # path the tensor-core kernel replaces at this K, for comparison
        agg_s = sil.aggregate(X, lab, K, status=status)
        fn = lambda: sil.score(X, lab, K, agg_s, path="simt", status=status)
        rs = fn()
        s = timed(fn, args.steps, stream)
        Ss = float(rs.S.item())
        variants["sqeuclidean_fp32_simt_pass2"] = {
            "ms": s / args.steps * 1e3, "hbm_gbs": N * (4 * D + 4) / (s / args.steps) / 1e9,
            "fp32_tflops": 2.0 * N * K * D / (s / args.steps) / 1e12, "S": Ss,
            "dS_vs_oracle": abs(Ss - head_check["oracle_S"])}
        # pass 2 on the TF32-ranked tensor-core kernel (exact FP32 recompute of
        # a_i and of every candidate inside the TF32 error band)
        fn = lambda: sil.score(X, lab, K, agg_s, path="tensor_tf32", status=status)  # noqa: E731
        rt = fn()
        s = timed(fn, args.steps, stream)
        St = float(rt.S.item())
        variants["sqeuclidean_fp32_tf32_pass2"] = {
            "ms": s / args.steps * 1e3, "hbm_gbs": N * (4 * D + 4) / (s / args.steps) / 1e9, "S": St,
            "dS_vs_oracle": abs(St - head_check["oracle_S"])}
        del agg_s, X64
        Xb = X.to(torch.bfloat16)
        fn = lambda: sil.silhouette(Xb, lab, K, status=status)  # noqa: E731
        rb = fn()
        s = timed(fn, args.steps, stream)
        Sb = float(rb.S.item())
        chk = oracle_full(Xb.cpu().double().numpy(), lab_h, K, "sqeuclidean", Sb)  # the stored BF16 values
        variants["sqeuclidean_bf16"] = {"points_per_s": N * args.steps / s, "ms": s / args.steps * 1e3,
                                        "S": Sb, "S_fp32": S_val, "dS_vs_fp32": abs(Sb - S_val),
                                        "dS_vs_oracle": chk["dS_vs_oracle"], "oracle_check": chk}
        del Xb
        torch.cuda.empty_cache()
        variants.update(variant_lines(dev, args.steps, budget_s=150.0,
                                      pk_sustained=pk["bf16_tflops_sustained"], pk_sm_mhz=pk["sm_max_mhz"]))

    if rank == 0 and not args.variants:
        head_check = oracle_full(X.cpu().double().numpy(), lab.cpu().numpy(), K, "sqeuclidean", S_val)
    cpu = None
    if rank == 0 and world >= 1 and not args.no_cpu_baseline and args.gpus == 1:
        cpu = cpu_oracle_sample(X.cpu().numpy(), lab.cpu().numpy(), K)

    if rank == 0:
        # pass 1: bucket_count, bucket_scan, bucket_scatter, shift_build,
        #         gather_reduce, publish_status;
        # pass 2: fin_global, fin_clusters, (tc_pack,) score, reduce_S
        launches_per_step = 6 + (5 if plan is not None else 4)
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": bench_config(N, D, world),
                "S": S_val, "dS_vs_oracle": head_check["dS_vs_oracle"], "oracle_check": head_check,
                "passes": pass_info, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
                "variants": variants}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
