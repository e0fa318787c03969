"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every expected value comes from ``oracle`` on the same seeded inputs.  Sizes
span several pass-1 tiles (128 rows) and pass-2 blocks with ragged tails,
every register-tile width of the SIMT kernel (d <= 16, 32, 64, 128) and the
wide-row kernel, column-sliced pass 1 (large k*d), empty label ids,
singleton clusters and the degenerate cases.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, assert_scores, case, dequant, to_dev
from paper_2303_14102_gb300 import sil, synth

pytestmark = pytest.mark.gpu
METRICS = ["sqeuclidean", "cosine"]


def run(X, lab, K, metric, dtype=torch.float32, col_scale=None, path="auto", fused=False):
    """sil_aggregate + sil_score, or (fused) both in one sil_silhouette call."""
    Xt, lt = to_dev(X, lab, dtype) if not isinstance(X, torch.Tensor) else (X, lab)
    st = sil.new_status(Xt.device)
    if fused:
        agg = (torch.empty(K, dtype=torch.int64, device=Xt.device),
               torch.empty(K, Xt.shape[1], dtype=torch.float64, device=Xt.device),
               torch.empty(K, dtype=torch.float64, device=Xt.device))
        r = sil.silhouette(Xt, lt, K, metric, col_scale=col_scale, want_s=True, save=True, path=path,
                           status=st, out=agg)
    else:
        agg = sil.aggregate(Xt, lt, K, metric, col_scale=col_scale, status=st)
        r = sil.score(Xt, lt, K, agg, metric, col_scale=col_scale, want_s=True, save=True, path=path,
                      status=st)
    torch.cuda.synchronize()
    return Xt, lt, agg, r, int(st.item())


@pytest.mark.parametrize("metric", METRICS)
def test_small_workload_against_bruteforce(metric):
    w = synth.workload_small()  # N=10,000, D=8, K=5
    Xt, lt, agg, r, st = run(w.X.numpy(), w.labels.numpy(), w.K, metric)
    assert st == 0
    ref = oracle.bruteforce(w.X.double().numpy(), w.labels.numpy(), w.K, metric)
    assert_scores(r.s, r.S, ref, what=metric)
    a, b, ks = sil.unpack_saved(r.saved, Xt.shape[0])
    np.testing.assert_allclose(a.cpu().double().numpy(), ref["a"], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(b.cpu().double().numpy(), ref["b"], rtol=1e-4, atol=1e-4)
    assert np.mean(ks.cpu().numpy() == ref["kstar"]) > 0.999


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("N,D,K", [(1, 3, 2), (7, 1, 3), (129, 5, 4), (1000, 17, 7), (4099, 33, 6),
                                   (3001, 64, 9), (2500, 65, 5), (2000, 130, 8), (1500, 257, 4),
                                   (3000, 12, 64)])
def test_ragged_shapes(metric, N, D, K):
    if metric == "cosine" and D == 1:
        pytest.skip("1-D cosine distances are 0 or 2: a, b vanish up to rounding")
    X, lab = case(1000 + N + D + K, N, D, K, metric)
    Xt, lt, agg, r, st = run(X, lab, K, metric)
    ref = oracle.bruteforce(X.astype(np.float64), lab, K, metric)
    if ref["status"] == oracle.EDEGENERATE:
        assert st & sil.SIL_EDEGENERATE and np.isnan(float(r.S))
        return
    assert st == 0
    assert_scores(r.s, r.S, ref, what=f"{metric} N={N} D={D} K={K}")


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("N,D,K", [(5000, 24, 3), (20000, 128, 1000), (3000, 256, 300)])
def test_aggregates(metric, N, D, K):
    X, lab = case(77 + D + K, N, D, K, metric, spread=50.0)
    Xt, lt = to_dev(X, lab)
    count, s1, s2 = sil.aggregate(Xt, lt, K, metric)
    rc, r1, r2 = oracle.aggregate(X.astype(np.float64), lab, K, metric)
    np.testing.assert_array_equal(count.cpu().numpy(), rc)  # counts bit-exact
    scale = np.abs(r1).max()
    np.testing.assert_allclose(s1.cpu().numpy(), r1, rtol=1e-6, atol=1e-6 * scale)
    np.testing.assert_allclose(s2.cpu().numpy(), r2, rtol=1e-6, atol=1e-6 * np.abs(r2).max())


@pytest.mark.parametrize("metric", METRICS)
def test_within_scatter_far_from_origin(metric):
    # centres at radius 1e3, sigma 1: W_k = s2 - |s1|^2/n cancels ~4 digits
    w = synth.blobs(40000, 32, 20, seed=5, sphere_radius=1e3)
    X = w.X.numpy()
    lab = w.labels.numpy()
    Xt, lt = to_dev(X, lab)
    count, s1, s2 = (t.cpu().numpy() for t in sil.aggregate(Xt, lt, 20, metric))
    rc, r1, r2 = oracle.aggregate(X.astype(np.float64), lab, 20, metric)
    W = s2 - (s1 ** 2).sum(1) / count
    Wr = r2 - (r1 ** 2).sum(1) / rc
    np.testing.assert_allclose(W, Wr, rtol=1e-5 if metric == "sqeuclidean" else 1e-3)


def test_accumulate_merges_row_shards():
    X, lab = case(9, 7777, 20, 6)
    Xt, lt = to_dev(X, lab)
    whole = sil.aggregate(Xt, lt, 6)
    acc = (torch.zeros(6, dtype=torch.int64, device="cuda"),
           torch.zeros(6, 20, dtype=torch.float64, device="cuda"),
           torch.zeros(6, dtype=torch.float64, device="cuda"))
    for lo, hi in [(0, 1000), (1000, 1001), (1001, 7777)]:
        sil.aggregate(Xt[lo:hi], lt[lo:hi], 6, out=acc, accumulate=True)
    assert torch.equal(acc[0], whole[0])  # counts bit-exact
    # FP32 partial sums per CTA: a different row split rounds differently (~1e-7 relative)
    torch.testing.assert_close(acc[1], whole[1], rtol=1e-6, atol=1e-6 * float(whole[1].abs().max()))
    torch.testing.assert_close(acc[2], whole[2], rtol=1e-6, atol=0.0)


def test_strided_rows():
    X, lab = case(10, 3000, 10, 5)
    big = np.zeros((3000, 16), np.float32)
    big[:, :10] = X
    Xt = torch.as_tensor(big).cuda()[:, :10]  # ldx = 16 > d
    lt = torch.as_tensor(lab).cuda()
    _, _, _, r, st = run(Xt, lt, 5, "sqeuclidean")
    ref = oracle.bruteforce(X.astype(np.float64), lab, 5)
    assert st == 0
    assert_scores(r.s, r.S, ref)


@pytest.mark.parametrize("metric", METRICS)
def test_bf16_storage(metric):
    X, lab = case(11, 6000, 40, 7, metric)
    Xt, lt = to_dev(X, lab, torch.bfloat16)
    _, _, _, r, st = run(Xt, lt, 7, metric)
    ref = oracle.bruteforce(dequant(Xt), lab, 7, metric)
    assert st == 0
    assert_scores(r.s, r.S, ref, what="bf16 " + metric)


@pytest.mark.parametrize("metric", METRICS)
def test_fp8_storage_with_column_scales(metric):
    X, lab = case(12, 6000, 24, 5, metric)
    q, scale = synth.to_fp8_e4m3(torch.as_tensor(X))
    Xt, lt = q.cuda(), torch.as_tensor(lab).cuda()
    cs = scale.cuda()
    _, _, _, r, st = run(Xt, lt, 5, metric, col_scale=cs)
    ref = oracle.bruteforce(dequant(Xt, cs), lab, 5, metric)
    assert st == 0
    assert_scores(r.s, r.S, ref, what="fp8 " + metric)


def test_simt_path_forced_equals_auto():
    X, lab = case(13, 5000, 16, 6)
    _, _, _, a, _ = run(X, lab, 6, "sqeuclidean", path="auto")
    _, _, _, b, _ = run(X, lab, 6, "sqeuclidean", path="simt")
    torch.testing.assert_close(a.s, b.s, rtol=0, atol=1e-5)


# ------------------------------------------------------------ edge cases
@pytest.mark.parametrize("fused", [False, True])
def test_degenerate_single_cluster(fused):
    X, _ = case(14, 500, 4, 3)
    lab = np.zeros(500, np.int32)
    _, _, _, r, st = run(X, lab, 3, "sqeuclidean", fused=fused)
    assert st & sil.SIL_EDEGENERATE
    assert np.isnan(float(r.S))
    assert torch.all(r.s == 0)


@pytest.mark.parametrize("fused", [False, True])
def test_bad_label_flagged(fused):
    X, lab = case(15, 500, 4, 3)
    lab[17] = 3
    _, _, _, r, st = run(X, lab, 3, "sqeuclidean", fused=fused)
    assert st & sil.SIL_ELABEL
    assert np.isnan(float(r.S))


@pytest.mark.parametrize("fused", [False, True])
def test_zero_row_cosine_flagged(fused):
    X, lab = case(16, 500, 4, 3, "cosine")
    X[3] = 0.0
    _, _, _, r, st = run(X, lab, 3, "cosine", fused=fused)
    assert st & sil.SIL_EZERONORM
    assert np.isnan(float(r.S))


@pytest.mark.parametrize("fused", [False, True])
def test_all_singletons_and_duplicates(fused):
    X, _ = case(17, 40, 3, 3)
    lab = np.arange(40, dtype=np.int32)
    _, _, _, r, st = run(X, lab, 40, "sqeuclidean", fused=fused)
    assert st == 0 and float(r.S) == 0.0
    Xd = np.repeat(np.array([[0, 0], [3, 4], [-5, 1]], np.float32), [300, 500, 200], axis=0)
    ld = np.repeat(np.array([0, 1, 2], np.int32), [300, 500, 200])
    _, _, _, r, st = run(Xd, ld, 3, "sqeuclidean", fused=fused)
    assert st == 0 and abs(float(r.S) - 1.0) < 1e-6


def test_empty_input():
    Xt = torch.zeros(0, 4, device="cuda")
    lt = torch.zeros(0, dtype=torch.int32, device="cuda")
    count, s1, s2 = sil.aggregate(Xt, lt, 3)
    assert int(count.sum()) == 0
    r = sil.score(Xt, lt, 3, (count, s1, s2))
    assert np.isnan(float(r.S))
    out = (torch.full((3,), 7, dtype=torch.int64, device="cuda"), torch.ones(3, 4, dtype=torch.float64, device="cuda"),
           torch.ones(3, dtype=torch.float64, device="cuda"))
    r = sil.silhouette(Xt, lt, 3, out=out)
    assert np.isnan(float(r.S)) and int(out[0].abs().sum()) == 0 and float(out[1].abs().sum()) == 0.0


# ------------------------------------------------------------- batched
@pytest.mark.parametrize("metric", METRICS)
def test_batched_matches_oracle_per_labeling(metric):
    X, _ = case(18, 3000, 12, 4, metric)
    rng = np.random.default_rng(3)
    ks = [2, 5, 17, 3, 40, 9]
    labs = np.stack([rng.integers(0, k, size=3000).astype(np.int32) for k in ks])
    Xt = torch.as_tensor(X).cuda()
    S = sil.score_batched(Xt, torch.as_tensor(labs).cuda(), ks, metric).cpu().numpy()
    for b, k in enumerate(ks):
        ref = oracle.linear(X.astype(np.float64), labs[b], k, metric)
        assert abs(S[b] - ref["S"]) <= TOL_S, (b, S[b], ref["S"])


# ------------------------------------------- pass-1 load paths and plans agree
@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("N,D,K", [(100003, 64, 100), (7777, 24, 6), (50001, 128, 1000), (3001, 256, 40),
                                   (20000, 600, 7), (30000, 16, 5000), (40000, 8, 20000)])
def test_pass1_load_paths_agree(metric, dtype, N, D, K, monkeypatch):
    # rows by TMA row gather (the default where a row fits one box), by
    # 16-byte register loads, and element by element at an odd row stride.
    # D = 600 splits the rows into column slices (cosine then takes its norms
    # from a separate kernel); K = 5000 and 20000 exceed the shared-memory
    # bucket tables of the sort kernels, which then use global atomics
    X, lab = case(600 + N + D, N, D, K, metric)
    Xt, lt = to_dev(X, lab, dtype)
    fast = sil.aggregate(Xt, lt, K, metric)
    monkeypatch.setenv("SIL_AGG_LDG", "1")
    regs = sil.aggregate(Xt, lt, K, metric)
    monkeypatch.delenv("SIL_AGG_LDG")
    torch.cuda.synchronize()
    assert torch.equal(fast[0], regs[0])
    torch.testing.assert_close(fast[1], regs[1], rtol=1e-6, atol=1e-6 * float(regs[1].abs().max()))
    torch.testing.assert_close(fast[2], regs[2], rtol=1e-6, atol=0.0)
    # the same rows at an odd row stride: no 16-byte loads are possible
    wide = torch.zeros(N, D + 1, dtype=dtype, device="cuda")
    wide[:, :D] = Xt
    slow = sil.aggregate(wide[:, :D], lt, K, metric)
    torch.cuda.synchronize()
    assert torch.equal(fast[0], slow[0])
    torch.testing.assert_close(fast[1], slow[1], rtol=1e-6, atol=1e-6 * float(slow[1].abs().max()))
    torch.testing.assert_close(fast[2], slow[2], rtol=1e-6, atol=0.0)
    rc, r1, r2 = oracle.aggregate(dequant(Xt), lab, K, metric)
    np.testing.assert_array_equal(fast[0].cpu().numpy(), rc)
    np.testing.assert_allclose(fast[1].cpu().numpy(), r1, rtol=1e-6, atol=1e-6 * np.abs(r1).max())
    # s2 sums n_k * D squared FP32 terms (partials over runs of <= 256 rows,
    # up to 16 columns per lane): a few 1e-6 relative at D = 600
    np.testing.assert_allclose(fast[2].cpu().numpy(), r2, rtol=1e-5, atol=1e-9 * np.abs(r2).max())


def test_batched_graph_replay_matches_direct_call():
    rng = np.random.default_rng(77)
    X = (rng.normal(size=(5000, 32)) + rng.integers(0, 4, size=(5000, 1)) * 3).astype(np.float32)
    ks = [2, 9, 300, 40]
    labs = np.stack([rng.integers(0, k, size=5000).astype(np.int32) for k in ks])
    Xt, lt = torch.as_tensor(X).cuda(), torch.as_tensor(labs).cuda()
    direct = sil.score_batched(Xt, lt, ks).cpu().numpy()
    g = sil.BatchedGraph(Xt, lt, ks)
    for _ in range(2):
        S = g.run().cpu().numpy()
        # pass 1 sums rows in an order that depends on scheduling: equal to FP32 rounding
        np.testing.assert_allclose(S, direct, rtol=0, atol=TOL_S)
    ref = [oracle.linear(X.astype(np.float64), labs[b], k)["S"] for b, k in enumerate(ks)]
    np.testing.assert_allclose(S, ref, rtol=0, atol=TOL_S)


# ------------------------------------------- full-size workloads, sampled
@pytest.mark.parametrize("metric", METRICS)
def test_at_scale_workload_full_size(metric):
    # the benchmark's headline workload (N = 1e7, D = 64, K = 100, FP32) in
    # its launch configuration, against the FP64 linear form over ALL 1e7
    # rows (Sec. II: S is the mean over every point): counts bit-exact, every
    # s_i within 1e-4 and S within 1e-6
    w = synth.workload_at_scale(device="cuda")
    st = sil.new_status(w.X.device)
    r = sil.silhouette(w.X, w.labels, w.K, metric, want_s=True, status=st)
    count = sil.aggregate(w.X, w.labels, w.K, metric)[0].cpu().numpy()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oracle.linear(w.X.cpu().double().numpy(), w.labels.cpu().numpy(), w.K, metric)
    assert ref["status"] == oracle.OK
    assert np.array_equal(count, ref["agg"][0])
    assert_scores(r.s, r.S, ref, what=f"at_scale {metric}")


def test_batched_workload_full_size_sampled():
    # all 256 labelings of the batched workload in one call; three of them
    # (first, median k, last) against the FP64 linear form over all 2e6 rows
    X, labs, ks = synth.workload_batched(device="cuda")
    S = sil.score_batched(X, labs, ks).cpu().numpy()
    assert S.shape == (len(ks),) and np.all(np.isfinite(S))
    X64 = X.cpu().double().numpy()
    order = np.argsort(ks)
    for b in (0, int(order[len(ks) // 2]), len(ks) - 1):
        ref = oracle.linear(X64, labs[b].cpu().numpy(), ks[b])
        assert abs(S[b] - ref["S"]) <= TOL_S, (b, ks[b], S[b], ref["S"])
