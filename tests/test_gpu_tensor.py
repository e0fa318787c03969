"""Parity of the tcgen05 tensor-core pass 2 with the FP64 oracle.

Two kernels.  The split-precision kernel (paths "auto" and "tensor"): FP32
storage runs the in-kernel BF16 hi/lo split (three MMAs per k-step), BF16
storage runs two, FP8 storage (d = 128, per-column scales folded into the
centroids) runs two on the widened codes.  The TF32 kernel (path
"tensor_tf32", FP32 rows of 32..64 columns) ranks the clusters with one TF32
product on the tile as TMA delivers it and recomputes a_i and every cluster
inside the provable error band exactly in FP32.  All must meet the
FP32 tolerances of the SIMT path.  Sizes cover one and two 32/64-wide K
atoms, padded D, K from 2 to 1000 (one cluster block of up to 256, and
several blocks whose per-block minima are combined), ragged last tiles and
multi-tile CTAs.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, assert_scores, case, dequant, to_dev
from paper_2303_14102_gb300 import sil, synth

pytestmark = pytest.mark.gpu
METRICS = ["sqeuclidean", "cosine"]


def run(Xt, lt, K, metric, path, save=True, cs=None):
    """path "<p>_fused": both passes in one sil_silhouette call; otherwise
    sil_aggregate + sil_score."""
    st = sil.new_status(Xt.device)
    if path.endswith("_fused"):
        r = sil.silhouette(Xt, lt, K, metric, col_scale=cs, want_s=True, save=save, path=path[:-6], status=st)
    else:
        agg = sil.aggregate(Xt, lt, K, metric, col_scale=cs, status=st)
        r = sil.score(Xt, lt, K, agg, metric, col_scale=cs, want_s=True, save=save, path=path, status=st)
    torch.cuda.synchronize()
    return r, int(st.item())


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("dtype,path", [(torch.float32, "tensor"), (torch.float32, "tensor_tf32"),
                                        (torch.float32, "tensor_fused"), (torch.float32, "tensor_tf32_fused"),
                                        (torch.bfloat16, "tensor")])
@pytest.mark.parametrize("N,D,K", [(1000, 64, 2), (4097, 64, 7), (20000, 64, 100), (3001, 128, 17),
                                   (5000, 100, 33), (2000, 40, 5), (300, 64, 256), (129, 64, 3),
                                   (700, 128, 128), (700, 128, 256), (3000, 64, 300),
                                   (2500, 128, 700), (1500, 64, 1000), (3000, 32, 7), (2000, 32, 300),
                                   (2000, 48, 129), (1000, 32, 16), (5000, 64, 512)])
def test_tensor_path_against_bruteforce(metric, dtype, path, N, D, K):
    if dtype == torch.bfloat16 and (D < 64 or (2 * D) % 16):
        pytest.skip("BF16 tensor path needs d >= 64 and 16-byte rows (TMA)")
    if path.startswith("tensor_tf32") and "tf32" not in sil.tensor_kernels(dtype, D, K):
        pytest.skip("the TF32 kernel serves FP32 rows of 32..64 columns")
    X, lab = case(700 + N + D + K, N, D, K, metric)
    Xt, lt = to_dev(X, lab, dtype)
    r, st = run(Xt, lt, K, metric, path)
    ref = oracle.bruteforce(dequant(Xt), lab, K, metric)
    if ref["status"] == oracle.EDEGENERATE:
        assert st & sil.SIL_EDEGENERATE
        return
    assert st == 0
    assert_scores(r.s, r.S, ref, what=f"tensor {metric} {dtype} N={N} D={D} K={K}")
    a, b, ks = sil.unpack_saved(r.saved, N)
    ok = ref["s"] != 0
    np.testing.assert_allclose(a.cpu().double().numpy()[ok], ref["a"][ok], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(b.cpu().double().numpy()[ok], ref["b"][ok], rtol=1e-4, atol=1e-4)
    assert np.mean(ks.cpu().numpy()[ok] == ref["kstar"][ok]) > 0.995


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("path", ["tensor", "tensor_tf32", "tensor_fused"])
def test_tensor_and_simt_agree_at_scale_recipe(metric, path):
    w = synth.workload_at_scale(device="cuda", N=300_000)
    ra, sa_ = run(w.X, w.labels, w.K, metric, path, save=False)
    rb, sb_ = run(w.X, w.labels, w.K, metric, "simt", save=False)
    assert sa_ == 0 and sb_ == 0
    assert float((ra.s - rb.s).abs().max()) <= TOL_SI
    assert abs(float(ra.S) - float(rb.S)) <= TOL_S


def test_tensor_path_far_from_origin():
    # centres at radius 1e3: the GEMM term is ~1e6 and cancels in d_k
    w = synth.blobs(20000, 128, 40, seed=9, sphere_radius=1e3)
    Xt, lt = w.X.cuda(), w.labels.cuda()
    r, st = run(Xt, lt, 40, "sqeuclidean", "tensor")
    assert st == 0
    ref = oracle.linear(w.X.double().numpy(), w.labels.numpy(), 40)
    assert_scores(r.s, r.S, ref)


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("D,K", [(64, 40), (32, 300)])
def test_tf32_far_from_origin(metric, D, K):
    # centres at radius 1e3: ||x|| ||mu'|| ~ 1e6, so the TF32 band spans
    # thousands and many clusters are recomputed exactly per point
    assert "tf32" in sil.tensor_kernels(torch.float32, D, K)
    w = synth.blobs(20000, D, K, seed=10 + D, sphere_radius=1e3)
    Xt, lt = w.X.cuda(), w.labels.cuda()
    r, st = run(Xt, lt, K, metric, "tensor_tf32")
    assert st == 0
    ref = oracle.linear(w.X.double().numpy(), w.labels.numpy(), K, metric)
    assert_scores(r.s, r.S, ref)
    _, b, ks = sil.unpack_saved(r.saved, 20000)
    np.testing.assert_allclose(b.cpu().double().numpy(), ref["b"], rtol=1e-5)


@pytest.mark.parametrize("path", ["tensor", "tensor_tf32", "simt"])
def test_fused_call_matches_the_two_calls(path):
    # sil_silhouette = sil_aggregate + sil_score: from the aggregates it
    # returned, sil_score gives bit-identical s_i and saved record
    N, D, K = 50_000, 64, 30
    X, lab = case(79, N, D, K)
    Xt, lt = to_dev(X, lab)
    agg = (torch.empty(K, dtype=torch.int64, device="cuda"), torch.empty(K, D, dtype=torch.float64, device="cuda"),
           torch.empty(K, dtype=torch.float64, device="cuda"))
    st = sil.new_status(Xt.device)
    rb = sil.silhouette(Xt, lt, K, want_s=True, save=True, path=path, status=st, out=agg)
    ra = sil.score(Xt, lt, K, agg, want_s=True, save=True, path=path, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.equal(ra.s, rb.s) and torch.equal(ra.saved, rb.saved)
    assert float(ra.S) == float(rb.S)


def test_fused_call_returns_the_aggregates():
    # the same tolerances as sil_aggregate's own parity test (the order of the
    # rows inside a cluster's bucket, and so the FP32 run sums, may vary)
    X, lab = case(78, 20000, 64, 30, spread=50.0)
    Xt, lt = to_dev(X, lab)
    out = (torch.empty(30, dtype=torch.int64, device="cuda"), torch.empty(30, 64, dtype=torch.float64, device="cuda"),
           torch.empty(30, dtype=torch.float64, device="cuda"))
    sil.silhouette(Xt, lt, 30, out=out)
    rc, r1, r2 = oracle.aggregate(X.astype(np.float64), lab, 30)
    np.testing.assert_array_equal(out[0].cpu().numpy(), rc)
    np.testing.assert_allclose(out[1].cpu().numpy(), r1, rtol=1e-6, atol=1e-6 * np.abs(r1).max())
    np.testing.assert_allclose(out[2].cpu().numpy(), r2, rtol=1e-6, atol=1e-6 * np.abs(r2).max())


@pytest.mark.parametrize("K,kernel", [(10, "tensor_tf32"), (48, "tensor_tf32"), (49, "tensor"), (100, "tensor")])
def test_auto_picks_the_tensor_kernel_by_cluster_count(K, kernel):
    # few clusters: the TF32-ranked kernel (no converter warps); more: the
    # split-precision kernel (one sweep over the ranked values)
    X, lab = case(5 + K, 3000, 64, K)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, K)
    ra = sil.score(Xt, lt, K, agg, want_s=True, path="auto")
    rt = sil.score(Xt, lt, K, agg, want_s=True, path=kernel)
    assert torch.equal(ra.s, rt.s)  # same aggregates, same kernel: bit-identical


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("N,D,K", [(3000, 256, 7), (2500, 256, 100), (1500, 160, 300), (2000, 256, 1000),
                                   (129, 200, 3)])
def test_wide_fp32_rows_in_chunks_against_bruteforce(metric, N, D, K):
    # FP32 rows of 129..256 columns: the GEMM accumulates four 64-column chunks
    X, lab = case(1300 + N + D + K, N, D, K, metric)
    Xt, lt = to_dev(X, lab)
    r, st = run(Xt, lt, K, metric, "tensor")
    ref = oracle.bruteforce(dequant(Xt), lab, K, metric)
    assert st == 0
    assert_scores(r.s, r.S, ref, what=f"wide tensor {metric} N={N} D={D} K={K}")
    a, b, ks = sil.unpack_saved(r.saved, N)
    ok = ref["s"] != 0
    np.testing.assert_allclose(a.cpu().double().numpy()[ok], ref["a"][ok], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(b.cpu().double().numpy()[ok], ref["b"][ok], rtol=1e-4, atol=1e-4)
    assert np.mean(ks.cpu().numpy()[ok] == ref["kstar"][ok]) > 0.995


@pytest.mark.parametrize("metric", METRICS)
def test_wide_fp32_tensor_and_simt_agree_on_grad_recipe(metric):
    w = synth.workload_grad(device="cuda", N=100_000)
    ra, sa_ = run(w.X, w.labels, w.K, metric, "tensor", save=False)
    rb, sb_ = run(w.X, w.labels, w.K, metric, "simt", save=False)
    assert sa_ == 0 and sb_ == 0
    assert float((ra.s - rb.s).abs().max()) <= TOL_SI
    assert abs(float(ra.S) - float(rb.S)) <= TOL_S


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("N,K", [(1000, 5), (4097, 100), (3000, 300), (2000, 1000)])
def test_fp8_tensor_path_against_bruteforce(metric, N, K):
    X, lab = case(900 + N + K, N, 128, K, metric)
    q, scale = synth.to_fp8_e4m3(torch.as_tensor(X))
    Xt, lt, cs = q.cuda(), torch.as_tensor(lab).cuda(), scale.cuda()
    r, st = run(Xt, lt, K, metric, "tensor", cs=cs)
    ref = oracle.bruteforce(dequant(Xt, cs), lab, K, metric)
    assert st == 0
    assert_scores(r.s, r.S, ref, what=f"fp8 tensor {metric} N={N} K={K}")
    a, b, ks = sil.unpack_saved(r.saved, N)
    ok = ref["s"] != 0
    np.testing.assert_allclose(b.cpu().double().numpy()[ok], ref["b"][ok], rtol=1e-4, atol=1e-4)
    assert np.mean(ks.cpu().numpy()[ok] == ref["kstar"][ok]) > 0.995


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("dtype,D,K", [(torch.float32, 100, 513), (torch.bfloat16, 128, 300),
                                       (torch.float8_e4m3fn, 128, 300), (torch.float32, 64, 1000)])
def test_own_cluster_term_of_unstaged_block_plans(metric, dtype, D, K):
    # plans of several cluster blocks whose centroids stay in global memory
    # take a_i from a separate kernel (lanes of a warp share a row) instead of
    # the converter warps: a_i and s_i element by element against brute force
    p = sil.tensor_plan_candidates(dtype, D, K, 1)[0]
    assert p[3] == 0 and -(-K // p[0]) > 1, p
    N = 3001
    X, lab = case(1300 + D + K, N, D, K, metric)
    cs = None
    if dtype == torch.float8_e4m3fn:
        q, scale = synth.to_fp8_e4m3(torch.as_tensor(X))
        Xt, lt, cs = q.cuda(), torch.as_tensor(lab).cuda(), scale.cuda()
    else:
        Xt, lt = to_dev(X, lab, dtype)
    r, st = run(Xt, lt, K, metric, "tensor", cs=cs)
    ref = oracle.bruteforce(dequant(Xt, cs), lab, K, metric)
    assert st == 0
    assert_scores(r.s, r.S, ref, what=f"own term {metric} {dtype} D={D} K={K}")
    a, b, ks = sil.unpack_saved(r.saved, N)
    ok = ref["s"] != 0
    np.testing.assert_allclose(a.cpu().double().numpy()[ok], ref["a"][ok], rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_precision_recipe_subsample(storage):
    # the precision workload's recipe (centres at radius 1e3, d = 128,
    # k = 1000) at reduced n; s_i of 20,000 seeded rows against the FP64
    # linear form with full-n FP64 aggregates of the stored values
    w = synth.workload_precision(device="cuda", N=200_000)
    cs = None
    if storage == "bf16":
        Xt = synth.to_bf16(w.X)
    else:
        Xt, cs = synth.to_fp8_e4m3(w.X)
    lt = w.labels
    r, st = run(Xt, lt, w.K, "sqeuclidean", "tensor", save=False, cs=cs)
    assert st == 0
    X64, lab = dequant(Xt, cs), lt.cpu().numpy()
    full = oracle.linear(X64, lab, w.K)
    idx = np.sort(np.random.default_rng(2026).choice(Xt.shape[0], 20_000, replace=False))
    sub = oracle.linear(X64, lab, w.K, agg=full["agg"], idx=idx)
    s = r.s.cpu().double().numpy()
    assert float(np.abs(s[idx] - sub["s"]).max()) <= TOL_SI
    assert float(np.abs(s - full["s"]).max()) <= TOL_SI
    # the bound stated for the low-precision storage forms
    assert abs(float(r.S) - full["S"]) <= 1e-4


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_precision_workload_full_size_sampled(storage):
    # the full precision workload (n = 1e8, d = 128, k = 1000, radius 1e3) in
    # the launch configuration the benchmark times; s_i of 20,000 seeded rows
    # against the FP64 linear form with FP64 aggregates of all 1e8 stored rows
    w = synth.workload_precision(device="cuda")
    if storage == "bf16":
        Xt, cs = synth.to_bf16(w.X), None
    else:
        Xt, cs = synth.to_fp8_e4m3(w.X)
    lt, K, N = w.labels, w.K, Xt.shape[0]
    del w  # the FP32 copy (51 GB) is no longer needed
    torch.cuda.empty_cache()
    r, st = run(Xt, lt, K, "sqeuclidean", "auto", save=False, cs=cs)
    assert st == 0
    s_gpu, S_gpu = r.s.cpu().double().numpy(), float(r.S)
    del r
    count = np.zeros(K, np.int64)
    s1 = np.zeros((K, 128), np.float64)
    s2 = np.zeros(K, np.float64)
    step = 4_000_000
    for lo in range(0, N, step):
        hi = min(N, lo + step)
        part = oracle.aggregate(dequant(Xt[lo:hi], cs), lt[lo:hi].cpu().numpy(), K)
        count += part[0]
        s1 += part[1]
        s2 += part[2]
    idx = np.sort(np.random.default_rng(2027).choice(N, 20_000, replace=False))
    it = torch.as_tensor(idx, device="cuda")
    sub = oracle.linear(dequant(Xt[it], cs), lt[it].cpu().numpy(), K, agg=(count, s1, s2),
                        idx=np.arange(idx.shape[0]))
    assert sub["status"] == oracle.OK
    assert float(np.abs(s_gpu[idx] - sub["s"]).max()) <= TOL_SI
    # S is the FP64 mean of the s_i the kernel wrote ...
    assert abs(S_gpu - float(np.mean(s_gpu))) <= 1e-6
    # ... so its distance from the oracle's S over all 1e8 rows is the mean of
    # the per-row differences s_i - s_i(oracle).  The sampled rows estimate
    # that mean; the pairing cancels the spread of s_i itself, so five
    # standard errors of the differences bound it far below the 1e-4 stated
    # for the low-precision forms.  (The oracle's linear form over all 1e8
    # rows at K = 1000 would take minutes of host time.)
    diff = s_gpu[idx] - sub["s"]
    se = float(np.std(diff)) / np.sqrt(diff.size)
    assert abs(float(np.mean(diff))) + 5 * se <= 1e-4


def test_fp32_d128_k256_uses_two_cluster_blocks():
    # split centroids for 256 clusters, two A buffers and a raw stage exceed
    # shared memory, so the tensor path runs two blocks of 128 clusters
    X, lab = case(7, 3000, 128, 256)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 256)
    rt = sil.score(Xt, lt, 256, agg, want_s=True, path="tensor")
    rs = sil.score(Xt, lt, 256, agg, want_s=True, path="simt")
    torch.cuda.synchronize()
    assert float((rt.s - rs.s).abs().max()) <= TOL_SI
    assert abs(float(rt.S) - float(rs.S)) <= TOL_S


def test_tensor_refuses_ineligible_shapes():
    X, lab = case(6, 500, 8, 3)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 3)
    with pytest.raises(sil.SilError):
        sil.score(Xt, lt, 3, agg, path="tensor")


@pytest.mark.parametrize("recipe", ["at_scale", "at_scale_tf32", "batched_labeling_0", "batched_labeling_0_tf32",
                                    "precision_bf16"])
def test_tensor_and_simt_agree_on_every_row_at_full_size(recipe):
    # every row, not a sample: a pipeline hazard that corrupts one row in a
    # million shows up here
    path = "tensor_tf32" if recipe.endswith("_tf32") else "tensor"
    if recipe.startswith("at_scale"):
        w = synth.workload_at_scale(device="cuda")
        X, lab, K = w.X, w.labels, w.K
    elif recipe.startswith("batched_labeling_0"):
        X, labs, ks = synth.workload_batched(device="cuda", B=1)
        lab, K = labs[0].contiguous(), ks[0]
    else:
        w = synth.workload_precision(device="cuda", N=20_000_000)
        X, lab, K = synth.to_bf16(w.X), w.labels, w.K
    agg = sil.aggregate(X, lab, K)
    rt = sil.score(X, lab, K, agg, want_s=True, save=True, path=path)
    rs = sil.score(X, lab, K, agg, want_s=True, save=True, path="simt")
    torch.cuda.synchronize()
    d = (rt.s - rs.s).abs()
    assert int((d > TOL_SI).sum()) == 0, (recipe, float(d.max()), int(d.argmax()))
    assert abs(float(rt.S) - float(rs.S)) <= TOL_S


# ------------------------------------------------ conditioning and launch plans
def _close_clusters(N, D, kmin, kmax, B=2):
    """Voronoi cells of k random points of a Gaussian-blob set: many clusters
    whose separation b_i is small next to ||x'||^2 (the ill-conditioned case
    of the expanded distance)."""
    X, labs, ks = synth.workload_batched(device="cuda", N=N, D=D, B=B, k_low=kmin, k_high=kmax)
    return X, labs, ks


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("dtype,D,path", [(torch.float32, 64, "tensor"), (torch.float32, 64, "tensor_tf32"),
                                          (torch.bfloat16, 64, "tensor"), (torch.float32, 32, "tensor"),
                                          (torch.float32, 32, "tensor_tf32"), (torch.float32, 160, "tensor")])
def test_close_clusters_match_the_oracle_without_bias(dtype, D, path, metric):
    # b_i of such rows comes from the difference form, so the error of S is
    # not the tensor cores' round-towards-zero bias times the cancellation.
    # D = 160 runs the chunked kernel, which reads such rows back from
    # global memory; D = 32 the 64-byte-swizzled one.
    X, labs, ks = _close_clusters(100_000 if D <= 64 else 40_000, D, 250, 450)
    Xs = X.to(dtype)
    for b, k in enumerate(ks):
        lab = labs[b].contiguous()
        agg = sil.aggregate(Xs, lab, k, metric)
        r = sil.score(Xs, lab, k, agg, metric, want_s=True, save=True, path=path)
        torch.cuda.synchronize()
        ref = oracle.linear(dequant(Xs), lab.cpu().numpy(), k, metric)
        assert abs(float(r.S) - ref["S"]) <= TOL_S, (k, float(r.S) - ref["S"])
        _, bt, _ = sil.unpack_saved(r.saved, X.shape[0])
        rel = (bt.cpu().double().numpy() - ref["b"]) / ref["b"]
        assert abs(float(np.mean(rel))) <= 2e-7, (k, float(np.mean(rel)))
        assert float((r.s.cpu().double() - torch.from_numpy(ref["s"])).abs().max()) <= TOL_SI


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("save", [False, True])
@pytest.mark.parametrize("dtype,D,k", [(torch.float32, 64, 120), (torch.float32, 32, 200), (torch.float32, 64, 400),
                                       (torch.bfloat16, 64, 120), (torch.bfloat16, 128, 400),
                                       (torch.float8_e4m3fn, 128, 120), (torch.float8_e4m3fn, 128, 400)])
def test_ill_conditioned_rows_are_finished_in_the_difference_form(metric, save, dtype, D, k):
    # Voronoi cells: most rows' expanded form is ill-conditioned, so b_i of
    # those rows is the GEMM's nearest cluster recomputed in the difference
    # form (one cluster block for k <= 256, two blocks and the combine kernel
    # above).  Every s_i, b_i and argmin against the oracle, with and without
    # the backward record (the argmin tracked in the main pass and the row
    # read from the A buffer, or found by a second pass over the accumulator
    # and the row read back from global memory), for every storage type.
    X, labs, ks = _close_clusters(30_000, D, k, k, B=1)
    lab = labs[0].contiguous()
    cs = None
    if dtype == torch.float8_e4m3fn:
        X, cs = synth.to_fp8_e4m3(X)
    else:
        X = X.to(dtype)
    agg = sil.aggregate(X, lab, k, metric, col_scale=cs)
    r = sil.score(X, lab, k, agg, metric, col_scale=cs, want_s=True, save=save, path="tensor")
    torch.cuda.synchronize()
    ref = oracle.linear(dequant(X, cs), lab.cpu().numpy(), k, metric)
    assert_scores(r.s, r.S, ref, what=f"close {metric} {dtype} D={D} k={k} save={save}")
    if save:
        a, b, ks_ = sil.unpack_saved(r.saved, X.shape[0])
        np.testing.assert_allclose(b.cpu().double().numpy(), ref["b"], rtol=1e-4, atol=1e-4)
        assert np.mean(ks_.cpu().numpy() == ref["kstar"]) > 0.999


@pytest.mark.parametrize("shape", ["close_d32", "blobs_d64", "close_d64_two_blocks"])
def test_every_plan_gives_the_same_scores(shape):
    # block widths, ring depths, staged or unstaged centroids and both rank
    # passes: the same s_i (bit for bit between the two rank passes of one
    # layout, whose MMAs are identical).  Across block widths a row can differ
    # where two clusters are nearly tied: the GEMM ranks them to ~1e-6 and
    # only the winner of each block is recomputed exactly, so a split of the
    # pair over two blocks recovers the true minimum.
    if shape == "blobs_d64":
        w = synth.workload_at_scale(device="cuda", N=60_000)
        X, lab, K = w.X, w.labels, w.K
    else:
        D = 32 if shape == "close_d32" else 64
        X, labs, ks = _close_clusters(60_000, D, 300, 300 if D == 32 else 500, B=1)
        lab, K = labs[0].contiguous(), ks[0]
    D = X.shape[1]
    agg = sil.aggregate(X, lab, K)
    plans = sil.tensor_plan_candidates(X.dtype, D, K, 12)
    assert any(p[4] == 1 for p in plans) and any(p[4] == 0 for p in plans)
    out = {}
    try:
        for p in plans:
            sil.tensor_plan_set(X.dtype, D, K, p)
            r = sil.score(X, lab, K, agg, want_s=True, path="tensor")
            torch.cuda.synchronize()
            out[p] = (r.s.clone(), float(r.S))
    finally:
        sil.tensor_plan_set(X.dtype, D, K, None)
    s0, S0 = out[plans[0]]
    for p, (s, S) in out.items():
        twin = p[:4] + (1 - p[4],)
        if twin in out:
            assert torch.equal(s, out[twin][0]), p
        assert float((s - s0).abs().max()) <= 2e-5, p
        assert abs(S - S0) <= 1e-7, p  # FP32 partial sums in another grid order


def test_autotune_keeps_a_plan_that_scores_correctly():
    X, labs, ks = _close_clusters(50_000, 32, 150, 150, B=1)
    lab, K = labs[0].contiguous(), ks[0]
    try:
        res = sil.autotune(X, lab, K, max_plans=4, reps=1)
        assert len(res) == 4 and all(t > 0 for t, _ in res)
        agg = sil.aggregate(X, lab, K)
        r = sil.score(X, lab, K, agg, path="tensor")
        torch.cuda.synchronize()
        ref = oracle.linear(X.cpu().double().numpy(), lab.cpu().numpy(), K)
        assert abs(float(r.S) - ref["S"]) <= TOL_S
    finally:
        sil.tensor_plan_set(X.dtype, 32, K, None)
