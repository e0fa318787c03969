"""Batched labelings (many labelings of the same rows, e.g. a k-sweep) scored
with one tensor-core launch for every labeling's pass 2, against the FP64
oracle and against the same call forced through one launch sequence per
labeling (SIL_BATCH_PER_LABELING=1).

The batch mixes block widths below and above 256 clusters (one TMEM
accumulator per tile instead of two), k = 2, a labeling with one cluster
(S = NaN for it only), empty label ids and singletons, both metrics, and a
CUDA-graph replay."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S
from paper_2303_14102_gb300 import sil, synth

pytestmark = pytest.mark.gpu


def labelings(X, ks, seed):
    """Nearest-of-k sampled points (the batched recipe) for each k."""
    rng = np.random.default_rng(seed)
    out = []
    for k in ks:
        C = X[rng.choice(X.shape[0], k, replace=False)]
        d = (C * C).sum(1)[None, :] - 2.0 * X @ C.T
        out.append(d.argmin(1).astype(np.int32))
    return np.stack(out)


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_one_launch_matches_oracle_and_per_labeling(metric, monkeypatch):
    w = synth.blobs(6000, 32, 40, seed=31)
    X = w.X.numpy()
    ks = [2, 17, 255, 256, 257, 300, 511, 512, 64]
    labs = labelings(X.astype(np.float64), ks, 32)
    labs[3][labs[3] == 7] = 0          # an empty label id
    labs[5][100] = 299                  # ... and a singleton (label 299 kept only here)
    labs[5][labs[5] == 299] = 298
    labs[5][100] = 299
    Xt, lt = torch.as_tensor(X).cuda(), torch.as_tensor(labs).cuda()
    st = sil.new_status(Xt.device)
    S = sil.score_batched(Xt, lt, ks, metric, status=st).cpu().numpy()
    assert int(st.item()) == 0
    monkeypatch.setenv("SIL_BATCH_PER_LABELING", "1")
    S_seq = sil.score_batched(Xt, lt, ks, metric).cpu().numpy()
    np.testing.assert_allclose(S, S_seq, rtol=0, atol=TOL_S)
    X64 = X.astype(np.float64)
    for b, k in enumerate(ks):
        ref = oracle.linear(X64, labs[b], k, metric)
        assert abs(S[b] - ref["S"]) <= TOL_S, (b, k, S[b], ref["S"])


def test_a_degenerate_labeling_is_nan_alone():
    w = synth.blobs(3000, 32, 10, seed=33)
    X = w.X.numpy()
    ks = [5, 3, 300]
    labs = labelings(X.astype(np.float64), ks, 34)
    labs[1][:] = 2  # one cluster: b undefined
    Xt, lt = torch.as_tensor(X).cuda(), torch.as_tensor(labs).cuda()
    st = sil.new_status(Xt.device)
    S = sil.score_batched(Xt, lt, ks, status=st).cpu().numpy()
    assert int(st.item()) & sil.SIL_EDEGENERATE
    assert np.isnan(S[1]) and np.isfinite(S[0]) and np.isfinite(S[2])
    for b in (0, 2):
        assert abs(S[b] - oracle.linear(X.astype(np.float64), labs[b], ks[b])["S"]) <= TOL_S


def test_graph_replay_of_the_one_launch_path():
    X, labs, ks = synth.workload_batched(device="cuda", N=50_000, B=12, k_high=512)
    direct = sil.score_batched(X, labs, ks).cpu().numpy()
    g = sil.BatchedGraph(X, labs, ks)
    for _ in range(2):
        np.testing.assert_allclose(g.run().cpu().numpy(), direct, rtol=0, atol=TOL_S)
    X64 = X.cpu().double().numpy()
    for b in (0, 11):
        assert abs(direct[b] - oracle.linear(X64, labs[b].cpu().numpy(), ks[b])["S"]) <= TOL_S


def test_autotuned_plan_scores_the_same():
    X, labs, ks = synth.workload_batched(device="cuda", N=40_000, B=6, k_high=512)
    assert sil.serves_one_launch(X, labs, ks)
    ref = sil.score_batched(X, labs, ks).cpu().numpy()
    try:
        res = sil.autotune_batched(X, labs, ks, reps=1)
        assert res["one_launch"] in [p for _, p in res["timings_ms"]]
        np.testing.assert_allclose(sil.score_batched(X, labs, ks).cpu().numpy(), ref, rtol=0, atol=TOL_S)
        for ranges, nab in ((1, 2), (64, 4)):
            sil.batched_plan_set(ranges, nab)
            np.testing.assert_allclose(sil.score_batched(X, labs, ks).cpu().numpy(), ref, rtol=0, atol=TOL_S)
    finally:
        sil.batched_plan_set(8, 0)
