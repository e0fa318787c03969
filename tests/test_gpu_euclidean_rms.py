"""The approximate Euclidean Silhouette of the Limitations section (a_i and b_i
the square roots of the point-to-cluster mean squared distances) on every
pass-2 kernel and entry point, against the oracle's linear form of it (which
the CPU pins tie to its quadratic definition, to Jensen's bound on the exact
Euclidean Silhouette and to a case where the two agree)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, assert_scores, case, dequant, to_dev
from paper_2303_14102_gb300 import sil

pytestmark = pytest.mark.gpu
M = "euclidean_rms"


def score(Xt, lt, K, path="auto"):
    st = sil.new_status(Xt.device)
    agg = sil.aggregate(Xt, lt, K, M, status=st)
    r = sil.score(Xt, lt, K, agg, M, want_s=True, path=path, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return agg, r


@pytest.mark.parametrize("path,dtype,N,D,K", [
    ("simt", torch.float32, 3001, 6, 5),        # centroids in shared memory
    ("simt", torch.float32, 2000, 300, 7),      # rows wider than the register tile
    ("tensor", torch.float32, 5000, 64, 20),    # tcgen05, FP32 split into BF16 hi + lo
    ("tensor", torch.float32, 4000, 64, 300),   # two cluster blocks and the combine kernel
    ("tensor_tf32", torch.float32, 5000, 64, 20),   # tcgen05, TF32 ranking, exact FP32 candidates
    ("tensor_tf32", torch.float32, 4000, 64, 300),
    ("tensor", torch.float32, 3000, 160, 9),    # FP32 rows in 64-column chunks
    ("tensor", torch.bfloat16, 5000, 64, 20),   # BF16 storage
])
def test_every_kernel_against_the_oracle(path, dtype, N, D, K):
    X, lab = case(300 + D + K, N, D, K)
    Xt, lt = to_dev(X, lab, dtype)
    _, r = score(Xt, lt, K, path)
    ref = oracle.linear(dequant(Xt), lab, K, M)
    assert_scores(r.s, r.S, ref, what=f"{path} {dtype} D={D} K={K}")


def test_scores_are_the_monotone_image_of_the_squared_scores():
    # with r = a/b of the squared means: s_sq = 1 - r and s_rms = 1 - sqrt(r)
    # when a <= b, else s_sq = 1/r - 1 and s_rms = 1/sqrt(r) - 1
    X, lab = case(77, 20000, 64, 30)
    Xt, lt = to_dev(X, lab)
    sq = sil.silhouette(Xt, lt, 30, "sqeuclidean", want_s=True).s.double().cpu().numpy()
    rms = sil.silhouette(Xt, lt, 30, M, want_s=True).s.double().cpu().numpy()
    expect = np.where(sq >= 0, 1 - np.sqrt(np.clip(1 - sq, 0, None)), np.sqrt(1 + sq) - 1)
    np.testing.assert_allclose(rms, expect, rtol=0, atol=1e-5)


def test_batched_no_workspace_and_chunked_entry_points():
    X, lab = case(91, 6000, 16, 9)
    Xt, lt = to_dev(X, lab)
    ref = oracle.linear(X.astype(np.float64), lab, 9, M)
    # batched: several labelings of the same rows
    rng = np.random.default_rng(5)
    ks = [9, 4, 23]
    labs = np.stack([lab] + [rng.integers(0, k, size=6000).astype(np.int32) for k in ks[1:]])
    S = sil.score_batched(Xt, torch.as_tensor(labs).cuda(), ks, M).cpu().numpy()
    for b, k in enumerate(ks):
        assert abs(S[b] - oracle.linear(X.astype(np.float64), labs[b], k, M)["S"]) <= TOL_S, b
    # the entry point without a workspace
    agg = sil.aggregate(Xt, lt, 9, M)
    got = sil.score_noalloc(Xt, lt, 9, agg, M, want_s=True)
    assert_scores(got.s, got.S, ref, what="noalloc")
    # host data streamed in row chunks
    r = sil.silhouette_chunked(torch.from_numpy(X), torch.from_numpy(lab), 9, M, chunk_rows=1700,
                               want_s=True)
    assert abs(r.S - ref["S"]) <= TOL_S
    assert float(np.abs(r.s.double().numpy() - ref["s"]).max()) <= TOL_SI


def test_no_gradient_for_the_approximation():
    X, lab = case(92, 500, 4, 3)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 3, M)
    with pytest.raises(sil.SilError):
        sil.score_backward(Xt, lt, 3, agg, M)
