"""Out-of-core streaming: data held in host memory, streamed through the GPU in
row chunks (pass 1 accumulating one set of aggregates, pass 2 scoring every
chunk against them), gives the oracle's S and s_i and the resident call's."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, case
from paper_2303_14102_gb300 import sil

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
@pytest.mark.parametrize("chunk", [7000, 1 << 22])  # eight chunks with a ragged tail; one chunk
def test_chunked_matches_oracle_and_resident_call(metric, chunk):
    N, D, K = 50_001, 16, 7
    X, lab = case(5, N, D, K, metric)
    ref = oracle.linear(X.astype(np.float64), lab, K, metric)
    Xh, lh = torch.from_numpy(X).pin_memory(), torch.from_numpy(lab).pin_memory()
    r = sil.silhouette_chunked(Xh, lh, K, metric, chunk_rows=chunk, want_s=True)
    assert r.chunks == -(-N // chunk)
    assert abs(r.S - ref["S"]) <= TOL_S
    assert float(np.abs(r.s.double().numpy() - ref["s"]).max()) <= TOL_SI
    # the same kernels on resident data: only the FP64 summation order of the
    # aggregates (and of S) differs
    dev = sil.silhouette(Xh.cuda(), lh.cuda(), K, metric, want_s=True)
    assert abs(r.S - float(dev.S)) <= 1e-7
    np.testing.assert_allclose(r.s.numpy(), dev.s.cpu().numpy(), rtol=0, atol=1e-5)


def test_chunked_bf16_from_pageable_memory():
    N, D, K = 20_000, 40, 9
    X, lab = case(6, N, D, K)
    Xb = torch.from_numpy(X).to(torch.bfloat16)  # not pinned: the copies are synchronous
    r = sil.silhouette_chunked(Xb, torch.from_numpy(lab), K, chunk_rows=3001)
    assert r.chunks == 7 and r.s is None
    ref = oracle.linear(Xb.double().numpy(), lab, K)
    assert abs(r.S - ref["S"]) <= TOL_S


def test_chunked_reports_a_bad_label():
    X, lab = case(7, 5000, 8, 4)
    lab[4321] = 4  # outside [0, K)
    with pytest.raises(sil.SilError):
        sil.silhouette_chunked(torch.from_numpy(X), torch.from_numpy(lab), 4, chunk_rows=1000)


def test_chunk_mean_is_the_row_weighted_mean():
    import numpy as np
    S = torch.tensor([0.5, 0.25, -0.125, 1.0], dtype=torch.float64, device="cuda")
    n = torch.tensor([3, 1, 8, 2], dtype=torch.int64, device="cuda")
    got = float(sil.chunk_mean(S, n))
    ref = float(np.sum(S.cpu().numpy() * n.cpu().numpy()) / n.sum().item())
    assert got == pytest.approx(ref, rel=1e-15, abs=1e-15)
    S[1] = float("nan")
    assert np.isnan(float(sil.chunk_mean(S, n)))
