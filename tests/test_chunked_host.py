"""Host logic of the out-of-core streaming call (no GPU): the row partition, the
identity the library's combination of per-chunk means relies on (pinned against
the oracle), and argument checks that answer before any device is touched."""
import numpy as np
import pytest
import torch

import oracle
from helpers import case
from paper_2303_14102_gb300 import sil


@pytest.mark.parametrize("N", [1, 9, 10, 11, 1000])
@pytest.mark.parametrize("chunk", [1, 3, 10, 4096])
def test_row_chunks_partition_the_rows(N, chunk):
    ch = sil.row_chunks(N, chunk)
    assert ch[0][0] == 0 and ch[-1][1] == N
    assert all(b == c for (_, b), (c, _) in zip(ch, ch[1:]))
    assert all(0 < b - a <= chunk for a, b in ch)
    assert len(ch) == -(-N // chunk)


def test_row_chunks_edge_cases():
    assert sil.row_chunks(0, 5) == []
    with pytest.raises(ValueError):
        sil.row_chunks(10, 0)
    with pytest.raises(ValueError):
        sil.row_chunks(-1, 5)


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_chunk_means_combine_to_the_mean_over_all_rows(metric):
    # a chunk scored against the aggregates of ALL rows has exactly those rows'
    # s_i; the row-weighted mean of the chunk means is S (Eq. 2 averaged over N)
    N, K = 900, 6
    X, lab = case(71, N, 5, K, metric)
    full = oracle.linear(X, lab, K, metric)
    chunks = sil.row_chunks(N, 250)
    parts = [oracle.linear(X, lab, K, metric, agg=full["agg"], idx=np.arange(a, b)) for a, b in chunks]
    for (a, b), p in zip(chunks, parts):
        np.testing.assert_allclose(p["s"], full["s"][a:b], rtol=0, atol=1e-15)
    n = np.array([b - a for a, b in chunks], dtype=np.float64)
    S = float(np.sum(n * np.array([p["S"] for p in parts])) / n.sum())  # what sil_chunk_mean computes
    assert abs(S - full["S"]) <= 1e-15
    assert abs(S - oracle.bruteforce(X, lab, K, metric)["S"]) <= 1e-12


def test_chunk_mean_rejects_bad_arguments():
    lib = sil.load()
    fake = __import__("ctypes").c_void_p(256)  # never dereferenced: refused on the host
    assert lib.sil_chunk_mean(fake, fake, 0, fake, None) == sil.SIL_EINVAL
    assert lib.sil_chunk_mean(None, fake, 3, fake, None) == sil.SIL_EINVAL
    assert lib.sil_chunk_mean(fake, fake, 3, None, None) == sil.SIL_EINVAL


def test_streaming_call_checks_arguments_before_touching_a_device():
    X = torch.zeros(10, 3)
    with pytest.raises(ValueError, match="int32"):
        sil.silhouette_chunked(X, torch.zeros(10, dtype=torch.int64), 2)
    with pytest.raises(ValueError, match="2-D"):
        sil.silhouette_chunked(torch.zeros(10), torch.zeros(10, dtype=torch.int32), 2)
    with pytest.raises(ValueError, match="one label per row"):
        sil.silhouette_chunked(X, torch.zeros(9, dtype=torch.int32), 2)
    with pytest.raises(ValueError, match="no rows"):
        sil.silhouette_chunked(torch.zeros(0, 3), torch.zeros(0, dtype=torch.int32), 2)
    with pytest.raises(ValueError, match="positive"):
        sil.silhouette_chunked(X, torch.zeros(10, dtype=torch.int32), 2, chunk_rows=0)
