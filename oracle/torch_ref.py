"""Differentiable quadratic Silhouette in plain PyTorch CPU ops (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The same definition
as ``oracle_bruteforce`` in ``sil_oracle.c`` -- Eq. 1-3 and the mean S of
Sec. II, pairwise distances Eq. 4 (squared Euclidean) or 1 - cs of Eq. 12
(cosine) -- written with tensor ops so that ``torch.autograd`` gives dS/dX
with labels fixed.  O(N^2 D) memory and time: tiny inputs only.
"""
from __future__ import annotations

import torch


def pairwise(X: torch.Tensor, metric: str) -> torch.Tensor:
    """N x N distance matrix with an exactly-zero diagonal (self excluded)."""
    if metric == "sqeuclidean":
        diff = X[:, None, :] - X[None, :, :]
        Dm = (diff * diff).sum(-1)
    elif metric == "cosine":
        Xh = X / X.norm(dim=1, keepdim=True)
        Dm = 1.0 - Xh @ Xh.T
    else:
        raise ValueError(metric)
    eye = torch.eye(X.shape[0], dtype=torch.bool)
    return Dm.masked_fill(eye, 0.0)


def silhouette(X: torch.Tensor, labels: torch.Tensor, K: int, metric: str = "sqeuclidean"):
    """Returns (S, s) for FP64 X (N x D) and int labels in [0, K)."""
    if X.dtype != torch.float64:
        raise TypeError("the reference works in float64")
    labels = labels.long()
    N = X.shape[0]
    onehot = torch.nn.functional.one_hot(labels, K).to(torch.float64)  # N x K
    counts = onehot.sum(0)  # N_k
    sums = pairwise(X, metric) @ onehot  # sum of distances from i to cluster k
    own_n = counts[labels]
    own_sum = sums.gather(1, labels[:, None])[:, 0]
    a = torch.where(own_n > 1, own_sum / (own_n - 1).clamp(min=1), torch.zeros_like(own_sum))
    means = sums / counts.clamp(min=1)
    blocked = onehot.bool() | (counts == 0)[None, :]
    b = means.masked_fill(blocked, float("inf")).min(dim=1).values
    m = torch.maximum(a, b)
    ok = (own_n > 1) & torch.isfinite(b) & (m > 0)
    s = torch.where(ok, (b - a) / torch.where(ok, m, torch.ones_like(m)), torch.zeros_like(m))
    return s.sum() / N, s
