"""torch.autograd.Function around libsil: S as a differentiable loss of X.

forward  = sil_aggregate + sil_score (saving a_i, b_i and b_i's argmin k*_i,
           12 bytes per point; the N x K distances are never stored)
backward = sil_score_backward: dS/dX with the labels fixed and k*_i held at
           its forward value (the min and max of Eq. 1 as subgradients)
"""
from __future__ import annotations

import torch

from . import sil


class SilhouetteFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, labels, K, metric, col_scale):
        agg = sil.aggregate(X, labels, K, metric, col_scale=col_scale)
        res = sil.score(X, labels, K, agg, metric, col_scale=col_scale, save=True)
        ctx.save_for_backward(X, labels, *agg, res.saved)
        ctx.K, ctx.metric, ctx.col_scale = K, metric, col_scale
        ctx.mark_non_differentiable(labels)
        return res.S

    @staticmethod
    def backward(ctx, gS):
        X, labels, count, s1, s2, saved = ctx.saved_tensors
        dX = sil.score_backward(X, labels, ctx.K, (count, s1, s2), ctx.metric, saved=saved,
                                grad_S=gS, col_scale=ctx.col_scale)
        return dX.to(X.dtype), None, None, None, None


def silhouette_loss(X: torch.Tensor, labels: torch.Tensor, K: int, metric: str = "sqeuclidean",
                    col_scale: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable Silhouette S of X (0-d float64 tensor)."""
    if metric not in ("sqeuclidean", "cosine"):
        raise ValueError(f"no gradient for metric {metric!r}")
    return SilhouetteFn.apply(X, labels, K, metric, col_scale)
