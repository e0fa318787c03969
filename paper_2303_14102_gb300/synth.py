"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no Silhouette arithmetic: it only draws Gaussian-blob
points, cluster sizes and labelings, and stores them in the requested
precision.  Both the CUDA path and the FP64 oracle are fed from here.

The paper's own experiment uses a proprietary 129-feature dataset (Sec. IV)
that is not available; these generators stand in for it with the shapes and
structure of the workloads measured here:

  small       N=10,000, D=8, K=5; centres U[-10,10]^D, sigma=1, equal sizes
  at_scale    N=10,000,000, D=64, K=100; centres U[-5,5]^D, sigma=1,
              truncated rank-Zipf(1.1) sizes, shuffled point order
  precision   N=100,000,000, D=128, K=1,000; centres at radius 1e3 (uniform
              directions), sigma=1, equal sizes; bf16 or fp8-e4m3 storage
  batched     N=2,000,000, D=32 blobs; 256 labelings, each nearest-of-k to
              k distinct sampled points, k ~ U{2..512}
  grad        N=1,000,000, D=256, K=1,000; centres U[-5,5]^D, sigma=1,
              equal sizes, rows normalised to unit length
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

SEED_BASE = 20230324


def zipf_sizes(N: int, K: int, exponent: float = 1.1) -> np.ndarray:
    """Truncated rank-Zipf sizes w_r ~ r^-exponent, r=1..K, summing exactly to N.

    Counts are the floors of the exact shares plus one for the largest
    remainders (ties to the lower rank).
    """
    w = np.arange(1, K + 1, dtype=np.float64) ** (-exponent)
    share = w / w.sum() * N
    counts = np.floor(share).astype(np.int64)
    rem = N - int(counts.sum())
    order = np.argsort(-(share - counts), kind="stable")
    counts[order[:rem]] += 1
    return counts


def equal_sizes(N: int, K: int) -> np.ndarray:
    counts = np.full(K, N // K, dtype=np.int64)
    counts[: N % K] += 1
    return counts


@dataclasses.dataclass
class Blobs:
    X: torch.Tensor          # N x D float32 (the values the method sees, before storage casts)
    labels: torch.Tensor     # N int32, dense ids in [0, K)
    centers: torch.Tensor    # K x D float32
    K: int


def blobs(N: int, D: int, K: int, *, seed: int, center_low: float = -5.0, center_high: float = 5.0,
          sphere_radius: float | None = None, sigma: float = 1.0, sizes: str = "equal",
          shuffle: bool = True, normalize: bool = False, device: str = "cpu") -> Blobs:
    """Gaussian mixture points with the generating component as label.

    Centres are uniform in [center_low, center_high]^D, or, with
    ``sphere_radius``, uniform directions scaled to that radius.  Cluster
    sizes are equal or truncated rank-Zipf(1.1).  With ``shuffle`` the point
    order is a seeded random permutation so labels are unsorted.  With
    ``normalize`` every row is scaled to unit length (a unit-norm embedding
    set).  All draws come from one torch generator on ``device``.
    """
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    if sphere_radius is not None:
        u = torch.randn(K, D, generator=g, device=device, dtype=torch.float64)
        centers = (u / u.norm(dim=1, keepdim=True) * sphere_radius).to(torch.float32)
    else:
        centers = (torch.rand(K, D, generator=g, device=device, dtype=torch.float64)
                   * (center_high - center_low) + center_low).to(torch.float32)
    counts = zipf_sizes(N, K) if sizes == "zipf" else equal_sizes(N, K)
    labels = torch.repeat_interleave(torch.arange(K, device=device, dtype=torch.int32),
                                     torch.as_tensor(counts, device=device))
    if shuffle:
        perm = torch.randperm(N, generator=g, device=device)
        labels = labels[perm]
    X = torch.randn(N, D, generator=g, device=device, dtype=torch.float32)
    X.mul_(sigma)
    X.add_(centers[labels.long()])
    if normalize:
        X.div_(X.norm(dim=1, keepdim=True))
    return Blobs(X=X, labels=labels.contiguous(), centers=centers, K=K)


def workload_small(device: str = "cpu", N: int = 10_000, D: int = 8, K: int = 5) -> Blobs:
    return blobs(N, D, K, seed=SEED_BASE + 0, center_low=-10.0, center_high=10.0, device=device)


def workload_at_scale(device: str = "cpu", N: int = 10_000_000, D: int = 64, K: int = 100) -> Blobs:
    return blobs(N, D, K, seed=SEED_BASE + 1, center_low=-5.0, center_high=5.0, sizes="zipf",
                 device=device)


def workload_precision(device: str = "cpu", N: int = 100_000_000, D: int = 128,
                       K: int = 1000) -> Blobs:
    return blobs(N, D, K, seed=SEED_BASE + 2, sphere_radius=1e3, device=device)


def workload_grad(device: str = "cpu", N: int = 1_000_000, D: int = 256, K: int = 1000) -> Blobs:
    return blobs(N, D, K, seed=SEED_BASE + 4, center_low=-5.0, center_high=5.0, normalize=True,
                 device=device)


def workload_batched(device: str = "cpu", N: int = 2_000_000, D: int = 32, B: int = 256,
                     k_low: int = 2, k_high: int = 512, blob_K: int = 64):
    """One blob dataset and B labelings (B x N int32) with k_b ~ U{k_low..k_high}.

    Labeling b takes k_b distinct points of the dataset (sampled without
    replacement, seeded per labeling) as centres and gives every point the
    index of its nearest centre by squared distance (ties to the lower
    index), so cluster sizes are uneven.  Returns (X, labels, ks).
    """
    base = blobs(N, D, blob_K, seed=SEED_BASE + 3, device=device)
    X = base.X
    g = torch.Generator(device="cpu")
    g.manual_seed(SEED_BASE + 3)
    ks = torch.randint(k_low, k_high + 1, (B,), generator=g).tolist()
    labels = torch.empty(B, N, dtype=torch.int32, device=device)
    for b, k in enumerate(ks):
        gb = torch.Generator(device="cpu")
        gb.manual_seed(SEED_BASE + 1000 + b)
        idx = torch.randperm(N, generator=gb)[:k].to(device)
        C = X[idx]
        cc = (C * C).sum(1)[None, :]
        for lo in range(0, N, 1 << 18):
            hi = min(N, lo + (1 << 18))
            # ||x||^2 is common to every centre of a row, so it does not change the argmin
            d = cc - 2.0 * (X[lo:hi] @ C.T)
            labels[b, lo:hi] = d.argmin(dim=1).to(torch.int32)
    return X, labels, ks


def to_bf16(X: torch.Tensor) -> torch.Tensor:
    """Round-to-nearest-even bf16 storage of X."""
    return X.to(torch.bfloat16)


def to_fp8_e4m3(X: torch.Tensor):
    """FP8 E4M3 storage with one positive scale per column: X ~= q * scale.

    scale_l = max_i |x_il| / 448 (448 is the largest finite E4M3 value), so
    every scaled value is representable; q is X / scale rounded to E4M3.
    Returns (q as torch.float8_e4m3fn, scale float32[D]).
    """
    amax = X.abs().amax(dim=0).to(torch.float32)
    scale = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
    q = (X / scale[None, :]).to(torch.float8_e4m3fn)
    return q, scale


def dequantize(q: torch.Tensor, scale: torch.Tensor | None = None) -> torch.Tensor:
    """The values a kernel sees for stored q (and per-column scale), as float64."""
    x = q.to(torch.float64)
    if scale is not None:
        x = x * scale.to(torch.float64)[None, :]
    return x
