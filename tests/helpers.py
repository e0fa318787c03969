"""Shared helpers for the GPU parity tests: seeded inputs and comparisons.

The expected values always come from the FP64 oracle (``oracle``) run on the
exact values the GPU sees (storage casts are undone exactly in FP64)."""
from __future__ import annotations

import numpy as np
import torch

# Tolerances stated for the FP32 path: |dS| <= 1e-6, |ds_i| <= 1e-4.
TOL_S = 1e-6
TOL_SI = 1e-4


def case(seed, N, D, K, metric="sqeuclidean", empty=True, singleton=True, spread=3.0):
    """Small clustered inputs with an unused label id and a one-point cluster."""
    rng = np.random.default_rng(seed)
    C = rng.uniform(-spread, spread, size=(K, D))
    lab = rng.integers(0, K, size=N).astype(np.int32)
    if empty and K > 3:
        lab[lab == K - 2] = 0
    if singleton and K > 2 and N > 2:
        lab[lab == K - 1] = 1
        lab[N // 2] = K - 1
    X = (C[lab] + rng.normal(size=(N, D))).astype(np.float32)
    if metric == "cosine":
        X += (0.1 * np.sign(X)).astype(np.float32)
    return X, lab


def to_dev(X, lab, dtype=torch.float32):
    Xt = torch.as_tensor(X).cuda().to(dtype)
    return Xt, torch.as_tensor(lab).cuda()


def dequant(Xt, col_scale=None):
    x = Xt.detach().cpu().to(torch.float64)
    if col_scale is not None:
        x = x * col_scale.detach().cpu().to(torch.float64)[None, :]
    return x.numpy()


def assert_scores(s_gpu, S_gpu, ref, tol_si=TOL_SI, tol_S=TOL_S, what=""):
    s = s_gpu.detach().cpu().double().numpy()
    ds = np.abs(s - ref["s"])
    assert float(ds.max(initial=0.0)) <= tol_si, f"{what} max|ds_i| = {ds.max()}"
    dS = abs(float(S_gpu) - ref["S"])
    assert dS <= tol_S, f"{what} |dS| = {dS} (gpu {float(S_gpu)}, oracle {ref['S']})"


def unique_argmin_mask(ref_b_all_margin, tol):
    return ref_b_all_margin > tol
