"""The error band of the TF32-ranked tensor-core pass 2, checked on the CPU.

The kernel ranks the clusters by v_k = cb_k - 2 inv acc_k with acc_k the
tensor-core product of x and mu'_k read as TF32 (10 mantissa bits) and summed
in FP32, and recomputes exactly every cluster with v_k <= min + 2E, where

    E = 2^-8 (1 + 2^-6) inv ||x|| R + 2^-22 (C + 2 inv ||x|| R),
    R = max_k ||mu'_k||,  C = max_k |cb_k|.

Here the same arithmetic is simulated in numpy (operands truncated to TF32,
products exact, FP32 accumulation in a random order, FP32 cb and FMA) on the
workload recipes and on adversarial inputs, and two facts are checked: every
ranked value lies within E of its exact value, and the exact nearest cluster is
always among the candidates.  The mean number of candidates per row on the
at-scale recipe is bounded too (it sets the kernel's recompute cost).
"""
import numpy as np
import pytest

from paper_2303_14102_gb300 import synth

E_REL = 2.0 ** -8 * (1 + 2.0 ** -6)
E_ABS = 2.0 ** -22


def tf32(a):
    """Truncate float32 values to TF32 (keep the top 10 mantissa bits)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def simulate(X, labels, K, cosine, rng):
    X = X.astype(np.float64)
    Xn = X / np.linalg.norm(X, axis=1, keepdims=True) if cosine else X
    n = np.bincount(labels, minlength=K).astype(np.float64)
    s1 = np.zeros((K, X.shape[1]))
    np.add.at(s1, labels, Xn)
    s2 = np.bincount(labels, weights=(Xn * Xn).sum(1), minlength=K)
    g = s1.sum(0) / n.sum()
    mu = s1 / n[:, None]
    W = s2 - (s1 * s1).sum(1) / n
    mup = (mu - g).astype(np.float32)                       # mu'_k as the kernel stores it
    bias = (mup.astype(np.float64) ** 2).sum(1) + W / n
    cb = (bias + 2 * mup.astype(np.float64) @ g).astype(np.float32)
    x32 = X.astype(np.float32)
    inv = (1.0 / np.linalg.norm(X, axis=1)) if cosine else np.ones(X.shape[0])
    # tensor-core product: TF32 operands, exact products, FP32 sums in a random order
    prod = tf32(x32)[:, None, :].astype(np.float32) * tf32(mup)[None, :, :]
    order = rng.permutation(X.shape[1])
    acc = np.zeros(prod.shape[:2], np.float32)
    for l in order:
        acc = (acc + prod[:, :, l]).astype(np.float32)
    v = (cb[None, :].astype(np.float32) + np.float32(-2.0) * inv[:, None].astype(np.float32) * acc).astype(np.float32)
    # exact: v_k = bias_k - 2 x'.mu'_k (with the FP32 mu' the kernel also uses)
    xp = Xn - g
    v_exact = bias[None, :] - 2 * xp @ mup.astype(np.float64).T
    R = float(np.linalg.norm(mup.astype(np.float64), axis=1).max())
    C = float(np.abs(cb).max())
    xr = inv * np.linalg.norm(X, axis=1) * R
    E = E_REL * xr + E_ABS * (C + 2 * xr)
    return v.astype(np.float64), v_exact, E


CASES = {
    "at_scale": lambda: synth.workload_at_scale(N=4000),
    "small_d32_k300": lambda: synth.blobs(4000, 32, 300, seed=3),
    "far_from_origin": lambda: synth.blobs(3000, 64, 40, seed=4, sphere_radius=1e3),
    "tight_blobs": lambda: synth.blobs(3000, 64, 64, seed=5, sigma=0.01, center_low=-0.1, center_high=0.1),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cosine", [False, True])
def test_ranked_values_lie_within_the_band(name, cosine):
    w = CASES[name]()
    X, lab = w.X.numpy(), w.labels.numpy()
    v, v_exact, E = simulate(X, lab, w.K, cosine, np.random.default_rng(0))
    err = np.abs(v - v_exact)
    assert np.all(err <= E[:, None]), float((err / E[:, None]).max())


@pytest.mark.parametrize("name", list(CASES))
def test_the_nearest_cluster_is_always_a_candidate(name):
    w = CASES[name]()
    X, lab = w.X.numpy(), w.labels.numpy()
    v, v_exact, E = simulate(X, lab, w.K, False, np.random.default_rng(1))
    rows = np.arange(X.shape[0])
    v[rows, lab] = np.inf              # own cluster excluded from b_i
    v_exact[rows, lab] = np.inf
    m = v.min(1)
    cand = v <= (m + 2 * E)[:, None]
    assert np.all(cand[rows, v_exact.argmin(1)])
    if name == "at_scale":
        assert cand.sum(1).mean() < 2.0, cand.sum(1).mean()
