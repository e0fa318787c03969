"""Pins of the FP64 oracle against things other than itself (CPU only).

Each pin ties the oracle to the paper or to mathematics it cannot fake:
hand-worked examples (tests/golden, each citing the equations used), the
paper's claim that the linear form equals the quadratic definition (Sec.
III, Eq. 4-11 and 13-18), an independent third-party routine (scikit-learn's
silhouette_samples), invariances of the definition, closed-form special
cases, library sums for the aggregates, and finite differences plus torch
autograd for the gradient.
"""
import glob
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from oracle import torch_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def frac(x):
    return float(Fraction(x))


def small_case(seed, N=60, D=3, K=4, metric="sqeuclidean", empty=True, singleton=True):
    rng = np.random.default_rng(seed)
    C = rng.uniform(-3, 3, size=(K, D))
    labels = rng.integers(0, K, size=N).astype(np.int32)
    if empty and K > 2:
        labels[labels == K - 2] = 0  # label id K-2 becomes empty
    if singleton:
        labels[labels == K - 1] = 1
        labels[0] = K - 1  # a one-point cluster
    X = C[labels] + rng.normal(size=(N, D))
    if metric == "cosine":
        X += 0.1 * np.sign(X)  # keep rows away from zero
    return X, labels


# ---------------------------------------------------------------- golden
@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
@pytest.mark.parametrize("form", ["bruteforce", "linear"])
def test_golden_hand_worked(path, form):
    g = json.load(open(path))
    if form not in g.get("forms", ["bruteforce", "linear"]):
        pytest.skip(f"{g['metric']} has no {form} form")
    X = np.array(g["X"], dtype=np.float64)
    lab = np.array(g["labels"], dtype=np.int32)
    r = getattr(oracle, form)(X, lab, g["K"], g["metric"])
    s_ref = np.array([frac(v) for v in g["s"]])
    np.testing.assert_allclose(r["s"], s_ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r["S"], s_ref.mean(), rtol=0, atol=1e-14)
    if "a" in g:
        np.testing.assert_allclose(r["a"], [frac(v) for v in g["a"]], rtol=1e-14, atol=1e-14)
    if "b" in g:
        np.testing.assert_allclose(r["b"], [frac(v) for v in g["b"]], rtol=1e-14, atol=1e-14)
    if "kstar" in g:
        np.testing.assert_array_equal(r["kstar"], g["kstar"])


# ------------------------------------------- linear form == quadratic form
@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
@pytest.mark.parametrize("seed,N,D,K", [(1, 50, 2, 3), (2, 120, 5, 6), (3, 200, 8, 4),
                                        (4, 31, 1, 5), (5, 150, 3, 12)])
def test_linear_equals_bruteforce(metric, seed, N, D, K):
    if metric == "cosine" and D == 1:
        pytest.skip("1-D cosine distances are exactly 0 or 2: a, b = 0 up to rounding")
    X, lab = small_case(seed, N, D, K, metric)
    bf = oracle.bruteforce(X, lab, K, metric)
    li = oracle.linear(X, lab, K, metric)
    np.testing.assert_allclose(li["a"], bf["a"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(li["b"], bf["b"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(li["s"], bf["s"], rtol=0, atol=1e-11)
    np.testing.assert_array_equal(li["kstar"], bf["kstar"])
    assert abs(li["S"] - bf["S"]) < 1e-12


def test_linear_subset_indexing():
    X, lab = small_case(7, 80, 4, 5)
    full = oracle.linear(X, lab, 5)
    idx = np.array([79, 3, 3, 0, 41])
    sub = oracle.linear(X, lab, 5, idx=idx, agg=full["agg"])
    np.testing.assert_array_equal(sub["s"], full["s"][idx])
    np.testing.assert_array_equal(sub["kstar"], full["kstar"][idx])


# ----------------------------------------------- independent library routine
@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine", "euclidean"])
@pytest.mark.parametrize("seed", [11, 12])
def test_matches_sklearn(metric, seed):
    skm = pytest.importorskip("sklearn.metrics")
    X, lab = small_case(seed, 90, 4, 5, metric)
    ref = skm.silhouette_samples(X, lab, metric=metric)
    bf = oracle.bruteforce(X, lab, 5, metric)
    np.testing.assert_allclose(bf["s"], ref, rtol=0, atol=1e-12)


# ----------------------------------------------------------- invariances
@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_label_permutation(metric):
    X, lab = small_case(21, 70, 3, 5, metric)
    perm = np.random.default_rng(0).permutation(5).astype(np.int32)
    a = oracle.bruteforce(X, lab, 5, metric)
    b = oracle.bruteforce(X, perm[lab], 5, metric)
    np.testing.assert_allclose(a["s"], b["s"], atol=1e-13)
    np.testing.assert_array_equal(perm[a["kstar"]][a["kstar"] >= 0], b["kstar"][a["kstar"] >= 0])


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_point_permutation(metric):
    X, lab = small_case(22, 70, 3, 5, metric)
    p = np.random.default_rng(1).permutation(70)
    a = oracle.linear(X, lab, 5, metric)
    b = oracle.linear(X[p], lab[p], 5, metric)
    np.testing.assert_allclose(a["s"][p], b["s"], atol=1e-12)
    assert abs(a["S"] - b["S"]) < 1e-13


def test_translation_sqeuclidean():
    X, lab = small_case(23, 70, 3, 5)
    shift = np.array([1e3, -2e3, 5e2])
    a = oracle.bruteforce(X, lab, 5)
    b = oracle.bruteforce(X + shift, lab, 5)
    np.testing.assert_allclose(a["s"], b["s"], atol=1e-8)
    c = oracle.linear(X + shift, lab, 5)  # the closed form survives a large offset in FP64
    np.testing.assert_allclose(a["s"], c["s"], atol=1e-8)


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_global_scale(metric):
    X, lab = small_case(24, 70, 3, 5, metric)
    a = oracle.linear(X, lab, 5, metric)
    b = oracle.linear(X * 7.5, lab, 5, metric)
    np.testing.assert_allclose(a["s"], b["s"], atol=1e-12)


def test_row_scale_cosine():
    X, lab = small_case(25, 70, 3, 5, "cosine")
    w = np.random.default_rng(2).uniform(0.1, 10, size=(70, 1))
    a = oracle.bruteforce(X, lab, 5, "cosine")
    b = oracle.bruteforce(X * w, lab, 5, "cosine")
    np.testing.assert_allclose(a["s"], b["s"], atol=1e-12)


@pytest.mark.parametrize("form", ["bruteforce", "linear"])
def test_cosine_is_half_sqeuclidean_of_normalised_rows(form):
    # 1 - xhat.yhat = ||xhat - yhat||^2 / 2, and s_i ignores a common scale of distances
    X, lab = small_case(26, 80, 4, 5, "cosine")
    Xh = X / np.linalg.norm(X, axis=1, keepdims=True)
    f = getattr(oracle, form)
    c = f(X, lab, 5, "cosine")
    q = f(Xh, lab, 5, "sqeuclidean")
    np.testing.assert_allclose(c["s"], q["s"], atol=1e-12)
    np.testing.assert_allclose(2 * c["a"], q["a"], atol=1e-12)
    np.testing.assert_allclose(2 * c["b"], q["b"], atol=1e-12)


# ------------------------------------------------------- special cases
def test_range_and_singletons():
    X, lab = small_case(27, 100, 3, 6)
    r = oracle.bruteforce(X, lab, 6)
    assert np.all(r["s"] >= -1) and np.all(r["s"] <= 1)
    counts = np.bincount(lab, minlength=6)
    assert np.all(r["s"][counts[lab] == 1] == 0.0)


def test_duplicated_points_give_one():
    X = np.repeat(np.array([[0.0, 0.0], [3.0, 4.0], [-5.0, 1.0]]), [4, 6, 3], axis=0)
    lab = np.repeat(np.array([0, 1, 2], np.int32), [4, 6, 3])
    for form in ("bruteforce", "linear"):
        r = getattr(oracle, form)(X, lab, 3)
        np.testing.assert_allclose(r["s"], 1.0, atol=1e-14)
        assert r["S"] == pytest.approx(1.0, abs=1e-14)


def test_all_singletons_give_zero():
    X, _ = small_case(28, 12, 2, 3)
    lab = np.arange(12, dtype=np.int32)
    r = oracle.bruteforce(X, lab, 12)
    assert np.all(r["s"] == 0.0) and r["S"] == 0.0


def test_one_cluster_is_degenerate():
    X, _ = small_case(29, 10, 2, 3)
    r = oracle.bruteforce(X, np.zeros(10, np.int32), 3)
    assert r["status"] == oracle.EDEGENERATE and np.isnan(r["S"])


def test_empty_ids_are_ignored():
    X, lab = small_case(30, 80, 3, 4, empty=False, singleton=False)
    gap = np.array([0, 3, 5, 9], np.int32)[lab]  # same partition, ids spread over [0, 10)
    a = oracle.linear(X, lab, 4)
    b = oracle.linear(X, gap, 10)
    np.testing.assert_allclose(a["s"], b["s"], atol=1e-13)


def test_bad_label_and_zero_norm_rejected():
    X, lab = small_case(31, 20, 2, 3)
    bad = lab.copy()
    bad[5] = 3
    with pytest.raises(ValueError):
        oracle.bruteforce(X, bad, 3)
    Z = X.copy()
    Z[4] = 0.0
    with pytest.raises(ValueError):
        oracle.aggregate(Z, lab, 3, "cosine")


# ------------------------------------------------------------ aggregates
@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_aggregates_against_library_sums(metric):
    X, lab = small_case(32, 300, 5, 7, metric)
    count, s1, s2 = oracle.aggregate(X, lab, 7, metric)
    np.testing.assert_array_equal(count, np.bincount(lab, minlength=7))
    V = X / np.linalg.norm(X, axis=1, keepdims=True) if metric == "cosine" else X
    onehot = np.eye(7)[lab]
    np.testing.assert_allclose(s1, onehot.T @ V, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(s2, onehot.T @ np.einsum("ij,ij->i", V, V), rtol=1e-13, atol=1e-12)


def test_aggregates_merge_over_shards():
    # the per-worker partial sums of Sec. III-A (footnote to Eq. 6) add up
    X, lab = small_case(33, 301, 4, 6)
    whole = oracle.aggregate(X, lab, 6)
    parts = [oracle.aggregate(X[lo:hi], lab[lo:hi], 6) for lo, hi in [(0, 97), (97, 250), (250, 301)]]
    np.testing.assert_array_equal(sum(p[0] for p in parts), whole[0])
    np.testing.assert_allclose(sum(p[1] for p in parts), whole[1], rtol=1e-13)
    np.testing.assert_allclose(sum(p[2] for p in parts), whole[2], rtol=1e-13)


# -------------------------------------------------------------- gradient
def _tie_free(seed, metric, N=200, D=4, K=4):
    X, lab = small_case(seed, N, D, K, metric, empty=False, singleton=False)
    return X, lab


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_torch_reference_matches_c_bruteforce(metric):
    X, lab = _tie_free(41, metric)
    S, s = torch_ref.silhouette(torch.tensor(X), torch.tensor(lab), 4, metric)
    bf = oracle.bruteforce(X, lab, 4, metric)
    np.testing.assert_allclose(s.numpy(), bf["s"], atol=1e-12)


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_linear_grad_matches_autograd(metric):
    X, lab = _tie_free(42, metric)
    Xt = torch.tensor(X, requires_grad=True)
    S, _ = torch_ref.silhouette(Xt, torch.tensor(lab), 4, metric)
    S.backward()
    g = oracle.linear_grad(X, lab, 4, metric)
    np.testing.assert_allclose(g, Xt.grad.numpy(), rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("metric", ["sqeuclidean", "cosine"])
def test_linear_grad_matches_finite_differences(metric):
    X, lab = _tie_free(43, metric)
    g = oracle.linear_grad(X, lab, 4, metric, gS=1.0)
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(12):
        i, l = rng.integers(0, 200), rng.integers(0, 4)
        Xp, Xm = X.copy(), X.copy()
        Xp[i, l] += h
        Xm[i, l] -= h
        fd = (oracle.bruteforce(Xp, lab, 4, metric)["S"] - oracle.bruteforce(Xm, lab, 4, metric)["S"]) / (2 * h)
        assert abs(fd - g[i, l]) <= 1e-7 + 1e-5 * abs(g[i, l]), (i, l, fd, g[i, l])


def test_grad_invariants():
    # translation invariance: gradients sum to zero; scale invariance: sum_m x_m.g_m = 0
    X, lab = _tie_free(44, "sqeuclidean", N=300, D=5, K=6)
    g = oracle.linear_grad(X, lab, 6)
    np.testing.assert_allclose(g.sum(0), 0.0, atol=1e-12)
    assert abs((X * g).sum()) < 1e-11
    Xc, labc = _tie_free(45, "cosine", N=300, D=5, K=6)
    gc = oracle.linear_grad(Xc, labc, 6, "cosine")
    np.testing.assert_allclose((Xc * gc).sum(1), 0.0, atol=1e-13)  # per-row scale invariance


# ------------------------------------- Euclidean distance and its RMS approximation
# The Limitations section: the plain Euclidean distance has no aggregate form;
# the square root of each point-to-cluster mean of squared distances (RMS)
# approximates it.  The exact form is pinned to scikit-learn above and to a
# hand-worked example (tests/golden); the approximation to the quadratic
# definition, to Jensen's inequality and to a case where it is exact.
@pytest.mark.parametrize("seed,N,D,K", [(21, 60, 2, 3), (22, 150, 5, 6), (23, 31, 1, 5), (24, 120, 3, 9)])
def test_rms_linear_equals_bruteforce(seed, N, D, K):
    X, lab = small_case(seed, N, D, K)
    bf = oracle.bruteforce(X, lab, K, "euclidean_rms")
    li = oracle.linear(X, lab, K, "euclidean_rms")
    np.testing.assert_allclose(li["a"], bf["a"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(li["b"], bf["b"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(li["s"], bf["s"], rtol=0, atol=1e-11)
    np.testing.assert_array_equal(li["kstar"], bf["kstar"])
    assert abs(li["S"] - bf["S"]) < 1e-12


@pytest.mark.parametrize("seed", [31, 32])
def test_rms_bounds_the_euclidean_means_from_above(seed):
    # sqrt(mean d^2) >= mean d for every cluster (Jensen), hence for a_i and
    # for the minimum b_i
    X, lab = small_case(seed, 120, 4, 5)
    rms = oracle.bruteforce(X, lab, 5, "euclidean_rms")
    euc = oracle.bruteforce(X, lab, 5, "euclidean")
    assert np.all(rms["a"] >= euc["a"] - 1e-12)
    assert np.all(rms["b"] >= euc["b"] - 1e-12)
    assert np.any(rms["b"] > euc["b"] + 1e-3)  # and it is an approximation


def test_rms_is_exact_when_every_mean_runs_over_one_point():
    # one two-point cluster among singletons: every mean a scored point takes
    # is over a single distance, so RMS and plain Euclidean agree
    rng = np.random.default_rng(41)
    X = rng.normal(size=(9, 3))
    lab = np.array([0, 0, 1, 2, 3, 4, 5, 6, 7], dtype=np.int32)
    rms = oracle.bruteforce(X, lab, 8, "euclidean_rms")
    euc = oracle.bruteforce(X, lab, 8, "euclidean")
    np.testing.assert_allclose(rms["s"], euc["s"], rtol=0, atol=1e-14)
    assert np.count_nonzero(euc["s"]) == 2
    np.testing.assert_allclose(oracle.linear(X, lab, 8, "euclidean_rms")["s"], euc["s"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [51, 52])
def test_rms_score_is_a_monotone_function_of_the_squared_score(seed):
    # with r = a/b of the squared means, s_sq = 1 - r and s_rms = 1 - sqrt(r)
    # (a <= b); s_sq = 1/r - 1 and s_rms = 1/sqrt(r) - 1 (a > b): same sign,
    # smaller magnitude
    X, lab = small_case(seed, 100, 3, 5)
    sq = oracle.linear(X, lab, 5, "sqeuclidean")["s"]
    rms = oracle.linear(X, lab, 5, "euclidean_rms")["s"]
    expect = np.where(sq >= 0, 1 - np.sqrt(np.clip(1 - sq, 0, None)), np.sqrt(1 + sq) - 1)
    np.testing.assert_allclose(rms, expect, rtol=0, atol=1e-12)
    assert np.all(np.abs(rms) <= np.abs(sq) + 1e-15)


@pytest.mark.parametrize("metric", ["euclidean", "euclidean_rms"])
def test_euclidean_forms_are_translation_and_scale_invariant(metric):
    X, lab = small_case(61, 80, 3, 4)
    S = oracle.bruteforce(X, lab, 4, metric)["S"]
    assert abs(oracle.bruteforce(X + 7.5, lab, 4, metric)["S"] - S) < 1e-12
    assert abs(oracle.bruteforce(3.0 * X, lab, 4, metric)["S"] - S) < 1e-12


def test_exact_euclidean_has_no_linear_form():
    X, lab = small_case(62, 20, 2, 3)
    with pytest.raises(ValueError):
        oracle.linear(X, lab, 3, "euclidean")
    with pytest.raises(ValueError):
        oracle.linear_grad(X, lab, 3, "euclidean_rms")
