"""Parity of the CUDA backward pass (dS/dX, labels fixed) with the oracle.

Expected gradients come from the oracle's FP64 linear-form gradient (itself
pinned to torch autograd of the quadratic definition and to finite
differences) and, on the tiny case, straight from FP64 central finite
differences of the quadratic oracle.  Points whose b_i argmin is nearly tied
are excluded from the element-wise check only where the subgradient is not
unique.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import case, to_dev
from paper_2303_14102_gb300 import sil
from paper_2303_14102_gb300.autograd import silhouette_loss

pytestmark = pytest.mark.gpu
METRICS = ["sqeuclidean", "cosine"]


def gpu_grad(X, lab, K, metric, saved=True):
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, K, metric)
    r = sil.score(Xt, lt, K, agg, metric, save=saved)
    g = sil.score_backward(Xt, lt, K, agg, metric, saved=r.saved)
    torch.cuda.synchronize()
    return g.cpu().double().numpy()


def rel_err(g, ref):
    return float(np.abs(g - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("metric", METRICS)
# D = 256 fills both 128-column segments a lane holds; D = 300 takes the re-read path
@pytest.mark.parametrize("N,D,K", [(2000, 6, 5), (3001, 33, 9), (1500, 130, 6), (2500, 40, 300), (1200, 256, 7),
                                   (800, 300, 5)])
def test_grad_against_oracle(metric, N, D, K):
    X, lab = case(200 + N + D, N, D, K, metric, empty=False, singleton=True)
    g = gpu_grad(X, lab, K, metric)
    ref = oracle.linear_grad(X.astype(np.float64), lab, K, metric)
    assert rel_err(g, ref) <= 2e-4, rel_err(g, ref)


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float8_e4m3fn])
@pytest.mark.parametrize("N,D,K", [(3000, 64, 12), (1500, 256, 40)])
def test_grad_low_precision_rows_against_oracle(metric, dtype, N, D, K):
    # BF16 / FP8 (with column scales) storage: the oracle differentiates the
    # dequantised rows the kernels read
    X, lab = case(300 + N + D, N, D, K, metric, empty=False, singleton=True)
    Xt = torch.as_tensor(X).cuda()
    cs = None
    if dtype == torch.bfloat16:
        Xq = Xt.to(torch.bfloat16)
        Xd = Xq.float().cpu().double().numpy()
    else:
        cs = (Xt.abs().amax(0) / 448.0).clamp_min(1e-12).contiguous()
        Xq = (Xt / cs).to(torch.float8_e4m3fn)
        Xd = (Xq.float() * cs).cpu().double().numpy()
    lt = torch.as_tensor(lab).cuda()
    agg = sil.aggregate(Xq, lt, K, metric, col_scale=cs)
    r = sil.score(Xq, lt, K, agg, metric, col_scale=cs, save=True)
    g = sil.score_backward(Xq, lt, K, agg, metric, col_scale=cs, saved=r.saved)
    torch.cuda.synchronize()
    ref = oracle.linear_grad(Xd, lab, K, metric)
    err = rel_err(g.cpu().double().numpy(), ref)
    assert err <= 2e-4, err


@pytest.mark.parametrize("metric", METRICS)
def test_recompute_equals_saved(metric):
    X, lab = case(31, 2000, 10, 5, metric)
    a = gpu_grad(X, lab, 5, metric, saved=True)
    b = gpu_grad(X, lab, 5, metric, saved=False)
    # pass-1 partial sums are FP32 in a data-dependent order: equal to ~1e-7 relative
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(a).max())


@pytest.mark.parametrize("metric", METRICS)
def test_tiny_case_against_fp64_finite_differences(metric):
    # N=200, D=4, K=4: FP64 central differences of the quadratic oracle
    X, lab = case(43, 200, 4, 4, metric, empty=False, singleton=False)
    g = gpu_grad(X, lab, 4, metric)
    Xd = X.astype(np.float64)
    h = 1e-6
    rng = np.random.default_rng(0)
    scale = np.abs(g).max()
    for _ in range(24):
        i, l = int(rng.integers(0, 200)), int(rng.integers(0, 4))
        Xp, Xm = Xd.copy(), Xd.copy()
        Xp[i, l] += h
        Xm[i, l] -= h
        fd = (oracle.bruteforce(Xp, lab, 4, metric)["S"] - oracle.bruteforce(Xm, lab, 4, metric)["S"]) / (2 * h)
        assert abs(fd - g[i, l]) <= 1e-4 * scale + 1e-7, (i, l, fd, g[i, l])


@pytest.mark.parametrize("metric", METRICS)
def test_autograd_function(metric):
    X, lab = case(44, 1000, 8, 5, metric)
    Xt, lt = to_dev(X, lab)
    Xt.requires_grad_(True)
    S = silhouette_loss(Xt, lt, 5, metric)
    (3.0 * S).backward()
    ref = 3.0 * oracle.linear_grad(X.astype(np.float64), lab, 5, metric)
    assert rel_err(Xt.grad.double().cpu().numpy(), ref) <= 2e-4
    ref_S = oracle.linear(X.astype(np.float64), lab, 5, metric)["S"]
    assert abs(float(S.detach()) - ref_S) <= 1e-6


def test_grad_invariants():
    # translation invariance: rows of dS/dX sum to 0; scale invariance: sum x.g = 0
    X, lab = case(45, 4000, 16, 7, "sqeuclidean", empty=False)
    g = gpu_grad(X, lab, 7, "sqeuclidean")
    scale = np.abs(g).max()
    assert np.abs(g.sum(0)).max() <= 1e-4 * scale * np.sqrt(4000)
    Xc, labc = case(46, 4000, 16, 7, "cosine", empty=False)
    gc = gpu_grad(Xc, labc, 7, "cosine")
    per_row = np.abs((Xc * gc).sum(1)) / (np.linalg.norm(Xc, axis=1) * np.abs(gc).max())
    assert per_row.max() <= 1e-4
