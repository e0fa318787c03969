"""Parity of the tcgen05 tensor-core pass 2 with the FP64 oracle.

FP32 storage runs the in-kernel BF16 hi/lo split (three MMAs per k-step),
BF16 storage runs two; both must meet the FP32 tolerances of the SIMT path.
Sizes cover one and two 64-wide K atoms, padded D, K from 2 to 256 (MMA N up
to 256, both TMEM accumulators), ragged last tiles and multi-tile CTAs.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, assert_scores, case, dequant, to_dev
from paper_2303_14102_gb300 import sil, synth

pytestmark = pytest.mark.gpu
METRICS = ["sqeuclidean", "cosine"]


def run(Xt, lt, K, metric, path, save=True):
    st = sil.new_status(Xt.device)
    agg = sil.aggregate(Xt, lt, K, metric, status=st)
    r = sil.score(Xt, lt, K, agg, metric, want_s=True, save=save, path=path, status=st)
    torch.cuda.synchronize()
    return r, int(st.item())


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("N,D,K", [(1000, 64, 2), (4097, 64, 7), (20000, 64, 100), (3001, 128, 17),
                                   (5000, 100, 33), (2000, 40, 5), (300, 64, 256), (129, 64, 3),
                                   (700, 128, 128)])
def test_tensor_path_against_bruteforce(metric, dtype, N, D, K):
    if dtype == torch.bfloat16 and (D < 64 or (2 * D) % 16):
        pytest.skip("BF16 tensor path needs d >= 64 and 16-byte rows (TMA)")
    X, lab = case(700 + N + D + K, N, D, K, metric)
    Xt, lt = to_dev(X, lab, dtype)
    r, st = run(Xt, lt, K, metric, "tensor")
    ref = oracle.bruteforce(dequant(Xt), lab, K, metric)
    if ref["status"] == oracle.EDEGENERATE:
        assert st & sil.SIL_EDEGENERATE
        return
    assert st == 0
    assert_scores(r.s, r.S, ref, what=f"tensor {metric} {dtype} N={N} D={D} K={K}")
    a, b, ks = sil.unpack_saved(r.saved, N)
    ok = ref["s"] != 0
    np.testing.assert_allclose(a.cpu().double().numpy()[ok], ref["a"][ok], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(b.cpu().double().numpy()[ok], ref["b"][ok], rtol=1e-4, atol=1e-4)
    assert np.mean(ks.cpu().numpy()[ok] == ref["kstar"][ok]) > 0.995


@pytest.mark.parametrize("metric", METRICS)
def test_tensor_and_simt_agree_at_scale_recipe(metric):
    w = synth.workload_at_scale(device="cuda", N=300_000)
    ra, sa_ = run(w.X, w.labels, w.K, metric, "tensor", save=False)
    rb, sb_ = run(w.X, w.labels, w.K, metric, "simt", save=False)
    assert sa_ == 0 and sb_ == 0
    assert float((ra.s - rb.s).abs().max()) <= TOL_SI
    assert abs(float(ra.S) - float(rb.S)) <= TOL_S


def test_tensor_path_far_from_origin():
    # centres at radius 1e3: the GEMM term is ~1e6 and cancels in d_k
    w = synth.blobs(20000, 128, 40, seed=9, sphere_radius=1e3)
    Xt, lt = w.X.cuda(), w.labels.cuda()
    r, st = run(Xt, lt, 40, "sqeuclidean", "tensor")
    assert st == 0
    ref = oracle.linear(w.X.double().numpy(), w.labels.numpy(), 40)
    assert_scores(r.s, r.S, ref)


def test_auto_picks_tensor_when_eligible():
    X, lab = case(5, 3000, 64, 10)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 10)
    ra = sil.score(Xt, lt, 10, agg, want_s=True, path="auto")
    rt = sil.score(Xt, lt, 10, agg, want_s=True, path="tensor")
    assert torch.equal(ra.s, rt.s)  # same aggregates, same kernel: bit-identical


def test_tensor_refuses_shapes_beyond_shared_memory():
    # FP32, d = 128, k = 256: split centroids + one A buffer + one raw stage > 227 KB
    X, lab = case(7, 300, 128, 256)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 256)
    with pytest.raises(sil.SilError):
        sil.score(Xt, lt, 256, agg, path="tensor")
    r = sil.score(Xt, lt, 256, agg, want_s=True, path="auto")  # falls back to SIMT
    torch.cuda.synchronize()
    assert np.isfinite(float(r.S))


def test_tensor_refuses_ineligible_shapes():
    X, lab = case(6, 500, 8, 3)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 3)
    with pytest.raises(sil.SilError):
        sil.score(Xt, lt, 3, agg, path="tensor")
