"""The exact (non-squared) Euclidean Silhouette by the quadratic method
(sil_score_euclidean), element by element against the oracle's brute force
with the plain Euclidean distance (Eq. 1-3, Sec. II).

Sizes span several 128-row CTAs and 64-point column tiles with ragged tails,
every register width of the kernel (d <= 16, 32, 64, 128), clusters whose run
of columns crosses tiles, empty label ids and singleton clusters, the three
storage types, and the error cases."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, assert_scores, case, dequant, to_dev
from paper_2303_14102_gb300 import sil, synth

pytestmark = pytest.mark.gpu


def run(Xt, lt, K, cs=None):
    st = sil.new_status(Xt.device)
    r = sil.score_euclidean(Xt, lt, K, col_scale=cs, want_s=True, save=True, status=st)
    torch.cuda.synchronize()
    return r, int(st.item())


def check(r, ref, N, what):
    assert_scores(r.s, r.S, ref, what=what)
    a, b, ks = sil.unpack_saved(r.saved, N)
    ok = np.isfinite(ref["b"])
    np.testing.assert_allclose(a.cpu().double().numpy(), ref["a"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(b.cpu().double().numpy()[ok], ref["b"][ok], rtol=1e-5)
    assert np.mean(ks.cpu().numpy()[ok] == ref["kstar"][ok]) > 0.995


@pytest.mark.parametrize("N,D,K", [(1, 3, 2), (129, 5, 4), (1000, 17, 7), (4097, 33, 6), (3001, 64, 9),
                                   (2500, 100, 5), (2000, 128, 40), (3000, 12, 64), (700, 1, 3)])
def test_ragged_shapes_against_bruteforce(N, D, K):
    X, lab = case(4000 + N + D + K, N, D, K)
    Xt, lt = to_dev(X, lab)
    r, st = run(Xt, lt, K)
    ref = oracle.bruteforce(X.astype(np.float64), lab, K, "euclidean")
    if ref["status"] == oracle.EDEGENERATE:
        assert st & sil.SIL_EDEGENERATE and np.isnan(float(r.S))
        return
    assert st == 0
    check(r, ref, N, f"N={N} D={D} K={K}")


def test_small_workload():
    w = synth.workload_small()  # N = 10,000, D = 8, K = 5
    r, st = run(w.X.cuda(), w.labels.cuda(), w.K)
    assert st == 0
    check(r, oracle.bruteforce(w.X.double().numpy(), w.labels.numpy(), w.K, "euclidean"), w.X.shape[0], "small")


def test_at_scale_recipe_at_20000_points():
    # the headline recipe (D = 64, K = 100, Zipf sizes: clusters from ~30 to
    # ~4,700 points, i.e. runs of columns over many tiles) at the largest
    # size the oracle's brute force finishes in seconds
    w = synth.workload_at_scale(N=20_000)
    r, st = run(w.X.cuda(), w.labels.cuda(), w.K)
    assert st == 0
    check(r, oracle.bruteforce(w.X.double().numpy(), w.labels.numpy(), w.K, "euclidean"), 20_000, "at_scale")


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_low_precision_storage(storage):
    X, lab = case(4100, 3000, 64, 11)
    if storage == "bf16":
        Xt, cs = torch.as_tensor(X).cuda().to(torch.bfloat16), None
    else:
        Xt, cs = synth.to_fp8_e4m3(torch.as_tensor(X).cuda())
    lt = torch.as_tensor(lab).cuda()
    r, st = run(Xt, lt, 11, cs)
    assert st == 0
    check(r, oracle.bruteforce(dequant(Xt, cs), lab, 11, "euclidean"), 3000, storage)


def test_two_calls_in_a_row_reuse_the_workspace():
    X1, l1 = case(4200, 5000, 24, 30)
    X2, l2 = case(4201, 3000, 24, 4)
    for X, lab, K in ((X1, l1, 30), (X2, l2, 4)):
        Xt, lt = to_dev(X, lab)
        r, st = run(Xt, lt, K)
        assert st == 0
        check(r, oracle.bruteforce(X.astype(np.float64), lab, K, "euclidean"), X.shape[0], f"K={K}")


def test_errors():
    X, lab = case(4300, 500, 8, 3)
    Xt, lt = to_dev(X, lab)
    # one cluster: b undefined
    r, st = run(Xt, torch.zeros_like(lt), 3)
    assert st & sil.SIL_EDEGENERATE and np.isnan(float(r.S))
    # a label outside [0, k)
    bad = lt.clone()
    bad[7] = 3
    r, st = run(Xt, bad, 3)
    assert st & sil.SIL_ELABEL and np.isnan(float(r.S))
    # rows wider than the register tile
    Xw, lw = to_dev(*case(4301, 100, 129, 3))
    with pytest.raises(sil.SilError):
        sil.score_euclidean(Xw, lw, 3)


def test_squared_form_differs_and_rms_bounds_it():
    # the exact Euclidean score is neither the squared-Euclidean one nor the
    # root-mean-square approximation, which bounds its a_i and b_i from above
    # (Jensen); checked on the GPU results themselves
    X, lab = case(4400, 4000, 16, 8)
    Xt, lt = to_dev(X, lab)
    r, st = run(Xt, lt, 8)
    assert st == 0
    rr = sil.score(Xt, lt, 8, sil.aggregate(Xt, lt, 8, "euclidean_rms"), "euclidean_rms", want_s=True, save=True)
    a, b, _ = sil.unpack_saved(r.saved, 4000)
    a2, b2, _ = sil.unpack_saved(rr.saved, 4000)  # squared means
    assert torch.all(a <= torch.sqrt(a2) * (1 + 1e-5) + 1e-6)
    assert torch.all(b <= torch.sqrt(b2) * (1 + 1e-5) + 1e-6)
