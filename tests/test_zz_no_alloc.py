"""sil_score_noalloc, the entry point for callers that cannot provide device
memory (a host framework owning all device memory through its own pool, or a
plugin whose host forbids allocation on its hot path).

It must give the same result as sil_score on the same inputs, and keep doing
so on back-to-back calls, although every call reuses the one scratch array
inside the library.  This file is collected after every parity file (only
the bounded-wait self-test follows it) so that a run stopping at its first
failure has run the others first.
"""
import ctypes

import numpy as np
import pytest
import torch

from helpers import TOL_S, TOL_SI, case, to_dev
from paper_2303_14102_gb300 import sil

pytestmark = pytest.mark.gpu


def _both(X, lab, K, metric):
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, K, metric)
    ref = sil.score(Xt, lt, K, agg, metric, want_s=True, save=True)
    st = sil.new_status(Xt.device)
    got = sil.score_noalloc(Xt, lt, K, agg, metric, want_s=True, save=True, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ref, got


def _same(ref, got, N):
    assert abs(float(got.S) - float(ref.S)) <= TOL_S
    assert float((got.s - ref.s).abs().max()) <= TOL_SI
    a0, b0, k0 = sil.unpack_saved(ref.saved, N)
    a1, b1, k1 = sil.unpack_saved(got.saved, N)
    torch.testing.assert_close(a1, a0, rtol=1e-5, atol=1e-5)
    torch.testing.assert_close(b1, b0, rtol=1e-5, atol=1e-5)
    assert torch.equal(k1, k0)


def test_matches_sil_score_on_two_calls_in_a_row():
    # first call: 7 clusters, squared Euclidean; second call: fewer clusters,
    # cosine, so stale scratch from the first call would show up
    X1, l1 = case(501, 5000, 24, 7, "sqeuclidean")
    ref1, got1 = _both(X1, l1, 7, "sqeuclidean")
    _same(ref1, got1, 5000)
    X2, l2 = case(502, 3001, 40, 3, "cosine")
    ref2, got2 = _both(X2, l2, 3, "cosine")
    _same(ref2, got2, 3001)


def test_sizes_beyond_the_scratch_are_refused():
    X, lab = case(503, 100, 8, 4)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 4)
    lib = sil.load()
    vp = ctypes.c_void_p
    S = torch.empty((), dtype=torch.float64, device="cuda")
    rc = lib.sil_score_noalloc(vp(Xt.data_ptr()), 0, 100, 8, 8, None, vp(lt.data_ptr()),
                               sil_max_k() + 1, 0, vp(agg[0].data_ptr()), vp(agg[1].data_ptr()),
                               vp(agg[2].data_ptr()), None, vp(S.data_ptr()), None, None, None)
    assert rc == sil.SIL_EUNSUPPORTED


def sil_max_k():
    return 1024
