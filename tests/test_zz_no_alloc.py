"""sil_score_noalloc, the entry point for callers that cannot provide device
memory (a host framework owning all device memory through its own pool, or a
plugin whose host forbids allocation on its hot path).

It must give the same result as sil_score on the same inputs, and as the FP64
oracle, and keep doing so on back-to-back calls, although every call reuses
the one scratch array inside the library; once a call has run on a device,
later calls must reserve no device memory.  The size limits are read from
include/sil.h.  This file is collected after every parity file (only the
bounded-wait self-test follows it) so that a run stopping at its first
failure has run the others first.
"""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL_S, TOL_SI, assert_scores, case, dequant, to_dev
from paper_2303_14102_gb300 import sil, synth

pytestmark = pytest.mark.gpu

_HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sil.h")


def header_limit(name):
    m = re.search(r"#define\s+" + name + r"\s+(\d+)", open(_HEADER).read())
    assert m, name
    return int(m.group(1))


MAX_K = header_limit("SIL_NOALLOC_MAX_K")
MAX_D = header_limit("SIL_NOALLOC_MAX_D")


def _both(Xt, lt, K, metric, cs=None):
    agg = sil.aggregate(Xt, lt, K, metric, col_scale=cs)
    ref = sil.score(Xt, lt, K, agg, metric, col_scale=cs, want_s=True, save=True)
    st = sil.new_status(Xt.device)
    got = sil.score_noalloc(Xt, lt, K, agg, metric, col_scale=cs, want_s=True, save=True, status=st)
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


def test_matches_sil_score_and_the_oracle_on_two_calls_in_a_row():
    # first call: 7 clusters, squared Euclidean; second call: fewer clusters,
    # cosine, so stale scratch from the first call would show up
    X1, l1 = case(501, 5000, 24, 7, "sqeuclidean")
    Xt, lt = to_dev(X1, l1)
    ref1, got1 = _both(Xt, lt, 7, "sqeuclidean")
    _same(ref1, got1, 5000)
    assert_scores(got1.s, got1.S, oracle.bruteforce(X1.astype(np.float64), l1, 7, "sqeuclidean"))
    X2, l2 = case(502, 3001, 40, 3, "cosine")
    Xt, lt = to_dev(X2, l2)
    ref2, got2 = _both(Xt, lt, 3, "cosine")
    _same(ref2, got2, 3001)
    assert_scores(got2.s, got2.S, oracle.bruteforce(X2.astype(np.float64), l2, 3, "cosine"))


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_low_precision_storage_at_the_largest_sizes(storage):
    # k and d at the limits of the fixed scratch, low-precision storage; the
    # oracle scores the dequantised values the kernel sees
    N, K, D = 6000, MAX_K, MAX_D
    w = synth.blobs(N, D, 64, seed=504)
    lab = np.random.default_rng(505).integers(0, K, size=N).astype(np.int32)
    lab[: 64 * 40] = np.repeat(np.arange(64), 40)  # some clusters of 40 points among many small ones
    if storage == "bf16":
        Xt, cs = synth.to_bf16(w.X.cuda()), None
    else:
        Xt, cs = synth.to_fp8_e4m3(w.X.cuda())
    lt = torch.as_tensor(lab).cuda()
    ref, got = _both(Xt, lt, K, "sqeuclidean", cs)
    _same(ref, got, N)
    assert_scores(got.s, got.S, oracle.linear(dequant(Xt, cs), lab, K))


def test_second_call_reserves_no_device_memory():
    # every buffer is allocated first; the first call may make the driver
    # reserve the scratch (lazy module loading), the second must not change
    # the device's free memory
    X, lab = case(506, 4000, 32, 9)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 9)
    s_out = torch.empty(4000, dtype=torch.float32, device="cuda")
    S = torch.empty((), dtype=torch.float64, device="cuda")
    st = sil.new_status(Xt.device)
    lib = sil.load()
    vp = ctypes.c_void_p
    stream = vp(torch.cuda.current_stream().cuda_stream)

    def call():
        return lib.sil_score_noalloc(vp(Xt.data_ptr()), 0, 4000, 32, 32, None, vp(lt.data_ptr()), 9, 0,
                                     vp(agg[0].data_ptr()), vp(agg[1].data_ptr()), vp(agg[2].data_ptr()),
                                     vp(s_out.data_ptr()), vp(S.data_ptr()), None, vp(st.data_ptr()), stream)

    assert call() == sil.SIL_OK
    torch.cuda.synchronize()
    S1 = float(S)
    free0 = torch.cuda.mem_get_info()[0]
    assert call() == sil.SIL_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(st.item()) == 0 and float(S) == S1


@pytest.mark.parametrize("k,d", [(MAX_K + 1, 8), (4, MAX_D + 1)])
def test_sizes_beyond_the_scratch_are_refused(k, d):
    X, lab = case(503, 100, d, 4)
    Xt, lt = to_dev(X, lab)
    agg = sil.aggregate(Xt, lt, 4)
    lib = sil.load()
    vp = ctypes.c_void_p
    S = torch.full((), 7.0, dtype=torch.float64, device="cuda")
    rc = lib.sil_score_noalloc(vp(Xt.data_ptr()), 0, 100, d, d, None, vp(lt.data_ptr()), k, 0,
                               vp(agg[0].data_ptr()), vp(agg[1].data_ptr()), vp(agg[2].data_ptr()), None,
                               vp(S.data_ptr()), None, None, None)
    assert rc == sil.SIL_EUNSUPPORTED
    torch.cuda.synchronize()
    assert float(S) == 7.0  # nothing was enqueued
