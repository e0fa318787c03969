"""The C-ABI library builds, loads and exports what include/sil.h declares;
host-side argument checks answer without touching a GPU (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2303_14102_gb300 import _build, sil

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "sil.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sil_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return sil.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sil_aggregate", "sil_score", "sil_score_backward", "sil_workspace_size"):
        assert required in names
    assert set(names) >= set(sil.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (sil_[a-z_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_no_torch_or_cxx_types_in_the_abi():
    code = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    assert "torch" not in code.lower() and "at::" not in code
    assert "std::" not in code and "class " not in code and "template" not in code


def test_version_and_strings(lib):
    assert lib.sil_version() >= 100
    assert b"SIL_ELABEL" in lib.sil_status_string(sil.SIL_ELABEL)
    assert b"unknown" in lib.sil_status_string(12345)


def test_workspace_and_saved_sizes(lib):
    a = lib.sil_workspace_size(1000, 8, 5, 0, 0, 1)
    b = lib.sil_workspace_size(100000, 8, 5, 0, 0, 1)
    assert 0 < a < b and a % 256 == 0
    assert lib.sil_workspace_size(10, 0, 5, 0, 0, 1) == 0
    assert lib.sil_saved_size(1000) == 12000


def _agg(lib, **kw):
    args = dict(X=ctypes.c_void_p(16), dtype=0, n=10, d=4, ldx=4, cs=None, labels=ctypes.c_void_p(16),
                k=3, dist=0, count=ctypes.c_void_p(16), s1=ctypes.c_void_p(16), s2=ctypes.c_void_p(16),
                flags=0, ws=ctypes.c_void_p(256), ws_bytes=1 << 30, status=None, stream=None)
    args.update(kw)
    return lib.sil_aggregate(*args.values())


def test_argument_errors_are_reported_before_any_launch(lib):
    # every case below fails validation, so no CUDA call is made (no GPU here)
    assert _agg(lib, d=0) == sil.SIL_EINVAL
    assert _agg(lib, k=0) == sil.SIL_EINVAL
    assert _agg(lib, ldx=3) == sil.SIL_EINVAL
    assert _agg(lib, dtype=7) == sil.SIL_EINVAL
    assert _agg(lib, dist=5) == sil.SIL_EINVAL
    assert _agg(lib, X=None) == sil.SIL_EINVAL
    assert _agg(lib, dtype=2, cs=None) == sil.SIL_EINVAL  # FP8 needs column scales
    assert _agg(lib, count=None) == sil.SIL_EINVAL
    assert _agg(lib, ws=None) == sil.SIL_EWORKSPACE
    assert _agg(lib, ws=ctypes.c_void_p(256 + 8)) == sil.SIL_EWORKSPACE
    assert _agg(lib, ws_bytes=100) == sil.SIL_EWORKSPACE
    assert _agg(lib, k=1 << 23) == sil.SIL_EUNSUPPORTED


def test_score_path_validation(lib):
    vp = ctypes.c_void_p
    rc = lib.sil_score(vp(16), 0, 10, 4, 4, None, vp(16), 3, 0, vp(16), vp(16), vp(16), None, vp(16),
                       None, 9, vp(256), 1 << 30, None, None)
    assert rc == sil.SIL_EINVAL
    rc = lib.sil_score_backward(vp(16), 0, 10, 4, 4, None, vp(16), 3, 0, vp(16), vp(16), vp(16), None,
                                None, vp(16), 2, vp(256), 1 << 30, None, None)
    assert rc == sil.SIL_EINVAL  # lddx < d
    ks = (ctypes.c_int32 * 2)(3, 0)
    rc = lib.sil_score_batched(vp(16), 0, 10, 4, 4, None, vp(16), 10, ks, 2, 0, vp(16), vp(256),
                               1 << 30, None, None)
    assert rc == sil.SIL_EINVAL  # a labeling with k = 0


def test_fused_call_validation(lib):
    vp = ctypes.c_void_p

    def call(count=vp(16), path=0, ws=vp(256), d=4, k=3):
        return lib.sil_silhouette(vp(16), 0, 10, d, 4, None, vp(16), k, 0, count, vp(16), vp(16), None, vp(16),
                                  None, path, ws, 1 << 30, None, None)
    assert call(count=None) == sil.SIL_EINVAL     # aggregates are outputs here
    assert call(path=9) == sil.SIL_EINVAL
    assert call(d=0) == sil.SIL_EINVAL
    assert call(k=0) == sil.SIL_EINVAL
    assert call(ws=vp(257)) == sil.SIL_EWORKSPACE  # misaligned workspace


def test_binding_refuses_cpu_tensors():
    import torch
    X = torch.zeros(4, 2)
    with pytest.raises(RuntimeError, match="CUDA"):
        sil.aggregate(X, torch.zeros(4, dtype=torch.int32), 2)


def test_euclidean_rms_is_a_distance_code_without_a_backward_pass(lib):
    assert _agg(lib, dist=3) == sil.SIL_EINVAL
    vp = ctypes.c_void_p
    rc = lib.sil_score_backward(vp(16), 0, 10, 4, 4, None, vp(16), 3, sil.METRICS["euclidean_rms"], vp(16),
                                vp(16), vp(16), None, None, vp(16), 4, vp(256), 1 << 30, None, None)
    assert rc == sil.SIL_EUNSUPPORTED


def test_autograd_refuses_the_rms_approximation():
    import torch
    from paper_2303_14102_gb300.autograd import silhouette_loss
    with pytest.raises(ValueError, match="no gradient"):
        silhouette_loss(torch.zeros(4, 2), torch.zeros(4, dtype=torch.int32), 2, "euclidean_rms")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no fallback: without libsil.so the binding raises instead of computing elsewhere
    monkeypatch.setattr(sil, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libsil.so"))
    with pytest.raises(RuntimeError, match="libsil.so not found"):
        sil.load(build_if_stale=False)


def test_tensor_plan_is_host_arithmetic():
    import torch
    # one block covers k <= 256 when it fits; k = 1000 in BF16 at d = 128 takes
    # four blocks of 256 (two A buffers beside the resident split centroids)
    assert sil.tensor_plan(torch.float32, 64, 100) == (112, 1)
    assert sil.tensor_plan(torch.bfloat16, 128, 1000) == (256, 4)
    # the precision recipe's other storage types: the fastest of the
    # best-modelled candidates when timed on a GB300 (FP8 blocks of 256,
    # FP32 seven blocks of 144 with one A buffer)
    assert sil.tensor_plan_candidates(torch.float8_e4m3fn, 128, 1000, 1)[0] == (256, 2, 1, 0, 0)
    assert sil.tensor_plan_candidates(torch.float32, 128, 1000, 1)[0] == (144, 1, 1, 0, 0)
    assert sil.tensor_plan_candidates(torch.bfloat16, 128, 1000, 1)[0] == (256, 2, 1, 0, 0)
    for dt, d, k in [(torch.float32, 128, 256), (torch.float8_e4m3fn, 128, 1000),
                     (torch.float32, 32, 513), (torch.bfloat16, 64, 4096)]:
        bk, nb = sil.tensor_plan(dt, d, k)
        assert bk % 16 == 0 and 16 <= bk <= 256
        assert (nb - 1) * bk < k <= nb * bk
    # FP32 rows up to 256 columns run in 64-column chunks; wider rows and
    # wide BF16 rows take the SIMT kernels
    assert sil.tensor_plan(torch.float32, 256, 100) is not None
    assert sil.tensor_plan(torch.float32, 257, 100) is None
    assert sil.tensor_plan(torch.bfloat16, 256, 100) is None


def test_tensor_plan_rejects_bad_arguments(lib):
    out = ctypes.c_int32(0)
    assert lib.sil_tensor_plan(0, 64, 100, None, ctypes.byref(out)) == sil.SIL_EINVAL
    assert lib.sil_tensor_plan(7, 64, 100, ctypes.byref(out), ctypes.byref(out)) == sil.SIL_EINVAL
    assert lib.sil_tensor_plan(0, 64, 0, ctypes.byref(out), ctypes.byref(out)) == sil.SIL_EINVAL


def test_tensor_plan_candidates_and_override():
    import torch
    cands = sil.tensor_plan_candidates(torch.float32, 64, 100, 8)
    assert 1 <= len(cands) <= 8
    assert cands[0][0] == sil.tensor_plan(torch.float32, 64, 100)[0]  # best modelled first
    for bk, nab, nxs, stz, rank in cands:
        assert bk % 16 == 0 and 1 <= nab <= 4 and 1 <= nxs <= 3 and stz in (0, 1) and rank in (0, 1)
    assert cands[0][4] == 0  # the model prefers the plain minimum pass
    try:
        sil.tensor_plan_set(torch.float32, 64, 100, (48, 2, 2, 0, 1))
        assert sil.tensor_plan(torch.float32, 64, 100) == (48, 3)
        assert sil.tensor_plan(torch.float32, 64, 101) == (112, 1)  # other shapes untouched
    finally:
        sil.tensor_plan_set(torch.float32, 64, 100, None)
    assert sil.tensor_plan(torch.float32, 64, 100) == (112, 1)


def test_tensor_plan_set_rejects_bad_plans(lib):
    assert lib.sil_tensor_plan_set(0, 64, 100, 40, 2, 2, 0, 0) == sil.SIL_EINVAL      # not a multiple of 16
    assert lib.sil_tensor_plan_set(0, 64, 100, 256, 4, 2, 1, 0) == sil.SIL_EUNSUPPORTED  # too much shared memory
    # two converter groups alternate tiles: odd rings would hand one slot to both
    assert lib.sil_tensor_plan_set(0, 64, 100, 112, 3, 2, 1, 0) == sil.SIL_EINVAL
    assert lib.sil_tensor_plan_set(0, 64, 100, 112, 2, 1, 1, 0) == sil.SIL_EINVAL
    assert lib.sil_tensor_plan_set(0, 128, 100, 64, 1, 1, 0, 0) == sil.SIL_OK     # one group: any depth
    assert lib.sil_tensor_plan_set(0, 128, 100, 0, 0, 0, 0, 0) == sil.SIL_OK      # back to the model
    assert lib.sil_tensor_plan_set(0, 300, 100, 64, 2, 2, 0, 0) == sil.SIL_EINVAL     # d > 256
    assert lib.sil_tensor_plan_set(0, 64, 100, 64, 2, 2, 0, 2) == sil.SIL_EINVAL      # rank pass is 0 or 1


@pytest.mark.parametrize("dtype_name", ["float32", "bfloat16", "float8_e4m3fn"])
def test_every_candidate_plan_is_one_the_library_accepts(dtype_name):
    # the enumerator and the validator must agree on every shape: a plan the
    # cost model ranks but the kernels cannot run safely (an odd ring shared by
    # two converter groups) must never be offered
    import torch
    dt = getattr(torch, dtype_name)
    ds = [1, 8, 31, 32, 33, 63, 64, 65, 100, 128] + ([129, 200, 256] if dt == torch.float32 else [])
    for d in ds:
        for k in (1, 2, 15, 16, 17, 100, 255, 256, 257, 1000, 4096):
            cands = sil.tensor_plan_candidates(dt, d, k, 64)
            assert cands, (dtype_name, d, k)
            assert sil.tensor_plan(dt, d, k)[0] == cands[0][0]
            try:
                for plan in cands:
                    bk, nab, nxs, stz, rank = plan
                    assert bk % 16 == 0 and 16 <= bk <= 256 and nab >= 1 and nxs >= 1
                    assert stz in (0, 1) and rank in (0, 1)
                    sil.tensor_plan_set(dt, d, k, plan)  # raises SilError if refused
                    bk2, nb = sil.tensor_plan(dt, d, k)
                    assert bk2 == bk and (nb - 1) * bk < k <= nb * bk, (dtype_name, d, k, plan)
            finally:
                sil.tensor_plan_set(dt, d, k, None)


def test_selftest_refuses_a_null_status_array(lib):
    assert lib.sil_selftest_bounded_wait(None, None) == sil.SIL_EINVAL


def test_tensor_kernel_query(lib):
    import torch
    assert sil.tensor_kernels(torch.float32, 64, 100) == {"split", "tf32"}  # the at-scale shape
    assert sil.tensor_kernels(torch.float32, 32, 512) == {"split", "tf32"}  # two cluster blocks
    assert sil.tensor_kernels(torch.float32, 40, 7) == {"split", "tf32"}    # padded columns
    assert sil.tensor_kernels(torch.float32, 128, 100) == {"split"}
    assert sil.tensor_kernels(torch.float32, 256, 1000) == {"split"}        # 64-column chunks
    assert sil.tensor_kernels(torch.bfloat16, 64, 100) == {"split"}
    assert sil.tensor_kernels(torch.float8_e4m3fn, 128, 1000) == {"split"}
    assert sil.tensor_kernels(torch.float8_e4m3fn, 64, 10) == set()
    assert sil.tensor_kernels(torch.float32, 16, 100) == set()
    assert sil.tensor_kernels(torch.float32, 257, 100) == set()
    assert lib.sil_tensor_kernel(7, 64, 100) == 0 and lib.sil_tensor_kernel(0, 64, 0) == 0


def test_exact_euclidean_argument_checks(lib):
    vp = ctypes.c_void_p
    fake = vp(256)  # never dereferenced: each call below is refused on the host
    assert lib.sil_euclidean_workspace_size(1000, 64, 10) > lib.sil_euclidean_workspace_size(100, 64, 10) > 0
    assert lib.sil_euclidean_workspace_size(1000, 0, 10) == 0
    assert lib.sil_score_euclidean(fake, 0, 100, 129, 129, None, fake, 3, None, fake, None, fake, 1 << 30,
                                   None, None) == sil.SIL_EUNSUPPORTED
    assert lib.sil_score_euclidean(fake, 0, 100, 8, 8, None, fake, 3, None, None, None, fake, 1 << 30,
                                   None, None) == sil.SIL_EINVAL
    assert lib.sil_score_euclidean(fake, 0, 100, 8, 8, None, fake, 3, None, fake, None, None, 0,
                                   None, None) == sil.SIL_EWORKSPACE


def test_batched_plan_set_checks(lib):
    try:
        assert lib.sil_batched_plan_set(0, 0) == sil.SIL_EINVAL
        assert lib.sil_batched_plan_set(65, 0) == sil.SIL_EINVAL
        assert lib.sil_batched_plan_set(8, 3) == sil.SIL_EINVAL
        assert lib.sil_batched_plan_set(16, 2) == sil.SIL_OK
    finally:
        assert lib.sil_batched_plan_set(8, 0) == sil.SIL_OK
