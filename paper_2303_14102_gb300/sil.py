"""Thin ctypes binding of libsil (C ABI in include/sil.h).

Argument marshalling only: every step of the Silhouette runs in the CUDA
kernels of libsil.so.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: without the compiled library or a CUDA
device every call raises.

Entry points mirror the C names:
  aggregate(X, labels, K, ...)          -> (count, s1, s2)     sil_aggregate
  score(X, labels, K, agg, ...)         -> Score(S, s, saved)  sil_score
  score_backward(X, labels, K, agg, ...)-> dX                  sil_score_backward
  score_batched(X, labels, ks, ...)     -> S[B]                sil_score_batched
  score_euclidean(X, labels, K, ...)    -> Score(S, s, saved)  sil_score_euclidean (exact, O(N^2))
  silhouette(X, labels, K, ...)         -> Score(S, s, saved)  sil_silhouette (both passes, one call)
  silhouette_chunked(X_host, labels_host, K, ...)
                                        -> S of host-resident data streamed in row chunks
Results stay on the device and nothing synchronises; ``check_status`` reads
the device status word (one sync) and raises on a data error.

Every call runs on the current stream of the tensors' device and, except
``score_noalloc``, uses one grow-only workspace per device: issue calls that
may overlap on ONE stream (or order their streams with events), as with a
library handle's workspace.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

from . import _build

SIL_OK, SIL_EINVAL, SIL_ELABEL, SIL_EDEGENERATE, SIL_EZERONORM = 0, 1, 2, 4, 8
SIL_ECUDA, SIL_ETIMEOUT, SIL_EWORKSPACE, SIL_EUNSUPPORTED = 16, 32, 64, 128
SIL_AGG_ACCUMULATE = 1
# "euclidean_rms": the square root of each point-to-cluster mean squared
# Euclidean distance in Eq. 2 (the approximation of the Limitations section)
METRICS = {"sqeuclidean": 0, "cosine": 1, "euclidean_rms": 2}
PATHS = {"auto": 0, "simt": 1, "tensor": 2, "tensor_tf32": 3}
EXPORTED = ("sil_workspace_size", "sil_saved_size", "sil_aggregate", "sil_score",
            "sil_score_backward", "sil_score_batched", "sil_tensor_plan", "sil_tensor_plan_candidates",
            "sil_tensor_plan_set", "sil_tensor_kernel", "sil_batched_plan_set", "sil_chunk_mean", "sil_score_noalloc", "sil_score_euclidean",
            "sil_euclidean_workspace_size", "sil_silhouette", "sil_selftest_bounded_wait", "sil_status_string",
            "sil_version")

_lock = threading.Lock()
_lib = None


class SilError(RuntimeError):
    """A non-zero return code or device status flag of libsil."""

    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


def load(build_if_stale: bool = True) -> ctypes.CDLL:
    """Load libsil.so (compiling it first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_stale:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libsil.so not found at {_build.LIB}; run __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            vp, i32, i64, sz, u32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t,
                                     ctypes.c_uint32)
            lib.sil_workspace_size.argtypes = [i64, i32, i32, i32, i32, i32]
            lib.sil_workspace_size.restype = sz
            lib.sil_saved_size.argtypes = [i64]
            lib.sil_saved_size.restype = sz
            lib.sil_aggregate.argtypes = [vp, i32, i64, i32, i64, vp, vp, i32, i32, vp, vp, vp, u32,
                                          vp, sz, vp, vp]
            lib.sil_aggregate.restype = ctypes.c_int
            lib.sil_score.argtypes = [vp, i32, i64, i32, i64, vp, vp, i32, i32, vp, vp, vp, vp, vp,
                                      vp, i32, vp, sz, vp, vp]
            lib.sil_score.restype = ctypes.c_int
            lib.sil_silhouette.argtypes = [vp, i32, i64, i32, i64, vp, vp, i32, i32, vp, vp, vp, vp, vp,
                                           vp, i32, vp, sz, vp, vp]
            lib.sil_silhouette.restype = ctypes.c_int
            lib.sil_score_backward.argtypes = [vp, i32, i64, i32, i64, vp, vp, i32, i32, vp, vp, vp,
                                               vp, vp, vp, i64, vp, sz, vp, vp]
            lib.sil_score_backward.restype = ctypes.c_int
            lib.sil_score_batched.argtypes = [vp, i32, i64, i32, i64, vp, vp, i64, vp, i32, i32, vp,
                                              vp, sz, vp, vp]
            lib.sil_score_batched.restype = ctypes.c_int
            lib.sil_score_noalloc.argtypes = [vp, i32, i64, i32, i64, vp, vp, i32, i32, vp, vp, vp,
                                              vp, vp, vp, vp, vp]
            lib.sil_score_noalloc.restype = ctypes.c_int
            lib.sil_tensor_plan.argtypes = [i32, i32, i32, vp, vp]
            lib.sil_tensor_plan.restype = ctypes.c_int
            lib.sil_tensor_plan_candidates.argtypes = [i32, i32, i32, vp, i32, vp]
            lib.sil_tensor_plan_candidates.restype = ctypes.c_int
            lib.sil_tensor_plan_set.argtypes = [i32, i32, i32, i32, i32, i32, i32, i32]
            lib.sil_tensor_plan_set.restype = ctypes.c_int
            lib.sil_score_euclidean.argtypes = [vp, i32, i64, i32, i64, vp, vp, i32, vp, vp, vp, vp, sz, vp, vp]
            lib.sil_score_euclidean.restype = ctypes.c_int
            lib.sil_euclidean_workspace_size.argtypes = [i64, i32, i32]
            lib.sil_euclidean_workspace_size.restype = sz
            lib.sil_chunk_mean.argtypes = [vp, vp, i32, vp, vp]
            lib.sil_chunk_mean.restype = ctypes.c_int
            lib.sil_batched_plan_set.argtypes = [i32, i32]
            lib.sil_batched_plan_set.restype = ctypes.c_int
            lib.sil_tensor_kernel.argtypes = [i32, i32, i32]
            lib.sil_tensor_kernel.restype = ctypes.c_int
            lib.sil_selftest_bounded_wait.argtypes = [vp, vp]
            lib.sil_selftest_bounded_wait.restype = ctypes.c_int
            lib.sil_status_string.argtypes = [i32]
            lib.sil_status_string.restype = ctypes.c_char_p
            lib.sil_version.restype = i32
            _lib = lib
    return _lib


def status_string(code: int) -> str:
    try:
        return load(build_if_stale=False).sil_status_string(int(code)).decode()
    except Exception:  # pragma: no cover - library not loadable
        return "unknown"


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return 0
    if t.dtype == torch.bfloat16:
        return 1
    if t.dtype == torch.float8_e4m3fn:
        return 2
    raise TypeError(f"unsupported storage dtype {t.dtype}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_X(X: torch.Tensor, labels: torch.Tensor):
    if not X.is_cuda:
        raise RuntimeError("libsil runs on CUDA tensors only (no CPU path)")
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D tensor with unit column stride")
    if labels.dtype != torch.int32 or not labels.is_cuda or labels.stride(-1) != 1:
        raise ValueError("labels must be a contiguous CUDA int32 tensor")


def _rc(rc: int, what: str):
    if rc != SIL_OK:
        raise SilError(rc, what)


class _Workspace:
    """Grow-only device workspace per device (one per process).  A grown
    buffer replaces the old one through torch's caching allocator, which
    reuses the old memory only in the order of the stream it was taken on."""

    def __init__(self):
        self._buf = {}
        self._lock = threading.Lock()

    def get(self, device, nbytes: int) -> torch.Tensor:
        key = torch.device(device).index
        with self._lock:
            buf = self._buf.get(key)
            if buf is None or buf.numel() < nbytes:
                buf = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=device)
                self._buf[key] = buf
            return buf


_WS = _Workspace()


def workspace_size(N: int, D: int, K: int, dtype=torch.float32, metric="sqeuclidean",
                   batch: int = 1) -> int:
    code = {torch.float32: 0, torch.bfloat16: 1, torch.float8_e4m3fn: 2}[dtype]
    return int(load().sil_workspace_size(N, D, K, code, METRICS[metric], batch))


def new_status(device) -> torch.Tensor:
    """A zeroed device status word (int32 storage of the uint32 flags)."""
    return torch.zeros(1, dtype=torch.int32, device=device)


def check_status(status: torch.Tensor, what: str = "libsil"):
    """Synchronise on the status word and raise SilError if a flag is set."""
    v = int(status.item()) & 0xFFFFFFFF
    if v:
        raise SilError(v, what)


def _ws_for(X, K, metric, batch=1):
    N, D = X.shape
    need = int(load().sil_workspace_size(N, D, K, _dtype_code(X), METRICS[metric], batch))
    return _WS.get(X.device, need), need


def aggregate(X: torch.Tensor, labels: torch.Tensor, K: int, metric: str = "sqeuclidean",
              col_scale: torch.Tensor | None = None, out=None, accumulate: bool = False,
              status: torch.Tensor | None = None):
    """Pass 1: (count int64[K], s1 f64[K, D], s2 f64[K]) on the device."""
    _check_X(X, labels)
    lib = load()
    N, D = X.shape
    if out is None:
        count = torch.zeros(K, dtype=torch.int64, device=X.device)
        s1 = torch.zeros(K, D, dtype=torch.float64, device=X.device)
        s2 = torch.zeros(K, dtype=torch.float64, device=X.device)
    else:
        count, s1, s2 = out
    ws, need = _ws_for(X, K, metric)
    rc = lib.sil_aggregate(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale), _ptr(labels),
                           K, METRICS[metric], _ptr(count), _ptr(s1), _ptr(s2),
                           SIL_AGG_ACCUMULATE if accumulate else 0, _ptr(ws), need, _ptr(status),
                           _stream_handle(X.device))
    _rc(rc, "sil_aggregate")
    return count, s1, s2


@dataclasses.dataclass
class Score:
    S: torch.Tensor                  # 0-d float64 on the device
    s: torch.Tensor | None           # float32[N] or None
    saved: torch.Tensor | None       # uint8[12 N] record for the backward pass


def score(X: torch.Tensor, labels: torch.Tensor, K: int, agg, metric: str = "sqeuclidean",
          col_scale: torch.Tensor | None = None, want_s: bool = False, save: bool = False,
          path: str = "auto", status: torch.Tensor | None = None) -> Score:
    """Pass 2 from the aggregates of :func:`aggregate` over the same rows."""
    _check_X(X, labels)
    lib = load()
    N, D = X.shape
    count, s1, s2 = agg
    S = torch.empty((), dtype=torch.float64, device=X.device)
    s = torch.empty(N, dtype=torch.float32, device=X.device) if want_s else None
    saved = torch.empty(int(lib.sil_saved_size(N)), dtype=torch.uint8, device=X.device) if save else None
    ws, need = _ws_for(X, K, metric)
    rc = lib.sil_score(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale), _ptr(labels), K,
                       METRICS[metric], _ptr(count), _ptr(s1), _ptr(s2), _ptr(s), _ptr(S),
                       _ptr(saved), PATHS[path], _ptr(ws), need, _ptr(status),
                       _stream_handle(X.device))
    _rc(rc, "sil_score")
    return Score(S=S, s=s, saved=saved)


def score_noalloc(X: torch.Tensor, labels: torch.Tensor, K: int, agg, metric: str = "sqeuclidean",
                  col_scale: torch.Tensor | None = None, want_s: bool = False, save: bool = False,
                  status: torch.Tensor | None = None) -> Score:
    """sil_score_noalloc: pass 2 using the library's own fixed scratch array.

    For callers that cannot provide a workspace (k <= 1024, d <= 256).  Calls
    on one device share that scratch, so their GPU work must not overlap.
    """
    _check_X(X, labels)
    lib = load()
    N, D = X.shape
    count, s1, s2 = agg
    S = torch.empty((), dtype=torch.float64, device=X.device)
    s = torch.empty(N, dtype=torch.float32, device=X.device) if want_s else None
    saved = torch.empty(int(lib.sil_saved_size(N)), dtype=torch.uint8, device=X.device) if save else None
    rc = lib.sil_score_noalloc(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale),
                               _ptr(labels), K, METRICS[metric], _ptr(count), _ptr(s1), _ptr(s2),
                               _ptr(s), _ptr(S), _ptr(saved), _ptr(status), _stream_handle(X.device))
    _rc(rc, "sil_score_noalloc")
    return Score(S=S, s=s, saved=saved)


def unpack_saved(saved: torch.Tensor, N: int):
    """(a float32[N], b float32[N], kstar int32[N]) views of a saved record."""
    f = saved.view(torch.float32)
    return f[:N], f[N:2 * N], saved.view(torch.int32)[2 * N:3 * N]


def score_backward(X: torch.Tensor, labels: torch.Tensor, K: int, agg, metric: str = "sqeuclidean",
                   saved: torch.Tensor | None = None, grad_S: torch.Tensor | None = None,
                   col_scale: torch.Tensor | None = None, out: torch.Tensor | None = None,
                   status: torch.Tensor | None = None) -> torch.Tensor:
    """grad_S * dS/dX (float32 N x D) with labels fixed."""
    _check_X(X, labels)
    lib = load()
    N, D = X.shape
    count, s1, s2 = agg
    dX = out if out is not None else torch.empty(N, D, dtype=torch.float32, device=X.device)
    if grad_S is not None:
        grad_S = grad_S.to(device=X.device, dtype=torch.float64).reshape(())
    ws, need = _ws_for(X, K, metric)
    rc = lib.sil_score_backward(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale),
                                _ptr(labels), K, METRICS[metric], _ptr(count), _ptr(s1), _ptr(s2),
                                _ptr(saved), _ptr(grad_S), _ptr(dX), dX.stride(0), _ptr(ws), need,
                                _ptr(status), _stream_handle(X.device))
    _rc(rc, "sil_score_backward")
    return dX


def score_batched(X: torch.Tensor, labels: torch.Tensor, ks, metric: str = "sqeuclidean",
                  col_scale: torch.Tensor | None = None,
                  status: torch.Tensor | None = None) -> torch.Tensor:
    """S (float64[B]) of the B labelings in the rows of ``labels`` (B x N int32)."""
    if labels.dim() != 2:
        raise ValueError("labels must be B x N")
    _check_X(X, labels[0])
    lib = load()
    N, D = X.shape
    B = labels.shape[0]
    k_host = (ctypes.c_int32 * B)(*[int(k) for k in ks])
    S = torch.empty(B, dtype=torch.float64, device=X.device)
    kmax = max(int(k) for k in ks)
    ws, need = _ws_for(X, kmax, metric, batch=B)
    rc = lib.sil_score_batched(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale),
                               _ptr(labels), labels.stride(0), k_host, B, METRICS[metric], _ptr(S),
                               _ptr(ws), need, _ptr(status), _stream_handle(X.device))
    _rc(rc, "sil_score_batched")
    return S


class BatchedGraph:
    """sil_score_batched captured once into a CUDA graph and replayed.

    All B labelings' launches (pass 1, finalisation, pass 2 and the mean for
    each) are recorded on a side stream at construction; run() replays them
    with one graph launch and returns the FP64 S of every labeling.  The
    graph keeps the device addresses of X, labels, the workspace and its
    output, so it is only valid while those tensors live and keep their
    contents' layout; build a new one for other inputs.
    """

    def __init__(self, X: torch.Tensor, labels: torch.Tensor, ks, metric: str = "sqeuclidean",
                 col_scale: torch.Tensor | None = None, status: torch.Tensor | None = None):
        self.X, self.labels, self.col_scale, self.status = X, labels, col_scale, status
        self.ks, self.metric = [int(k) for k in ks], metric
        score_batched(X, labels, self.ks, metric, col_scale=col_scale, status=status)  # sizes the workspace
        # the graph keeps this workspace's address: hold the buffer even if a
        # later, larger call replaces it in the cache
        self._ws, _ = _ws_for(X, max(self.ks), metric, batch=len(self.ks))
        torch.cuda.synchronize(X.device)
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(X.device)
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                self.S = score_batched(X, labels, self.ks, metric, col_scale=col_scale, status=status)
        torch.cuda.synchronize(X.device)

    def run(self) -> torch.Tensor:
        self.graph.replay()
        return self.S


def tensor_plan(dtype: torch.dtype, D: int, K: int):
    """(clusters per block, number of blocks) of the tensor-core pass 2, or None."""
    lib = load()
    bk, nb = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.sil_tensor_plan(_DTYPES[dtype], D, K, ctypes.byref(bk), ctypes.byref(nb))
    if rc == SIL_EUNSUPPORTED:
        return None
    _rc(rc, "sil_tensor_plan")
    return bk.value, nb.value


_DTYPES = {torch.float32: 0, torch.bfloat16: 1, torch.float8_e4m3fn: 2}
def tensor_kernels(dtype: torch.dtype, D: int, K: int) -> set:
    """Tensor-core kernels serving this shape: {"split"} (paths "auto" and
    "tensor"), {"tf32"} (path "tensor_tf32"), both or neither."""
    bits = int(load().sil_tensor_kernel(_DTYPES[dtype], D, K))
    return {name for bit, name in ((1, "split"), (2, "tf32")) if bits & bit}


def tensor_plan_candidates(dtype: torch.dtype, D: int, K: int, max_plans: int = 8):
    """Feasible tensor-path plans (block_k, A buffers, X stages, staged centroids, rank pass),
    best modelled first."""
    lib = load()
    buf = (ctypes.c_int32 * (5 * max_plans))()
    n = ctypes.c_int32(0)
    _rc(lib.sil_tensor_plan_candidates(_DTYPES[dtype], D, K, buf, max_plans, ctypes.byref(n)),
        "sil_tensor_plan_candidates")
    return [tuple(buf[5 * i:5 * i + 5]) for i in range(n.value)]


def tensor_plan_set(dtype: torch.dtype, D: int, K: int, plan=None) -> None:
    """Make `plan` (from tensor_plan_candidates) the choice for this shape; None restores the model."""
    lib = load()
    bk, nab, nxs, stz, rank = plan if plan is not None else (0, 0, 0, 0, 0)
    _rc(lib.sil_tensor_plan_set(_DTYPES[dtype], D, K, bk, nab, nxs, stz, rank), "sil_tensor_plan_set")


def autotune(X: torch.Tensor, labels: torch.Tensor, K: int, metric: str = "sqeuclidean",
             col_scale: torch.Tensor | None = None, max_plans: int = 6, reps: int = 3):
    """Time pass 2 under each of the best-modelled plans of the split-precision
    tensor kernel for this shape on these inputs and keep the fastest for the
    rest of the process.

    Returns [(seconds per call, plan), ...] in the order tried (empty when that
    kernel does not serve the shape).  The timing runs the real kernels on the
    caller's data; nothing is cached across processes.
    """
    N, D = X.shape
    plans = tensor_plan_candidates(X.dtype, D, K, max_plans)
    if not plans or tensor_plan(X.dtype, D, K) is None:
        return []
    agg = aggregate(X, labels, K, metric, col_scale=col_scale)
    stream = torch.cuda.current_stream(X.device)
    results = []
    for plan in plans:
        tensor_plan_set(X.dtype, D, K, plan)
        score(X, labels, K, agg, metric, col_scale=col_scale, path="tensor")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            score(X, labels, K, agg, metric, col_scale=col_scale, path="tensor")
        e1.record(stream)
        torch.cuda.synchronize(X.device)
        results.append((e0.elapsed_time(e1) / 1e3 / reps, plan))
    best = min(results)[1]
    tensor_plan_set(X.dtype, D, K, best)
    return results


def batched_plan_set(ranges: int = 8, a_buffers: int = 0) -> None:
    """Plan of the one-launch batched pass 2: CTAs per labeling block and A buffers (0: model)."""
    _rc(load().sil_batched_plan_set(int(ranges), int(a_buffers)), "sil_batched_plan_set")


def serves_one_launch(X: torch.Tensor, labels: torch.Tensor, ks) -> bool:
    """Whether sil_score_batched runs every labeling's pass 2 as one launch for these inputs."""
    N, D = X.shape
    return (X.dtype == torch.float32 and 32 <= D <= 64 and max(int(k) for k in ks) <= 512
            and labels.stride(0) % 4 == 0 and X.stride(0) % 4 == 0 and "split" in tensor_kernels(X.dtype, D, 256))


def autotune_batched(X: torch.Tensor, labels: torch.Tensor, ks, metric: str = "sqeuclidean",
                     col_scale: torch.Tensor | None = None, max_plans: int = 4, reps: int = 2):
    """Pick launch plans of sil_score_batched by timing them on these inputs.

    Where every labeling's pass 2 runs as one launch: the plan of that launch
    (CTAs per labeling block in 4, 8, 16, 32, 64 and 2 or 4 A buffers), timed on
    the whole batched call; returns {"one_launch": (ranges, a_buffers)}.
    Otherwise :func:`autotune` for each distinct k that the split-precision
    kernel serves, on the first labeling with that k; returns {k: fastest
    plan} (None where another kernel scores the shape)."""
    if serves_one_launch(X, labels, ks):
        stream = torch.cuda.current_stream(X.device)
        results = []
        for ranges in (4, 8, 16, 32, 64):
            for nab in (2, 4):
                batched_plan_set(ranges, nab)
                score_batched(X, labels, ks, metric, col_scale=col_scale)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    score_batched(X, labels, ks, metric, col_scale=col_scale)
                e1.record(stream)
                torch.cuda.synchronize(X.device)
                results.append((e0.elapsed_time(e1) / reps, (ranges, nab)))
        best_plan = min(results)[1]
        batched_plan_set(*best_plan)
        return {"one_launch": best_plan, "timings_ms": results}
    best = {}
    for b, k in enumerate(int(k) for k in ks):
        if k in best:
            continue
        if "split" not in tensor_kernels(X.dtype, X.shape[1], k):
            best[k] = None
            continue
        res = autotune(X, labels[b], k, metric, col_scale=col_scale, max_plans=max_plans, reps=reps)
        best[k] = min(res)[1] if res else None
    return best


def score_euclidean(X: torch.Tensor, labels: torch.Tensor, K: int, col_scale: torch.Tensor | None = None,
                    want_s: bool = False, save: bool = False, status: torch.Tensor | None = None) -> Score:
    """sil_score_euclidean: the exact (non-squared) Euclidean Silhouette by the
    quadratic method (O(N^2 D); no aggregates needed)."""
    _check_X(X, labels)
    lib = load()
    N, D = X.shape
    S = torch.empty((), dtype=torch.float64, device=X.device)
    s = torch.empty(N, dtype=torch.float32, device=X.device) if want_s else None
    saved = torch.empty(int(lib.sil_saved_size(N)), dtype=torch.uint8, device=X.device) if save else None
    need = int(lib.sil_euclidean_workspace_size(N, D, K))
    ws = _WS.get(X.device, need)
    rc = lib.sil_score_euclidean(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale), _ptr(labels), K,
                                 _ptr(s), _ptr(S), _ptr(saved), _ptr(ws), need, _ptr(status),
                                 _stream_handle(X.device))
    _rc(rc, "sil_score_euclidean")
    return Score(S=S, s=s, saved=saved)


def silhouette(X: torch.Tensor, labels: torch.Tensor, K: int, metric: str = "sqeuclidean",
               col_scale: torch.Tensor | None = None, want_s: bool = False,
               path: str = "auto", status: torch.Tensor | None = None, save: bool = False,
               out=None) -> Score:
    """Both passes: the Silhouette S (and optionally every s_i) of one labeling,
    in one call of sil_silhouette.  ``out`` = (count, s1, s2) device tensors
    receive the aggregates."""
    _check_X(X, labels)
    lib = load()
    N, D = X.shape
    if out is None:
        out = (torch.empty(K, dtype=torch.int64, device=X.device),
               torch.empty(K, D, dtype=torch.float64, device=X.device),
               torch.empty(K, dtype=torch.float64, device=X.device))
    count, s1, s2 = out
    S = torch.empty((), dtype=torch.float64, device=X.device)
    s = torch.empty(N, dtype=torch.float32, device=X.device) if want_s else None
    saved = torch.empty(int(lib.sil_saved_size(N)), dtype=torch.uint8, device=X.device) if save else None
    ws, need = _ws_for(X, K, metric)
    rc = lib.sil_silhouette(_ptr(X), _dtype_code(X), N, D, X.stride(0), _ptr(col_scale), _ptr(labels), K,
                            METRICS[metric], _ptr(count), _ptr(s1), _ptr(s2), _ptr(s), _ptr(S), _ptr(saved),
                            PATHS[path], _ptr(ws), need, _ptr(status), _stream_handle(X.device))
    _rc(rc, "sil_silhouette")
    return Score(S=S, s=s, saved=saved)


def selftest_bounded_wait(device=None) -> tuple[int, int, int]:
    """Failure-detection self-test (about one second, no data): how the
    library's bounded kernel waits end when nothing completes them -- the three
    words of sil_selftest_bounded_wait (expected: SIL_ETIMEOUT, SIL_ETIMEOUT, 1)."""
    lib = load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = torch.zeros(3, dtype=torch.int32, device=dev)
    _rc(lib.sil_selftest_bounded_wait(_ptr(out), _stream_handle(dev)), "sil_selftest_bounded_wait")
    torch.cuda.synchronize(dev)
    return tuple(int(v) & 0xFFFFFFFF for v in out.cpu().tolist())


# ----------------------------------------------------------- out of core
def row_chunks(N: int, chunk_rows: int) -> list[tuple[int, int]]:
    """[start, stop) ranges of at most ``chunk_rows`` rows covering rows 0..N-1 in order."""
    if chunk_rows <= 0:
        raise ValueError("chunk_rows must be positive")
    if N < 0:
        raise ValueError("N must be non-negative")
    return [(a, min(a + chunk_rows, N)) for a in range(0, N, chunk_rows)]


def chunk_mean(S_chunks: torch.Tensor, n_chunks: torch.Tensor) -> torch.Tensor:
    """sil_chunk_mean: S of all rows from per-chunk means (device float64[m])
    and row counts (device int64[m]), as a 0-d device float64."""
    out = torch.empty((), dtype=torch.float64, device=S_chunks.device)
    rc = load().sil_chunk_mean(_ptr(S_chunks), _ptr(n_chunks), int(S_chunks.numel()), _ptr(out),
                               _stream_handle(S_chunks.device))
    _rc(rc, "sil_chunk_mean")
    return out


@dataclasses.dataclass
class ChunkedScore:
    S: float                         # the Silhouette of all rows
    s: torch.Tensor | None           # float32[N] on the host (pinned), or None
    chunks: int                      # row chunks streamed per pass


def silhouette_chunked(X_host: torch.Tensor, labels_host: torch.Tensor, K: int,
                       metric: str = "sqeuclidean", chunk_rows: int = 1 << 22, device=None,
                       col_scale: torch.Tensor | None = None, want_s: bool = False) -> ChunkedScore:
    """S (and optionally every s_i) of data held in HOST memory, streamed through the GPU.

    For datasets larger than the device, or held by the host anyway.  The
    aggregates are sums over rows (Eq. 6, 8, 16), so pass 1 adds every chunk's
    into one set (SIL_AGG_ACCUMULATE), like the per-worker partial sums the
    paper merges; pass 2 streams the chunks again and scores each against the
    aggregates of ALL rows (a_i, b_i of a point depend only on them), and S is
    the row-weighted mean of the chunk means.  Each chunk is copied from host
    memory on a copy stream into one of two device buffers, so the copy of
    chunk c+1 overlaps the kernels of chunk c (pinned host tensors make the
    copies asynchronous).  Every step of both passes, and the row-weighted mean
    of the chunk means (sil_chunk_mean), runs in libsil's kernels; this
    function only moves chunks.  It synchronises once, at the end, and raises
    SilError on a data error.
    """
    if X_host.is_cuda or labels_host.is_cuda:
        raise ValueError("silhouette_chunked streams host tensors; use silhouette() for device data")
    if X_host.dim() != 2 or X_host.stride(1) != 1:
        raise ValueError("X_host must be a 2-D tensor with unit column stride")
    if labels_host.dtype != torch.int32 or labels_host.dim() != 1 or labels_host.stride(0) != 1:
        raise ValueError("labels_host must be a contiguous 1-D int32 tensor")
    N, D = X_host.shape
    if labels_host.numel() != N:
        raise ValueError("one label per row")
    if N == 0:
        raise ValueError("no rows")
    chunks = row_chunks(N, chunk_rows)
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    load()
    rows = min(chunk_rows, N)
    Xd = [torch.empty(rows, D, dtype=X_host.dtype, device=device) for _ in range(2)]
    ld = [torch.empty(rows, dtype=torch.int32, device=device) for _ in range(2)]
    agg = (torch.zeros(K, dtype=torch.int64, device=device),
           torch.zeros(K, D, dtype=torch.float64, device=device),
           torch.zeros(K, dtype=torch.float64, device=device))
    status = new_status(device)
    S_dev = torch.empty(len(chunks), dtype=torch.float64, device=device)
    n_dev = torch.tensor([b - a for a, b in chunks], dtype=torch.int64).to(device)
    s_host = torch.empty(N, dtype=torch.float32).pin_memory() if want_s else None
    compute = torch.cuda.current_stream(device)
    copy_stream = torch.cuda.Stream(device)
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    for ev in consumed:
        ev.record(compute)

    def stage(i, a, b):
        # chunk i into buffer i % 2 once the kernels that last read it are done
        buf = i % 2
        copy_stream.wait_event(consumed[buf])
        with torch.cuda.stream(copy_stream):
            Xd[buf][:b - a].copy_(X_host[a:b], non_blocking=True)
            ld[buf][:b - a].copy_(labels_host[a:b], non_blocking=True)
            copied[buf].record(copy_stream)
        compute.wait_event(copied[buf])
        return Xd[buf][:b - a], ld[buf][:b - a], buf

    try:
        with torch.cuda.device(device):
            for i, (a, b) in enumerate(chunks):  # pass 1: one set of aggregates over all chunks
                x, lab, buf = stage(i, a, b)
                aggregate(x, lab, K, metric, col_scale=col_scale, out=agg, accumulate=i > 0, status=status)
                consumed[buf].record(compute)
            for i, (a, b) in enumerate(chunks):  # pass 2: every chunk against all rows' aggregates
                x, lab, buf = stage(len(chunks) + i, a, b)
                r = score(x, lab, K, agg, metric, col_scale=col_scale, want_s=want_s, status=status)
                S_dev[i].copy_(r.S)
                if want_s:
                    s_host[a:b].copy_(r.s, non_blocking=True)
                consumed[buf].record(compute)
            S = chunk_mean(S_dev, n_dev)
    finally:
        # also when a call raised: no copy may still target the buffers freed on return
        copy_stream.synchronize()
        compute.synchronize()
    check_status(status, "silhouette_chunked")
    return ChunkedScore(S=float(S.item()), s=s_host, chunks=len(chunks))
