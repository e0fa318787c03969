"""FP64 CPU oracle for the linear-complexity Silhouette (arXiv 2303.14102).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product path (the CUDA library and its binding) never imports
this package, and this package never imports the product.

The arithmetic lives in ``sil_oracle.c`` (plain double-precision C, OpenMP
over independent points); this module only marshals numpy arrays.  A
differentiable pure-PyTorch restatement of the quadratic definition for
autograd lives in ``oracle.torch_ref``.

Passages followed (Sec./Eq. of the paper):
  aggregate     Eq. 5-6 (Psi), Eq. 8 (Y), Eq. 15-16 (Omega)
  bruteforce    Eq. 1-3 and the mean S of Sec. II; distances Eq. 4 / Eq. 12,
                the plain Euclidean distance, and the Limitations section's
                approximation of it (square root of each mean squared distance)
  linear        Eq. 10-11 (squared Euclidean; then the square root of each
                mean for the approximation), Eq. 17-18 (cosine)
  linear_grad   dS/dX of the linear form, labels fixed (no counterpart in
                the paper; derivation in the design notes)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sil_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ELABEL, EDEGENERATE, EZERONORM = 0, 1, 2, 3, 4
# "euclidean": the plain distance (quadratic form only); "euclidean_rms": the
# square root of each point-to-cluster mean squared distance (Limitations)
METRICS = {"sqeuclidean": 0, "cosine": 1, "euclidean": 2, "euclidean_rms": 3}


def build(force: bool = False) -> str:
    """Compile sil_oracle.c into liboracle.so with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def bind(path: str):
    """ctypes handle on a compiled oracle library at ``path`` (argtypes set)."""
    lib = ctypes.CDLL(path)
    dp, ip32, ip64 = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                      ctypes.POINTER(ctypes.c_int64))
    i64, i32, ci = ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    lib.oracle_num_threads.restype = ci
    lib.oracle_set_num_threads.argtypes = [ci]
    lib.oracle_set_num_threads.restype = None
    lib.oracle_aggregate.argtypes = [dp, i64, i32, ip32, i32, ci, ip64, dp, dp]
    lib.oracle_aggregate.restype = ci
    lib.oracle_bruteforce.argtypes = [dp, i64, i32, ip32, i32, ci, dp, dp, dp, ip32, dp]
    lib.oracle_bruteforce.restype = ci
    lib.oracle_linear.argtypes = [dp, i64, i32, ip32, i32, ci, ip64, dp, dp, ip64, i64,
                                  dp, dp, dp, ip32]
    lib.oracle_linear.restype = ci
    lib.oracle_linear_grad.argtypes = [dp, i64, i32, ip32, i32, ci, ctypes.c_double, dp]
    lib.oracle_linear_grad.restype = ci
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(_LIB)
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _prep(X, labels):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim != 2:
        raise ValueError("X must be N x D")
    labels = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    if labels.shape != (X.shape[0],):
        raise ValueError("labels must have one entry per row of X")
    return X, labels


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Run the oracle's loops on ``n`` threads from now on (1: single thread)."""
    _load().oracle_set_num_threads(int(n))


def aggregate(X, labels, K: int, metric: str = "sqeuclidean", lib=None):
    """Per-cluster (count, s1, s2): N_k, Y_k or Omega_k, Psi_k or sum ||x_hat||^2."""
    X, labels = _prep(X, labels)
    N, D = X.shape
    count = np.zeros(K, np.int64)
    s1 = np.zeros((K, D), np.float64)
    s2 = np.zeros(K, np.float64)
    st = (lib or _load()).oracle_aggregate(_p(X, ctypes.c_double), N, D, _p(labels, ctypes.c_int32), K,
                                  METRICS[metric], _p(count, ctypes.c_int64),
                                  _p(s1, ctypes.c_double), _p(s2, ctypes.c_double))
    if st != OK:
        raise ValueError(f"oracle_aggregate status {st}")
    return count, s1, s2


def bruteforce(X, labels, K: int, metric: str = "sqeuclidean", lib=None):
    """Quadratic Silhouette by definition.  Returns dict(s, a, b, kstar, S, status)."""
    X, labels = _prep(X, labels)
    N, D = X.shape
    s, a, b = (np.zeros(N, np.float64) for _ in range(3))
    kstar = np.zeros(N, np.int32)
    S = np.zeros(1, np.float64)
    st = (lib or _load()).oracle_bruteforce(_p(X, ctypes.c_double), N, D, _p(labels, ctypes.c_int32), K,
                                   METRICS[metric], _p(s, ctypes.c_double), _p(a, ctypes.c_double),
                                   _p(b, ctypes.c_double), _p(kstar, ctypes.c_int32),
                                   _p(S, ctypes.c_double))
    if st not in (OK, EDEGENERATE):
        raise ValueError(f"oracle_bruteforce status {st}")
    return dict(s=s, a=a, b=b, kstar=kstar, S=float(S[0]), status=st)


def linear(X, labels, K: int, metric: str = "sqeuclidean", agg=None, idx=None, lib=None):
    """Linear-form Silhouette (Eq. 10-11 / 17-18) from FP64 aggregates.

    ``agg`` = (count, s1, s2) from :func:`aggregate` (computed when None);
    ``idx`` = indices of the points to score (all when None).  S is the mean
    over the scored points, which is the global S only when idx is None.
    """
    X, labels = _prep(X, labels)
    N, D = X.shape
    if agg is None:
        agg = aggregate(X, labels, K, metric, lib=lib)
    count, s1, s2 = (np.ascontiguousarray(agg[0], np.int64),
                     np.ascontiguousarray(agg[1], np.float64),
                     np.ascontiguousarray(agg[2], np.float64))
    if idx is not None:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    M = N if idx is None else idx.shape[0]
    s, a, b = (np.zeros(M, np.float64) for _ in range(3))
    kstar = np.zeros(M, np.int32)
    st = (lib or _load()).oracle_linear(_p(X, ctypes.c_double), N, D, _p(labels, ctypes.c_int32), K,
                               METRICS[metric], _p(count, ctypes.c_int64), _p(s1, ctypes.c_double),
                               _p(s2, ctypes.c_double), _p(idx, ctypes.c_int64), M,
                               _p(s, ctypes.c_double), _p(a, ctypes.c_double),
                               _p(b, ctypes.c_double), _p(kstar, ctypes.c_int32))
    if st not in (OK, EDEGENERATE):
        raise ValueError(f"oracle_linear status {st}")
    S = float(s.mean()) if (st == OK and M > 0) else float("nan")
    return dict(s=s, a=a, b=b, kstar=kstar, S=S, status=st, agg=(count, s1, s2))


def linear_grad(X, labels, K: int, metric: str = "sqeuclidean", gS: float = 1.0, lib=None):
    """gS * dS/dX (N x D, FP64) with labels and the b_i argmin held fixed."""
    X, labels = _prep(X, labels)
    N, D = X.shape
    dX = np.zeros((N, D), np.float64)
    st = (lib or _load()).oracle_linear_grad(_p(X, ctypes.c_double), N, D, _p(labels, ctypes.c_int32), K,
                                    METRICS[metric], float(gS), _p(dX, ctypes.c_double))
    if st != OK:
        raise ValueError(f"oracle_linear_grad status {st}")
    return dX
