"""Mutation check of the oracle pins (CPU only).

Each case plants one plausible mistake (a dropped term, a wrong sign, a wrong
denominator or index, a missing normalisation) in a temporary copy of the
oracle's C source, compiles that copy, and asserts that at least one pin --
the hand-worked golden values, the linear-equals-quadratic identity of Sec.
III, the library sums for the aggregates, or torch autograd of the quadratic
definition -- rejects it.  The committed oracle is never modified.
"""
import glob
import json
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from oracle import torch_ref

HERE = os.path.dirname(__file__)
SRC = os.path.join(os.path.dirname(HERE), "oracle", "sil_oracle.c")

MUTANTS = {
    "own_cluster_over_n": ("ai = count[c] > 1 ? cluster_mean(numer, (double)(count[c] - 1), metric) : 0.0;",
                           "ai = count[c] > 1 ? cluster_mean(numer, (double)count[c], metric) : 0.0;"),
    "drop_psi": ("numer = (double)count[k] * xi_sq + s2[k] - 2.0 * dot;",
                 "numer = (double)count[k] * xi_sq - 2.0 * dot;"),
    "cross_term_sign": ("numer = (double)count[k] * xi_sq + s2[k] - 2.0 * dot;",
                        "numer = (double)count[k] * xi_sq + s2[k] + 2.0 * dot;"),
    "eq2_branch": ("return b / a - 1.0;", "return a / b - 1.0;"),
    "b_includes_own": ("if (k == c || count[k] == 0) continue;", "if (count[k] == 0) continue;"),
    "cosine_no_normalise": ("numer = (double)count[k] - dot * inv_norm;",
                            "numer = (double)count[k] - dot;"),
    "aggregate_index": ("s1_t[((size_t)t * K + k) * D + l] += v;",
                        "s1_t[((size_t)t * K + k) * D + 0] += v;"),
    "bruteforce_self_in_a": ("ai = count[c] > 1 ? cluster_mean(sums[c], (double)(count[c] - 1), metric) : 0.0;",
                             "ai = count[c] > 1 ? cluster_mean(sums[c], (double)count[c], metric) : 0.0;"),
    "rms_no_square_root": ("if (metric == METRIC_EUCLIDEAN_RMS) return m > 0.0 ? sqrt(m) : 0.0;",
                           "if (metric == METRIC_EUCLIDEAN_RMS) return m;"),
    "rms_root_of_the_sum": ("if (metric == METRIC_EUCLIDEAN_RMS) return m > 0.0 ? sqrt(m) : 0.0;",
                            "if (metric == METRIC_EUCLIDEAN_RMS) return summed > 0.0 ? sqrt(summed) / members : 0.0;"),
    "euclidean_no_square_root": ("return metric == METRIC_EUCLIDEAN ? sqrt(s) : s;", "return s;"),
    "rms_linear_takes_cosine_form": ("if (metric != METRIC_COSINE)\n        numer",
                                     "if (metric == METRIC_SQEUCLIDEAN)\n        numer"),
    "cosine_one_norm": ("return 1.0 - dot / (row_norm(x, D) * row_norm(y, D));",
                        "return 1.0 - dot / row_norm(x, D);"),
    "grad_alpha_denominator": ("alpha[i] = dsa / (double)(count[c] - 1);",
                               "alpha[i] = dsa / (double)count[c];"),
    "grad_projection_sign": ("g[l] = gS * (g[l] - proj * x[l] / nrm) / nrm;",
                             "g[l] = gS * (g[l] + proj * x[l] / nrm) / nrm;"),
    "grad_dsdb": ("*dsb = a / (b * b);", "*dsb = a / b;"),
}


def _case(seed, N, D, K, metric):
    rng = np.random.default_rng(seed)
    C = rng.uniform(-3, 3, size=(K, D))
    lab = rng.integers(0, K, size=N).astype(np.int32)
    X = C[lab] + rng.normal(size=(N, D))
    if metric == "cosine":
        X += 0.1 * np.sign(X)
    return X, lab


def _failed_pins(lib):
    failed = []
    for path in sorted(glob.glob(os.path.join(HERE, "golden", "*.json"))):
        g = json.load(open(path))
        X, lab = np.array(g["X"], float), np.array(g["labels"], np.int32)
        s_ref = np.array([float(Fraction(v)) for v in g["s"]])
        for form in g.get("forms", ("bruteforce", "linear")):
            try:
                r = getattr(oracle, form)(X, lab, g["K"], g["metric"], lib=lib)
                if not np.allclose(r["s"], s_ref, rtol=0, atol=1e-12):
                    failed.append(f"golden:{os.path.basename(path)}:{form}")
            except ValueError:
                failed.append(f"golden:{os.path.basename(path)}:{form}:raised")
    for metric in ("sqeuclidean", "cosine", "euclidean_rms"):
        X, lab = _case(5, 80, 4, 5, metric)
        bf = oracle.bruteforce(X, lab, 5, metric, lib=lib)
        li = oracle.linear(X, lab, 5, metric, lib=lib)
        if not np.allclose(bf["s"], li["s"], rtol=0, atol=1e-10):
            failed.append(f"linear_vs_bruteforce:{metric}")
        if metric == "euclidean_rms":
            continue
        count, s1, s2 = oracle.aggregate(X, lab, 5, metric, lib=lib)
        V = X / np.linalg.norm(X, axis=1, keepdims=True) if metric == "cosine" else X
        if not np.allclose(s1, np.eye(5)[lab].T @ V, rtol=1e-12, atol=1e-12):
            failed.append(f"aggregate_sums:{metric}")
        Xt = torch.tensor(X, requires_grad=True)
        S, _ = torch_ref.silhouette(Xt, torch.tensor(lab), 5, metric)
        S.backward()
        g = oracle.linear_grad(X, lab, 5, metric, lib=lib)
        if not np.allclose(g, Xt.grad.numpy(), rtol=1e-8, atol=1e-12):
            failed.append(f"grad_vs_autograd:{metric}")
    return failed


def test_unmutated_oracle_passes_every_pin():
    assert _failed_pins(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    c_path.write_text(mutated)
    so_path = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(so_path),
                    str(c_path), "-lm"], check=True)
    failed = _failed_pins(oracle.bind(str(so_path)))
    assert failed, f"no pin rejects mutant {name}"
