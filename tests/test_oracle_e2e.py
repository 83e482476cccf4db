"""End-to-end pins for the oracle (Algorithm 1) against brute force and the paper's printed numbers."""
import json
import os

import numpy as np

from oracle import smp
from paper_1610_06656_gb300 import configs, synth


def test_brute_force_identity_pi_full_sampling():
    """Pi = I (k = d) and q^ = 1: M~ = A^T B exactly and WAltMin returns its truncated SVD."""
    d, n1, n2, r = 64, 16, 12, 3
    A, B = synth.lowrank_plus_noise(d, n1, n2, 3, 0.0, 0.5, seed=10, dtype=np.float64)
    out = smp.smp_pca(A, B, r, d, 1e12, 8, seed=1, sample_seed=2, pi=np.eye(d))
    M = A.T @ B
    assert out["rows"].shape[0] == n1 * n2
    np.testing.assert_allclose(out["vals"], M[out["rows"], out["cols"]], rtol=1e-12, atol=1e-12)
    U, S, V = out["U"], out["S"], out["V"]
    Ue, Se, Vte = np.linalg.svd(M)
    np.testing.assert_allclose(S, Se[:r], rtol=1e-9)
    assert np.linalg.norm((U * S) @ V.T - (Ue[:, :r] * Se[:r]) @ Vte[:r], 2) < 1e-9 * Se[0]


def test_tiny_workload_error_is_near_optimal():
    """The tiny workload (d = 2,000, n = 200, k = 100, r = 5): the error sits above the Eckart-Young optimum and
    well below the trivial error 1."""
    w = configs.WORKLOADS["tiny"]
    A, B = synth.lowrank_plus_noise(w["d"], w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"], seed=1000,
                                    dtype=np.float64)
    m = smp.default_m(w["n1"], w["n2"], w["r"])
    out = smp.smp_pca(A, B, w["r"], w["k"], m, w["T"], seed=1, sample_seed=2)
    M = A.T @ B
    err = smp.spectral_error(M, out["U"], out["S"], out["V"])
    opt = smp.optimal_error(M, w["r"])
    assert opt - 1e-12 <= err < 0.5
    _, qhat = smp.q_matrix(out["state"].sA, out["state"].sB, m)    # |Omega| ~ sum q^ (< m: q is clipped at 1)
    assert abs(out["rows"].shape[0] - qhat.sum()) < 6 * np.sqrt((qhat * (1 - qhat)).sum())


def test_table1_optimal_error_of_the_paper_generator(golden_dir):
    """Table 1, Synthetic: Optimal = 0.0271 for A = B = G D. The ratio sigma_6/sigma_1 of D G^T G D is governed by
    D (about 1/36 once G^T G is close to a multiple of I), so a smaller d = n reproduces it to a few percent."""
    g = json.load(open(os.path.join(golden_dir, "table1_synthetic.json")))
    A = synth.gd_matrix(1500, 1500, seed=4)
    M = A.T @ A
    assert abs(smp.optimal_error(M, g["r"]) - g["optimal"]) < 0.08 * g["optimal"]


def test_pca_case_a_equals_b():
    """A = B (Section 3, Remark 3): one sketch serves both sides and the result approximates A^T A."""
    A, _ = synth.lowrank_plus_noise(3000, 80, 80, 4, 0.05, 0.3, seed=11, same_ab=True, dtype=np.float64)
    M = A.T @ A
    errs = []
    for k in (60, 400):
        out = smp.smp_pca(A, None, 4, k, smp.default_m(80, 80, 4), 10, seed=5, sample_seed=6, same_ab=True)
        errs.append(smp.spectral_error(M, out["U"], out["S"], out["V"]))
    # the sketch error dominates here and shrinks like 1/sqrt(k) (Lemma B.7)
    assert smp.optimal_error(M, 4) - 1e-12 <= errs[1] < 0.2
    assert errs[1] < 0.75 * errs[0]
