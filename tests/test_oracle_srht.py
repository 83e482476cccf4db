"""Pins for the oracle's block SRHT sketch (Section 4, the Spark implementation's sketching matrix)."""
import numpy as np
import pytest

from oracle import smp
from paper_1610_06656_gb300 import configs, synth


@pytest.mark.parametrize("R", [2, 8, 64, 1024])
def test_fwht_is_the_sylvester_hadamard_product(R):
    from scipy.linalg import hadamard
    X = np.random.default_rng(R).standard_normal((R, 5))
    np.testing.assert_allclose(smp.fwht(X), hadamard(R) @ X, rtol=0, atol=1e-12 * np.sqrt(R) * np.abs(X).max() * R)


def test_parseval():
    """H_R D is sqrt(R) times an orthogonal matrix: ||fwht(D x)||^2 = R ||x||^2."""
    x = np.random.default_rng(1).standard_normal(4096)
    D = smp.srht_signs(7, 0, 4096)
    assert abs(np.sum(smp.fwht(D * x) ** 2) / (4096 * np.sum(x ** 2)) - 1.0) < 1e-12


def test_brute_force_pi():
    """d = 40 in blocks of 16 (the last one partial): Pi built entry by entry from popcounts equals the FWHT path."""
    d, n1, n2, k, p = 40, 6, 5, 9, 4
    rng = np.random.default_rng(2)
    A, B = rng.standard_normal((d, n1)), rng.standard_normal((d, n2))
    R = 1 << p
    Pi = np.zeros((k, d))
    D = smp.srht_signs(3, 0, d)
    for b in range((d + R - 1) // R):
        S = smp.srht_rows(3, b, k, p)
        for a in range(k):
            for t in range(b * R, min(d, (b + 1) * R)):
                Pi[a, t] = (-1.0) ** bin(int(S[a]) & (t - b * R)).count("1") * D[t] / np.sqrt(k)
    st = smp.sketch_srht(A, B, k, 3, p)
    np.testing.assert_allclose(st.At, Pi @ A, atol=1e-12)
    np.testing.assert_allclose(st.Bt, Pi @ B, atol=1e-12)
    np.testing.assert_allclose(st.sA, (A ** 2).sum(0), rtol=1e-14)


def test_sampled_rows_are_uniform_and_signs_balanced():
    from scipy import stats
    S = np.concatenate([smp.srht_rows(5, b, 1000, 4) for b in range(40)])   # 40,000 draws over 16 rows
    counts = np.bincount(S, minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-6
    D = smp.srht_signs(5, 0, 100000)
    assert abs(D.mean()) < 5 / np.sqrt(100000)


def test_norm_preserved_in_expectation():
    """E ||Pi x||^2 = ||x||^2: the mean over 400 seeds of ||Pi x||^2 / ||x||^2 is within 1.5% of 1 for a vector
    spread over three blocks."""
    x = np.random.default_rng(4).standard_normal((3000, 1))
    r = [float(np.sum(smp.sketch_srht(x, None, 16, s, 10, same_ab=True).At ** 2) / np.sum(x ** 2))
         for s in range(400)]
    assert abs(np.mean(r) - 1.0) < 0.015


def test_same_quality_as_the_gaussian_sketch():
    """Section 4's footnote: the SRHT keeps the output quality of the Gaussian sketch. Tiny workload (blocks of
    256 rows): SMP-PCA's spectral error with either sketch is within 10% of the other."""
    w = configs.WORKLOADS["tiny"]
    A, B = synth.lowrank_plus_noise(w["d"], w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"], seed=1000,
                                    dtype=np.float64)
    m = smp.default_m(w["n1"], w["n2"], w["r"])
    M = A.T @ B
    e = {}
    for name, lg in (("gaussian", None), ("srht", 8)):
        out = smp.smp_pca(A, B, w["r"], w["k"], m, w["T"], seed=1, sample_seed=2, srht_log2=lg)
        e[name] = smp.spectral_error(M, out["U"], out["S"], out["V"])
    print("spectral errors:", e)
    assert abs(e["srht"] - e["gaussian"]) < 0.1 * e["gaussian"]
