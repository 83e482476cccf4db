"""Pins for the oracle's LELA path (the two-pass comparison method of Section 4, Table 1): the exact entries
against hand-worked and brute-force sums, LELA against SMP-PCA with Pi = I (whose estimates are then exact), full
sampling of an exactly rank-r product, and Table 1's ordering Optimal <= LELA <= SMP-PCA."""
import numpy as np

from oracle import smp
from paper_1610_06656_gb300 import configs, synth


def test_exact_entries_hand_worked():
    """A = [1 2; 3 4; 5 6], B = [1 0 2; 0 1 1; 1 1 0]: A^T B = [6 8 5; 8 10 8], worked out by hand."""
    A = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    B = np.array([[1.0, 0.0, 2.0], [0.0, 1.0, 1.0], [1.0, 1.0, 0.0]])
    rows = np.array([0, 0, 0, 1, 1, 1])
    cols = np.array([0, 1, 2, 0, 1, 2])
    assert smp.exact_entries(rows, cols, A, B).tolist() == [6.0, 8.0, 5.0, 8.0, 10.0, 8.0]


def test_exact_entries_brute_force_loops():
    """Random entries of a ragged Omega against a plain triple loop (sum over t of A[t, i] B[t, j])."""
    rng = np.random.default_rng(3)
    d, n1, n2 = 37, 9, 7
    A, B = rng.standard_normal((d, n1)), rng.standard_normal((d, n2))
    rows = rng.integers(0, n1, 25)
    cols = rng.integers(0, n2, 25)
    got = smp.exact_entries(rows, cols, A, B, chunk=4)   # several chunks and a ragged last one
    for e in range(25):
        s = 0.0
        for t in range(d):
            s += float(A[t, rows[e]]) * float(B[t, cols[e]])
        assert abs(got[e] - s) <= 1e-12 * (1.0 + abs(s))


def test_column_norms_pass():
    rng = np.random.default_rng(4)
    A, B = rng.standard_normal((20, 5)), rng.standard_normal((20, 3))
    sA, sB = smp.column_norms_sq(A, B)
    for i in range(5):
        assert abs(sA[i] - sum(float(x) * float(x) for x in A[:, i])) < 1e-12
    for j in range(3):
        assert abs(sB[j] - sum(float(x) * float(x) for x in B[:, j])) < 1e-12
    sA2, sB2 = smp.column_norms_sq(A, None, same_ab=True)
    assert sA2 is sB2 and np.array_equal(sA2, sA)


def test_lela_equals_smp_with_identity_pi():
    """With Pi = I (k = d) the rescaled JL estimate of Eq. (2) is exactly A_i^T B_j, so SMP-PCA and LELA draw the
    same Omega and feed WAltMin the same values up to rounding."""
    d, n1, n2, r = 48, 14, 11, 2
    A, B = synth.lowrank_plus_noise(d, n1, n2, 3, 0.1, 0.5, seed=20, dtype=np.float64)
    m = 0.6 * n1 * n2
    s = smp.smp_pca(A, B, r, d, m, 6, seed=1, sample_seed=5, pi=np.eye(d))
    l = smp.lela(A, B, r, m, 6, sample_seed=5)
    assert np.array_equal(s["rows"], l["rows"]) and np.array_equal(s["cols"], l["cols"])
    np.testing.assert_allclose(l["vals"], s["vals"], rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(l["S"], s["S"], rtol=1e-9)
    M = A.T @ B
    assert abs(smp.spectral_error(M, l["U"], l["S"], l["V"]) - smp.spectral_error(M, s["U"], s["S"], s["V"])) < 1e-9


def test_lela_full_sampling_recovers_rank_r():
    """q^ = 1 everywhere and A^T B of rank r exactly: LELA returns A^T B itself."""
    d, n, r = 30, 15, 3
    A, B = synth.lowrank_plus_noise(d, n, n, r, 0.0, 0.5, seed=21, dtype=np.float64)
    out = smp.lela(A, B, r, 1e12, 8, sample_seed=2)
    assert out["rows"].shape[0] == n * n
    M = A.T @ B
    assert smp.spectral_error(M, out["U"], out["S"], out["V"]) < 1e-8


def test_lela_pca_case():
    """A = B (PCA): the same as passing B = A explicitly."""
    d, n, r = 40, 12, 2
    A, _ = synth.lowrank_plus_noise(d, n, n, 2, 0.1, 0.5, seed=22, dtype=np.float64)
    a = smp.lela(A, None, r, 60.0, 5, sample_seed=3, same_ab=True)
    b = smp.lela(A, A.copy(), r, 60.0, 5, sample_seed=3)
    assert np.array_equal(a["rows"], b["rows"])
    np.testing.assert_allclose(a["S"], b["S"], rtol=1e-12)


def test_table1_ordering_on_the_tiny_workload():
    """Table 1's ordering: Optimal <= LELA <= SMP-PCA. On the tiny workload (d = 2,000, n = 200, k = 100, r = 5)
    the exact entries put LELA within 1% of the Eckart-Young optimum, well below SMP-PCA's estimate-based error."""
    w = configs.WORKLOADS["tiny"]
    A, B = synth.lowrank_plus_noise(w["d"], w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"], seed=1000,
                                    dtype=np.float64)
    m = smp.default_m(w["n1"], w["n2"], w["r"])
    M = A.T @ B
    opt = smp.optimal_error(M, w["r"])
    l = smp.lela(A, B, w["r"], m, w["T"], sample_seed=2)
    s = smp.smp_pca(A, B, w["r"], w["k"], m, w["T"], seed=1, sample_seed=2)
    e_l = smp.spectral_error(M, l["U"], l["S"], l["V"])
    e_s = smp.spectral_error(M, s["U"], s["S"], s["V"])
    assert opt - 1e-12 <= e_l <= 1.01 * opt
    assert e_l < e_s


def test_table1_ordering_on_the_gd_model():
    """Table 1's generator, A = B = G D (D_ii = 1 / i, one shared G), at d = n = 1,000 with r = 5, T = 10 and
    m = 4 n r ln n: LELA's exact entries reach the Eckart-Young optimum (sigma_6 / sigma_1, near 1 / 36), and
    SMP-PCA with k = 200 stays above LELA, the ordering Table 1 prints for d = n = 100,000."""
    n, r = 1000, 5
    A = synth.gd(n, n, seed=7)
    M = A.T @ A
    opt = smp.optimal_error(M, r)
    assert 0.025 < opt < 1.0 / 30
    m = smp.default_m(n, n, r)
    l = smp.lela(A, None, r, m, 10, sample_seed=2, same_ab=True)
    s = smp.smp_pca(A, None, r, 200, m, 10, seed=1, sample_seed=2, same_ab=True)
    e_l = smp.spectral_error(M, l["U"], l["S"], l["V"])
    e_s = smp.spectral_error(M, s["U"], s["S"], s["V"])
    assert opt - 1e-12 <= e_l <= opt * (1 + 1e-4)
    assert e_l < e_s


def test_gd_generator_scaling():
    """synth.gd is G D with D_ii = 1 / i: column i of A / (1 / i) is a standard Gaussian column (mean 0, variance
    1), and the squared column norms fall as d / i^2."""
    d, n = 4000, 50
    A = synth.gd(d, n, seed=5)
    G = A * np.arange(1, n + 1)
    assert abs(G.mean()) < 0.01 and abs(G.var() - 1.0) < 0.02
    sq = (A ** 2).sum(0)
    np.testing.assert_allclose(sq * np.arange(1, n + 1) ** 2 / d, 1.0, atol=0.12)


def test_lela_with_multinomial_sampling():
    """LELA on the Appendix's row-wise multinomial Omega: the same draws as the SMP-PCA oracle makes for the same
    norms, and with a generous budget an exactly rank-r product is recovered."""
    d, n, r = 40, 20, 2
    A, B = synth.lowrank_plus_noise(d, n, n, r, 0.0, 0.5, seed=23, dtype=np.float64)
    m = 40.0 * n * r
    out = smp.lela(A, B, r, m, 10, sample_seed=4, sampler="multinomial")
    rows, cols, qhat, _ = smp.sample_omega_multinomial(*smp.column_norms_sq(A, B), m, 4)
    assert np.array_equal(out["rows"], rows) and np.array_equal(out["cols"], cols)
    assert smp.spectral_error(A.T @ B, out["U"], out["S"], out["V"]) < 1e-6
