"""Pins for the oracle's row-wise multinomial sampler (Appendix, "Sampling") and its blocked prefix sum."""
import math

import numpy as np
import pytest

from oracle import smp
from paper_1610_06656_gb300 import configs, synth


def test_blocked_prefix_exact_on_integers_and_close_to_fsum():
    rng = np.random.default_rng(0)
    x = rng.integers(0, 1000, size=5000).astype(np.float64)           # integer sums are exact in binary64
    np.testing.assert_array_equal(smp.blocked_prefix(x), np.cumsum(x.astype(np.int64)).astype(np.float64))
    y = rng.uniform(0.0, 1.0, size=3000)
    ref = np.array([math.fsum(y[:j + 1]) for j in range(0, 3000, 97)])
    np.testing.assert_allclose(smp.blocked_prefix(y)[::97], ref, rtol=1e-13)


def test_row_totals_follow_the_appendix():
    """Draws per row c_i = round(m_i) with m_i = m (||A_i||^2 / (2 ||A||_F^2) + 1 / (2 n1)) (the Appendix's row
    total, with the B-term normaliser of Eq. (1)); the totals sum to m within n1 / 2."""
    rng = np.random.default_rng(1)
    sA, sB = rng.uniform(0.01, 3.0, 60), rng.uniform(0.01, 3.0, 45)
    m = 1234.5
    rows, cols, qhat, cnt = smp.sample_omega_multinomial(sA, sB, m, 3)
    per_row = np.bincount(rows, weights=cnt, minlength=60)
    mi = m * (sA / (2 * sA.sum()) + 1.0 / (2 * 60))
    np.testing.assert_array_equal(per_row, np.floor(mi + 0.5))
    assert abs(per_row.sum() - m) <= 60 / 2


def test_draw_frequencies_match_the_multinomial():
    """Chi-square of the column counts of each row against q~_ij = q_ij / m_i (large m: about 20,000 draws per
    row); every row's statistic stays below the 1e-6 tail of its chi-square law."""
    from scipy import stats
    rng = np.random.default_rng(2)
    n1, n2 = 4, 30
    sA, sB = rng.uniform(0.1, 2.0, n1), rng.uniform(0.01, 5.0, n2)
    m = 80000.0
    rows, cols, qhat, cnt = smp.sample_omega_multinomial(sA, sB, m, 11)
    q, _ = smp.q_matrix(sA, sB, m)
    for i in range(n1):
        c = np.zeros(n2)
        c[cols[rows == i]] = cnt[rows == i]
        expect = c.sum() * q[i] / q[i].sum()
        chi2 = float(((c - expect) ** 2 / expect).sum())
        assert chi2 < stats.chi2.isf(1e-6, n2 - 1), (i, chi2)


def test_weights_are_unbiased():
    """E[sum over Omega of M_ij count_ij / (c_i q~_ij)] = sum_ij M_ij: averaged over 200 seeds the weighted sum of a
    fixed positive M is within 1% of the full sum (its standard error here is about 0.3%)."""
    rng = np.random.default_rng(3)
    n1, n2 = 20, 25
    sA, sB = rng.uniform(0.1, 2.0, n1), rng.uniform(0.1, 2.0, n2)
    M = rng.uniform(0.5, 1.5, size=(n1, n2))
    tot = []
    for seed in range(200):
        rows, cols, qhat, _ = smp.sample_omega_multinomial(sA, sB, 150.0, seed)
        tot.append(float((M[rows, cols] / qhat).sum()))
    assert abs(np.mean(tot) / M.sum() - 1.0) < 0.01


def test_dominant_column_takes_every_draw():
    """alpha = 0 (all A columns zero) and every B column but the first zero: q~_i0 = 1, so each row draws column 0
    c_i times and Omega is the first column."""
    n1, n2 = 7, 2500                                          # n2 spans three prefix blocks
    sA = np.zeros(n1)
    sB = np.zeros(n2)
    sB[0] = 4.0
    rows, cols, qhat, cnt = smp.sample_omega_multinomial(sA, sB, 100.0, 5)
    np.testing.assert_array_equal(rows, np.arange(n1))
    np.testing.assert_array_equal(cols, np.zeros(n1))
    c = math.floor(100.0 / (2 * n1) + 0.5)
    np.testing.assert_array_equal(cnt, np.full(n1, c))
    np.testing.assert_array_equal(qhat, np.ones(n1))              # (c (q / q)) / c


def test_error_within_twice_the_bernoulli_models():
    """The Appendix bounds the multinomial model's error by twice the Bernoulli model's: on the tiny workload the
    SMP-PCA error with multinomial Omega stays below twice the Bernoulli one."""
    w = configs.WORKLOADS["tiny"]
    A, B = synth.lowrank_plus_noise(w["d"], w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"], seed=1000,
                                    dtype=np.float64)
    m = smp.default_m(w["n1"], w["n2"], w["r"])
    M = A.T @ B
    errs = {}
    for sampler in ("bernoulli", "multinomial"):
        out = smp.smp_pca(A, B, w["r"], w["k"], m, w["T"], seed=1, sample_seed=2, sampler=sampler)
        errs[sampler] = smp.spectral_error(M, out["U"], out["S"], out["V"])
    print("spectral errors:", errs)
    assert errs["multinomial"] <= 2.0 * errs["bernoulli"]
