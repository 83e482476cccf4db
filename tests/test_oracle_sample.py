"""Pins for the oracle's biased sampling (Eq. (1), Algorithm 1 step 3)."""
import math

import numpy as np

from oracle import philox, smp


def _norms(n, seed):
    rng = np.random.default_rng(seed)
    return rng.gamma(0.7, 2.0, size=n) * (np.arange(1, n + 1) ** -0.6)


def test_q_sums_to_m_with_unequal_sizes():
    """sum_ij q_ij = m (Section 2.1, after Eq. (1)); with n1 != n2 a swapped normaliser breaks this."""
    sA, sB = _norms(37, 1), _norms(91, 2)
    m = 900.0
    q, qhat = smp.q_matrix(sA, sB, m)
    assert abs(q.sum() - m) < 1e-12 * m
    assert np.all(qhat <= 1.0) and np.all(qhat == np.minimum(q, 1.0))
    # each half carries m / 2: the A-term of row i summed over j is m ||A_i||^2 / (2 ||A||_F^2)
    alpha, beta = smp.sampling_terms(sA, sB, m)
    assert abs(alpha.sum() * 91 - m / 2) < 1e-12 * m
    assert abs(beta.sum() * 37 - m / 2) < 1e-12 * m


def test_frobenius_is_left_to_right():
    s = np.array([1.0, 1e-16, 1e-16, -1.0 + 2 ** -52])
    seq = ((s[0] + s[1]) + s[2]) + s[3]
    assert smp.frobenius_sq(s) == seq


def test_omega_size_matches_expectation():
    sA, sB = _norms(150, 3), _norms(120, 4)
    m = 3000.0
    _, qhat = smp.q_matrix(sA, sB, m)
    rows, cols, qv = smp.sample_omega(sA, sB, m, seed=77)
    mean, var = qhat.sum(), (qhat * (1 - qhat)).sum()
    assert abs(rows.shape[0] - mean) < 6 * math.sqrt(var)
    np.testing.assert_array_equal(qv, qhat[rows, cols])


def test_omega_is_canonical_and_deterministic():
    sA, sB = _norms(40, 5), _norms(50, 6)
    r1 = smp.sample_omega(sA, sB, 500.0, seed=3)
    r2 = smp.sample_omega(sA, sB, 500.0, seed=3)
    for a, b in zip(r1, r2):
        np.testing.assert_array_equal(a, b)
    rows, cols, _ = r1
    key = rows * 50 + cols
    assert np.all(np.diff(key) > 0)


def test_inclusion_frequency_is_qhat():
    """Each entry is kept independently with probability q^_ij: over many seeds the empirical frequency matches."""
    sA, sB = _norms(12, 7), _norms(10, 8)
    m = 30.0
    _, qhat = smp.q_matrix(sA, sB, m)
    S = 400
    hits = np.zeros_like(qhat)
    for s in range(S):
        rows, cols, _ = smp.sample_omega(sA, sB, m, seed=1000 + s)
        hits[rows, cols] += 1
    freq = hits / S
    sd = np.sqrt(np.maximum(qhat * (1 - qhat), 1e-12) / S)
    z = np.abs(freq - qhat) / sd
    assert z.max() < 5.5
    assert np.all(hits[qhat >= 1.0] == S)


def test_coin_matches_definition_entrywise():
    sA, sB = _norms(6, 9), _norms(7, 10)
    m = 10.0
    _, qhat = smp.q_matrix(sA, sB, m)
    rows, cols, _ = smp.sample_omega(sA, sB, m, seed=5)
    kept = set(zip(rows.tolist(), cols.tolist()))
    for i in range(6):
        for j in range(7):
            x0, x1, _, _ = philox.philox4x32_10_scalar((i, j, 0, philox.TAG_SAMPLE), philox.seed_key(5))
            u = ((x0 >> 5) * 2.0 ** 26 + (x1 >> 6)) * 2.0 ** -53
            assert ((i, j) in kept) == (u < qhat[i, j])


def test_zero_side_contributes_nothing():
    sA = np.zeros(5)
    sB = _norms(6, 11)
    alpha, beta = smp.sampling_terms(sA, sB, 12.0)
    assert np.all(alpha == 0.0)
    assert abs(beta.sum() * 5 - 6.0) < 1e-12


def test_full_sampling_keeps_everything():
    sA, sB = _norms(9, 12), _norms(8, 13)
    rows, _, qv = smp.sample_omega(sA, sB, 1e9, seed=1)
    assert rows.shape[0] == 72 and np.all(qv == 1.0)
