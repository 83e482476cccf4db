"""Pins for the oracle's WAltMin (Algorithm 2) and canonical form."""
import math

import numpy as np

from oracle import smp


def _lowrank(n1, n2, r, seed, noise=0.0):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((n1, r)))[0]
    V = np.linalg.qr(rng.standard_normal((n2, r)))[0]
    S = np.geomspace(10.0, 1.0, r)
    M = (U * S) @ V.T
    if noise:
        M = M + noise * rng.standard_normal((n1, n2)) / math.sqrt(max(n1, n2))
    return M


def _all_entries(n1, n2):
    rows, cols = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    return rows.ravel(), cols.ravel()


def test_rank_one_half_step_closed_form():
    """At r = 1 the V-update is v_j = sum_i w_ij u_i M~_ij / sum_i w_ij u_i^2 (Appendix C, proof of the main
    theorem: the closed-form WAltMin update)."""
    rng = np.random.default_rng(1)
    n1, n2 = 30, 20
    rows, cols = _all_entries(n1, n2)
    keep = rng.random(rows.shape[0]) < 0.4
    rows, cols = rows[keep], cols[keep]
    vals = rng.standard_normal(rows.shape[0])
    w = 1.0 / rng.uniform(0.1, 1.0, rows.shape[0])
    u = rng.standard_normal((n1, 1))
    V = smp.weighted_ls(n2, cols, rows, vals, w, u)
    for j in range(n2):
        s = cols == j
        num = np.sum(w[s] * u[rows[s], 0] * vals[s])
        den = np.sum(w[s] * u[rows[s], 0] ** 2)
        assert abs(V[j, 0] - num / den) <= 1e-8 * abs(num / den) + 1e-14


def test_row_without_samples_is_zero():
    U = np.ones((3, 2))
    V = smp.weighted_ls(4, np.array([0, 0, 2]), np.array([0, 1, 2]), np.ones(3), np.ones(3), U)
    assert np.all(V[1] == 0.0) and np.all(V[3] == 0.0)


def test_full_sampling_recovers_exact_low_rank_svd():
    """q^ = 1 (w = 1) on an exactly rank-r matrix: WAltMin returns its SVD (Algorithm 2 with full Omega)."""
    n1, n2, r = 40, 30, 4
    M = _lowrank(n1, n2, r, seed=2)
    rows, cols = _all_entries(n1, n2)
    sA = np.ones(n1)
    Uh, Vh = smp.waltmin(n1, n2, rows, cols, M[rows, cols], np.ones(rows.shape[0]), r, 5, sA)
    U, S, V = smp.canonical(Uh, Vh)
    Ur, Sr, Vrt = np.linalg.svd(M)
    # the ridge reading (lambda = 1e-10 tr(G)/r) biases the solve by at most ~1e-10 * cond(G) ~ 3e-9 here
    np.testing.assert_allclose(S, Sr[:r], rtol=1e-8)
    assert np.linalg.norm((U * S) @ V.T - M, 2) < 1e-8 * Sr[0]


def test_full_sampling_converges_to_truncated_svd():
    """With full observation the alternating LS fixed point is the truncated SVD (Eckart-Young)."""
    n1, n2, r = 50, 40, 3
    M = _lowrank(n1, n2, r + 3, seed=3)
    rows, cols = _all_entries(n1, n2)
    Uh, Vh = smp.waltmin(n1, n2, rows, cols, M[rows, cols], np.ones(rows.shape[0]), r, 60, np.ones(n1))
    U, S, V = smp.canonical(Uh, Vh)
    err = smp.spectral_error(M, U, S, V)
    assert abs(err - smp.optimal_error(M, r)) < 1e-8


def test_weights_are_inverse_probabilities():
    q = np.array([1.0, 0.5, 0.25, 0.0])
    np.testing.assert_array_equal(smp.weights(q), [1.0, 2.0, 4.0, 0.0])


def test_trim_zeroes_heavy_rows_only():
    U0 = np.linalg.qr(np.random.default_rng(4).standard_normal((50, 2)))[0]
    sA = np.ones(50)
    sA[7] = 1e-6                      # a light column: its row bound 8 sqrt(r) ||A_7|| / ||A||_F is tiny
    out = smp.trim(U0, sA, smp.frobenius_sq(sA))
    assert np.all(out[7] == 0.0)
    keep = np.arange(50) != 7
    np.testing.assert_array_equal(out[keep], U0[keep])


def test_split_subsets_partition_omega():
    rows, cols = _all_entries(60, 70)
    T = 4
    sub = smp.split_subsets(rows, cols, T, seed=9)
    assert sub.min() == 0 and sub.max() == 2 * T
    counts = np.bincount(sub, minlength=2 * T + 1)
    p = 1.0 / (2 * T + 1)
    assert np.all(np.abs(counts - rows.shape[0] * p) < 6 * math.sqrt(rows.shape[0] * p * (1 - p)))
    np.testing.assert_array_equal(sub, smp.split_subsets(rows, cols, T, seed=9))


def test_split_mode_on_dense_sampling_converges_to_low_rank():
    """Split mode (Algorithm 2, step 3) on an exactly rank-2 matrix: each half-step sees a fresh subset of about
    30 samples per row and the error falls geometrically with T (Lemma C.2's descent)."""
    n1, n2, r = 300, 250, 2
    M = _lowrank(n1, n2, r, seed=5)
    rows, cols = _all_entries(n1, n2)
    errs = []
    for T in (3, 8):
        Uh, Vh = smp.waltmin(n1, n2, rows, cols, M[rows, cols], np.ones(rows.shape[0]), r, T, np.ones(n1),
                             split=smp.SPLIT_OMEGA, split_seed=3)
        errs.append(smp.spectral_error(M, *smp.canonical(Uh, Vh)))
    assert errs[1] < 1e-3 and errs[1] < 0.1 * errs[0]


def test_canonical_form():
    rng = np.random.default_rng(6)
    Uh, Vh = rng.standard_normal((20, 3)), rng.standard_normal((15, 3))
    U, S, V = smp.canonical(Uh, Vh)
    np.testing.assert_allclose((U * S) @ V.T, Uh @ Vh.T, atol=1e-12)
    np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-12)
    assert np.all(np.diff(S) <= 0)
    for c in range(3):
        i = np.argmax(np.abs(U[:, c]))
        assert U[i, c] > 0
