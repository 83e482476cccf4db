"""Pins for the oracle's single pass (Algorithm 1, step 2) and the rescale factors."""
import math

import numpy as np

from oracle import philox, smp
from paper_1610_06656_gb300 import synth


def test_pi_entries_have_variance_one_over_k():
    k = 64
    P = philox.pi_block(99, k, 0, 20000)
    assert P.shape == (k, 20000)
    assert abs(P.var() * k - 1.0) < 6 * math.sqrt(2.0 / P.size)
    assert abs(P.mean()) < 6 / math.sqrt(k * P.size)


def test_pi_block_boundaries_are_consistent():
    """Pi is a function of (seed, a, t) only, so any split of the rows gives the same columns."""
    k = 36  # not a multiple of 8: the last Philox group feeds rows 32..35
    full = philox.pi_block(5, k, 1000, 300)
    parts = np.concatenate([philox.pi_block(5, k, 1000, 7), philox.pi_block(5, k, 1007, 293)], axis=1)
    np.testing.assert_array_equal(full, parts)
    big = philox.pi_block(5, 40, 1000, 300)
    np.testing.assert_allclose(full, big[:36] * math.sqrt(40) / math.sqrt(36), rtol=1e-14)


def test_pi_rows_above_2_32():
    t0 = (1 << 32) - 2
    P = philox.pi_block(1, 8, t0, 4)
    # row index t feeds the counter as (t lo, t hi); the column for t = 2^32 must differ from t = 0
    assert not np.allclose(P[:, 2], philox.pi_block(1, 8, 0, 1)[:, 0])


def test_identity_pi_gives_exact_sketch_and_products():
    A, B = synth.lowrank_plus_noise(40, 7, 9, 3, 0.1, 0.5, seed=1, dtype=np.float64)
    st = smp.sketch(A, B, k=40, seed=0, block_rows=16, pi=np.eye(40))
    np.testing.assert_array_equal(st.At, A)
    np.testing.assert_array_equal(st.Bt, B)
    rows, cols = np.meshgrid(np.arange(7), np.arange(9), indexing="ij")
    est = smp.estimate(rows.ravel(), cols.ravel(), st.At, st.Bt, st.sA, st.sB)
    np.testing.assert_allclose(est.reshape(7, 9), A.T @ B, rtol=1e-12, atol=1e-12)


def test_sketch_equals_brute_force_pi_product():
    d, n1, n2, k = 300, 6, 5, 24
    A, B = synth.lowrank_plus_noise(d, n1, n2, 2, 0.1, 0.5, seed=2, dtype=np.float32)
    Pfull = np.stack([[philox.pi_block(17, k, t, 1)[a, 0] for t in range(d)] for a in range(k)])
    st = smp.sketch(A, B, k, 17, block_rows=64)
    np.testing.assert_allclose(st.At, Pfull @ A.astype(np.float64), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st.Bt, Pfull @ B.astype(np.float64), rtol=1e-12, atol=1e-12)


def test_blocks_in_any_order():
    A, B = synth.lowrank_plus_noise(500, 8, 8, 2, 0.1, 0.5, seed=3, dtype=np.float32)
    ref = smp.sketch(A, B, 16, 4, block_rows=100)
    st = smp.SketchState(8, 8, 16, 4)
    for r0 in [400, 0, 300, 100, 200]:
        st.accumulate(A[r0:r0 + 100], B[r0:r0 + 100], r0)
    np.testing.assert_allclose(st.At, ref.At, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st.sB, ref.sB, rtol=1e-13)


def test_column_norms_exact_on_integers():
    rng = np.random.default_rng(0)
    A = rng.integers(-1000, 1000, size=(777, 5)).astype(np.float32)
    st = smp.sketch(A, None, 8, 0, block_rows=100, same_ab=True)
    exact = [sum(int(v) ** 2 for v in A[:, i]) for i in range(5)]
    assert [int(v) for v in st.sA] == exact
    assert st.sA is st.sB and st.At is st.Bt


def test_rescaled_sketch_columns_carry_true_norms():
    A, B = synth.lowrank_plus_noise(400, 10, 12, 3, 0.1, 0.5, seed=4)
    st = smp.sketch(A, B, 20, 8)
    DA = smp.rescale_factors(st.At, st.sA)
    np.testing.assert_allclose(np.linalg.norm(st.At * DA[None, :], axis=0),
                               np.linalg.norm(A.astype(np.float64), axis=0), rtol=1e-12)


def test_jl_norm_preservation_on_average():
    """E ||Pi x||^2 = ||x||^2 for Pi with N(0, 1/k) entries (Lemma B.3/B.4 setting)."""
    A = np.random.default_rng(5).standard_normal((600, 400))    # independent columns
    k = 50
    st = smp.sketch(A, None, k, 21, same_ab=True)
    ratio = (st.At ** 2).sum(0) / st.sA
    assert abs(ratio.mean() - 1.0) < 6 * math.sqrt(2.0 / k) / math.sqrt(400)


def test_zero_column_rescale_is_zero():
    A = np.zeros((10, 3))
    A[:, 1] = 1.0
    st = smp.sketch(A, None, 4, 0, same_ab=True)
    D = smp.rescale_factors(st.At, st.sA)
    assert D[0] == 0.0 and D[2] == 0.0 and D[1] > 0
