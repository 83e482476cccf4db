"""Pins for the oracle's rescaled JL estimate (Eq. (2))."""
import json
import math
import os

import numpy as np

from oracle import smp
from paper_1610_06656_gb300 import synth


def test_parallel_columns_are_exact():
    """cos(theta) = +-1 gives the exact dot product (Section 2.1, discussion of Figure 3(a))."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((300, 4))
    B = np.stack([2.5 * A[:, 0], -0.3 * A[:, 2], A[:, 3] * 7.0], axis=1)
    st = smp.sketch(A, B, 12, seed=3)
    rows = np.array([0, 2, 3])
    cols = np.array([0, 1, 2])
    est = smp.estimate(rows, cols, st.At, st.Bt, st.sA, st.sB)
    exact = np.einsum("ti,ti->i", A[:, rows], B[:, cols])
    np.testing.assert_allclose(est, exact, rtol=1e-12)


def test_compact_form_equals_entrywise_form():
    """M~ = D_A At^T Bt D_B (Appendix B) equals Eq. (2) entry by entry."""
    A, B = synth.lowrank_plus_noise(200, 9, 11, 3, 0.1, 0.5, seed=5)
    st = smp.sketch(A, B, 16, seed=1)
    DA, DB = smp.rescale_factors(st.At, st.sA), smp.rescale_factors(st.Bt, st.sB)
    full = (DA[:, None] * (st.At.T @ st.Bt)) * DB[None, :]
    rows, cols = np.meshgrid(np.arange(9), np.arange(11), indexing="ij")
    est = smp.estimate(rows.ravel(), cols.ravel(), st.At, st.Bt, st.sA, st.sB)
    np.testing.assert_allclose(est.reshape(9, 11), full, rtol=1e-12)


def test_zero_sketch_gives_zero_estimate():
    At = np.zeros((4, 2))
    At[:, 1] = 1.0
    Bt = np.ones((4, 2))
    est = smp.estimate(np.array([0, 1]), np.array([0, 1]), At, Bt, np.array([1.0, 1.0]), np.array([1.0, 1.0]))
    assert est[0] == 0.0 and est[1] != 0.0


def test_figure_3a_mean_squared_errors(golden_dir):
    """Reproduce the printed MSEs of Figure 3(a): rescaled JL 0.053 vs JL 0.129 (dim 1,000, k = 10)."""
    g = json.load(open(os.path.join(golden_dir, "fig3a_mse.json")))
    d, k, npairs = g["dim"], g["k"], 3000
    rng = np.random.default_rng(12)
    c = rng.uniform(-1.0, 1.0, npairs)
    X = rng.standard_normal((d, npairs))
    X /= np.linalg.norm(X, axis=0)
    Zp = rng.standard_normal((d, npairs))
    Zp -= X * (X * Zp).sum(0)
    Zp /= np.linalg.norm(Zp, axis=0)
    Y = X * c + Zp * np.sqrt(1 - c * c)
    err_jl, err_rs = [], []
    for p in range(npairs):    # an independent Pi per pair, as in the figure's repeated trials
        st = smp.sketch(X[:, p:p + 1], Y[:, p:p + 1], k, seed=1000 + p)
        err_rs.append(smp.estimate([0], [0], st.At, st.Bt, st.sA, st.sB)[0] - c[p])
        err_jl.append(float(st.At[:, 0] @ st.Bt[:, 0]) - c[p])
    mse_rs, mse_jl = np.mean(np.square(err_rs)), np.mean(np.square(err_jl))
    assert abs(mse_rs - g["mse_rescaled_jl"]) < 0.15 * g["mse_rescaled_jl"]
    assert abs(mse_jl - g["mse_jl"]) < 0.12 * g["mse_jl"]
    assert mse_rs < 0.6 * mse_jl


def test_entrywise_jl_bound():
    """|M~_ij - A_i^T B_j| <= eps ||A_i|| ||B_j|| with eps ~ sqrt(log n / k) (Lemma B.6) for nearly all entries."""
    A, B = synth.lowrank_plus_noise(2000, 60, 60, 5, 0.3, 0.5, seed=8)
    k = 400
    st = smp.sketch(A, B, k, seed=9)
    rows, cols = np.meshgrid(np.arange(60), np.arange(60), indexing="ij")
    est = smp.estimate(rows.ravel(), cols.ravel(), st.At, st.Bt, st.sA, st.sB).reshape(60, 60)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    scale = np.outer(np.linalg.norm(A64, axis=0), np.linalg.norm(B64, axis=0))
    dev = np.abs(est - A64.T @ B64) / scale
    eps = 3.0 * math.sqrt(math.log(60) / k)
    assert np.mean(dev <= eps) > 0.999
