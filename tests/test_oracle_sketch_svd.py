"""Pins for the oracle's SVD(A~^T B~) baseline (Section 4, the comparison with the SVD of the sketched product).

The oracle is the plain definition (top-r SVD of the dense product); these tests pin it to a closed form, to the
exact product when Pi = I, to the Eckart-Young residual found by an independent power iteration, and to the
paper's qualitative finding that SMP-PCA beats it on columns drawn from a narrow cone.
"""
import numpy as np

from oracle import smp
from paper_1610_06656_gb300 import synth


def _orth(rng, n, k):
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return Q


def test_closed_form_factors():
    """A~ = diag(s) P^T, B~ = Q^T with orthonormal P, Q: A~^T B~ = P diag(s) Q^T, so the top-r triplets are
    (P_c, s_c, Q_c) up to the sign rule."""
    rng = np.random.default_rng(1)
    n1, n2, k, r = 40, 30, 12, 5
    P, Q = _orth(rng, n1, k), _orth(rng, n2, k)
    s = np.sort(rng.uniform(1.0, 10.0, size=k))[::-1]
    U, S, V = smp.sketch_svd(s[:, None] * P.T, Q.T, r)
    np.testing.assert_allclose(S, s[:r], rtol=1e-13)
    for c in range(r):
        sg = np.sign(U[:, c] @ P[:, c])
        np.testing.assert_allclose(U[:, c], sg * P[:, c], atol=1e-13)
        np.testing.assert_allclose(V[:, c], sg * Q[:, c], atol=1e-13)
        i = int(np.argmax(np.abs(U[:, c])))
        assert U[i, c] > 0


def test_identity_pi_gives_exact_product_svd():
    """Pi = I (k = d): A~ = A, so the baseline is the truncated SVD of A^T B; checked against the eigen
    decomposition of (A^T B)(A^T B)^T (a different LAPACK path)."""
    d, n1, n2, r = 50, 20, 16, 4
    A, B = synth.lowrank_plus_noise(d, n1, n2, 6, 0.05, 0.5, seed=3, dtype=np.float64)
    st = smp.sketch(A, B, d, seed=1, pi=np.eye(d))
    U, S, V = smp.sketch_svd(st.At, st.Bt, r)
    M = A.T @ B
    lam, E = np.linalg.eigh(M @ M.T)
    lam, E = lam[::-1], E[:, ::-1]
    np.testing.assert_allclose(S, np.sqrt(lam[:r]), rtol=1e-10)
    assert np.linalg.norm(U @ U.T - E[:, :r] @ E[:, :r].T, 2) < 1e-9
    np.testing.assert_allclose(V, M.T @ U / S, atol=1e-9)


def test_residual_is_eckart_young():
    """||A~^T B~ - U S V^T||_2 equals sigma_{r+1}, the residual's norm found by plain power iteration."""
    A, B = synth.lowrank_plus_noise(400, 60, 50, 8, 0.1, 0.5, seed=4, dtype=np.float64)
    st = smp.sketch(A, B, 40, seed=7)
    r = 5
    U, S, V = smp.sketch_svd(st.At, st.Bt, r)
    R = st.At.T @ st.Bt - (U * S) @ V.T
    x = np.random.default_rng(0).standard_normal(R.shape[1])
    for _ in range(3000):
        x = R.T @ (R @ x)
        x /= np.linalg.norm(x)
    res = np.linalg.norm(R @ x)
    sig = np.sqrt(np.maximum(np.sort(np.linalg.eigvalsh((st.At.T @ st.Bt).T @ (st.At.T @ st.Bt)))[::-1], 0.0))
    assert abs(res - sig[r]) < 1e-8 * sig[0]
    assert S[-1] >= sig[r] - 1e-9 * sig[0]


def test_smp_pca_beats_sketch_svd_in_a_narrow_cone():
    """Section 4: on unit columns drawn from a cone, the rescaled JL estimate makes SMP-PCA's error smaller than
    SVD(A~^T B~)'s, and the gap grows as the cone narrows."""
    d, n, k, r, T = 1000, 100, 50, 3, 10
    ratios = []
    for theta in (0.5, 0.1):
        A, B = synth.cone(d, n, n, theta, seed=5)
        m = smp.default_m(n, n, r)
        out = smp.smp_pca(A, B, r, k, m, T, seed=1, sample_seed=2)
        M = A.T @ B
        e_smp = smp.spectral_error(M, out["U"], out["S"], out["V"])
        U, S, V = smp.sketch_svd(out["state"].At, out["state"].Bt, r)
        e_svd = smp.spectral_error(M, U, S, V)
        ratios.append(e_svd / e_smp)
    print("error ratios SVD(A~^T B~) / SMP-PCA:", ratios)
    assert ratios[0] > 1.0 and ratios[1] > ratios[0]
