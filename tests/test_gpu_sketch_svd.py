"""Parity of the baseline SVD(A~^T B~) (smp_sketch_svd, block power iteration on the sketched product) with the
oracle's definition (the top-r SVD of the dense product in binary64).

The sketches the GPU iterates on come from the oracle through smp_sketch_import (rounded to binary32 for a binary32
context), so the comparison isolates the iteration. Binary32 products and a Ritz-vector stopping test of 2e-5 give
singular values within 1e-5 relative and the spectral error within 1e-5; binary64 contexts 1e-10.
"""
import numpy as np
import pytest

from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    return torch, smp, pipeline


def _import(torch, smp, s, At, Bt, sA, sB, dt):
    """At, Bt: oracle sketches (k x n); the context takes n x k rows."""
    a = torch.from_numpy(np.ascontiguousarray(At.T.astype(dt))).cuda()
    b = torch.from_numpy(np.ascontiguousarray(Bt.T.astype(dt))).cuda()
    smp.smp_sketch_import(s.ctx, a, b, torch.from_numpy(sA).cuda(), torch.from_numpy(sB).cuda())


def _proj_dist(U1, U2):
    return float(np.linalg.norm(U1 @ U1.T - U2 @ U2.T, 2))


def test_closed_form(env):
    """A~ = diag(s) P^T, B~ = Q^T (P, Q orthonormal): the triplets are (P_c, s_c, Q_c)."""
    torch, smp, pipeline = env
    rng = np.random.default_rng(2)
    n1, n2, k, r = 300, 200, 40, 6
    P, _ = np.linalg.qr(rng.standard_normal((n1, k)))
    Q, _ = np.linalg.qr(rng.standard_normal((n2, k)))
    sv = np.linspace(10.0, 1.0, k)
    s = pipeline.Solver(n1, n2, k, torch.float32, seed=1)
    _import(torch, smp, s, sv[:, None] * P.T, Q.T, np.ones(n1), np.ones(n2), np.float32)
    U, S, V = (x.cpu().numpy() for x in s.sketch_svd(r, seed=9))
    np.testing.assert_allclose(S, sv[:r], rtol=1e-5)
    Ur, Sr, Vr = O.sketch_svd(sv[:, None] * P.T, Q.T, r)
    np.testing.assert_allclose(U, Ur, atol=2e-5)
    np.testing.assert_allclose(V, Vr, atol=2e-5)
    s.close()


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-10)])
def test_matches_oracle_on_synthetic_sketches(env, dtype, tol):
    """Tiny workload shape (d = 2,000, n = 200, k = 100, r = 5): oracle sketches imported, baseline on the GPU
    against the oracle's."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float64)
    ref = O.sketch(A, B, 100, 1)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    s = pipeline.Solver(200, 200, 100, tdt, seed=1)
    npdt = np.float32 if dtype == "f32" else np.float64
    At = ref.At.astype(npdt).astype(np.float64)
    Bt = ref.Bt.astype(npdt).astype(np.float64)
    _import(torch, smp, s, At, Bt, ref.sA, ref.sB, npdt)
    r = 5
    U, S, V = (x.cpu().numpy() for x in s.sketch_svd(r, seed=4))
    Ur, Sr, Vr = O.sketch_svd(At, Bt, r)
    np.testing.assert_allclose(S, Sr, rtol=tol)
    M = A.T @ B
    e_gpu = O.spectral_error(M, U, S, V)
    e_ref = O.spectral_error(M, Ur, Sr, Vr)
    assert abs(e_gpu - e_ref) <= tol * max(1.0, e_ref)
    full = np.linalg.svd(At.T @ Bt, compute_uv=False)
    gap = full[r - 1] / full[r]
    if gap > 1.05:
        assert _proj_dist(U, Ur) < 50 * tol / (gap - 1)
        assert _proj_dist(V, Vr) < 50 * tol / (gap - 1)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-5 if dtype == "f32" else 1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-5 if dtype == "f32" else 1e-12)
    s.close()


def test_same_ab_and_wide_k(env):
    """A = B (one sketch) with k = 700 > the 512-row sketch tile and r = 20 (block of 48 columns)."""
    torch, smp, pipeline = env
    A, _ = synth.lowrank_plus_noise(1500, 260, 260, 30, 0.1, 0.5, seed=1003, dtype=np.float64)
    ref = O.sketch(A, None, 700, 3, same_ab=True)
    s = pipeline.Solver(260, 260, 700, torch.float32, seed=3, same_ab=True)
    At = ref.At.astype(np.float32).astype(np.float64)
    a = torch.from_numpy(np.ascontiguousarray(At.T.astype(np.float32))).cuda()
    smp.smp_sketch_import(s.ctx, a, a, torch.from_numpy(ref.sA).cuda(), torch.from_numpy(ref.sA).cuda())
    r = 20
    U, S, V = (x.cpu().numpy() for x in s.sketch_svd(r, seed=4))
    Ur, Sr, Vr = O.sketch_svd(At, At, r)
    np.testing.assert_allclose(S, Sr, rtol=1e-5)
    M = A.T @ A
    assert abs(O.spectral_error(M, U, S, V) - O.spectral_error(M, Ur, Sr, Vr)) < 1e-5
    s.close()


def test_end_to_end_against_smp_pca(env):
    """Cone data (half-angle 0.1): the GPU's SMP-PCA beats the GPU's SVD(A~^T B~) by a wide margin, as in the
    paper's comparison, and the baseline's error matches the oracle's on the same data."""
    torch, smp, pipeline = env
    A, B = synth.cone(1000, 100, 100, 0.1, seed=5)
    s = pipeline.Solver(100, 100, 50, torch.float64, seed=1)
    r = 3
    m = O.default_m(100, 100, r)
    out = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), r, 10, m=m, sample_seed=2, walt_seed=3)
    U, S, V = (x.cpu().numpy() for x in s.sketch_svd(r, seed=4))
    M = A.T @ B
    e_smp = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_svd = O.spectral_error(M, U, S, V)
    ref = O.sketch(A, B, 50, 1)
    Ur, Sr, Vr = O.sketch_svd(ref.At, ref.Bt, r)
    assert abs(e_svd - O.spectral_error(M, Ur, Sr, Vr)) < 1e-6
    assert e_svd > 10 * e_smp
    s.close()


def test_state_and_argument_errors(env):
    torch, smp, pipeline = env
    s = pipeline.Solver(50, 40, 16, torch.float32, seed=1)
    with pytest.raises(smp.SmpError) as e:
        s.sketch_svd(3)
    assert e.value.status == smp.SMP_ESTATE
    z = torch.zeros(16, 50, device="cuda")
    smp.smp_sketch_import(s.ctx, torch.zeros(50, 16, device="cuda"), torch.zeros(40, 16, device="cuda"),
                          torch.ones(50, dtype=torch.float64, device="cuda"),
                          torch.ones(40, dtype=torch.float64, device="cuda"))
    with pytest.raises(smp.SmpError) as e:
        s.sketch_svd(17)
    assert e.value.status == smp.SMP_EINVAL
    del z
    s.close()
