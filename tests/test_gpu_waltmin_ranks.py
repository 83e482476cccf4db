"""WAltMin (Algorithm 2) at the ranks above 12 the batched, serving and precision forms use (r up to 20) and up to
the C ABI's limit (r = 32), against the oracle: the half-steps of these ranks run on other kernels than r <= 12
(the two-pass lane Gram for r <= 20, the shuffle Gram above, one warp per output row for the binary64 solves), and
the subspace iteration's block order 2 r + 8 exceeds 32 (the four-warp Cholesky and the register substitution for
orders up to 48 and 72). Sizes: n1 = 200, n2 = 170 columns, k = 100, Omega from the sampler of Eq. (1) at
m = 4 n r ln n (near full sampling at these n)."""
import numpy as np
import pytest

from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, csr_rows, omega_numpy, torch_cuda

pytestmark = pytest.mark.gpu

D, N1, N2, K = 2000, 200, 170, 100


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    A, B = synth.lowrank_plus_noise(D, N1, N2, 32, 0.1, 0.5, seed=1200, dtype=np.float32)
    ref = O.sketch(A, B, K, 41, block_rows=700)
    return torch, smp, pipeline, ref


def _setup(env, r):
    torch, smp, pipeline, ref = env
    s = pipeline.Solver(N1, N2, K, torch.float32, seed=41)
    At32 = np.ascontiguousarray(ref.At.T.astype(np.float32))
    Bt32 = np.ascontiguousarray(ref.Bt.T.astype(np.float32))
    smp.smp_sketch_import(s.ctx, torch.from_numpy(At32).cuda(), torch.from_numpy(Bt32).cuda(),
                          torch.from_numpy(ref.sA).cuda(), torch.from_numpy(ref.sB).cuda())
    m = O.default_m(N1, N2, r)
    nnz = s.sample(m, seed=6)
    rows, cols, qh = O.sample_omega(ref.sA, ref.sB, m, 6)
    om = omega_numpy(s)
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    np.testing.assert_array_equal(om["col"], cols)
    vals32 = O.estimate(rows, cols, At32.T.astype(np.float64), Bt32.T.astype(np.float64), ref.sA,
                        ref.sB).astype(np.float32)
    assert nnz == len(rows)
    return s, rows, cols, qh, vals32


def _product(U, S, V):
    return (U * S) @ V.T


@pytest.mark.parametrize("r", [13, 20, 28])
@pytest.mark.parametrize("fp64", [False, True])
def test_waltmin_from_given_init(env, r, fp64):
    """T = 4 rounds from the same orthonormal U0 (the half-steps alone), binary32 or binary64 Gram / iterates."""
    torch, smp, pipeline, ref = env
    s, rows, cols, qh, vals32 = _setup(env, r)
    U0 = np.linalg.qr(np.random.default_rng(r).standard_normal((N1, r)))[0]
    flags = smp.SMP_INIT_GIVEN | (smp.SMP_FP64_ALS if fp64 else 0)
    U, S, V = s.waltmin(torch.from_numpy(vals32).cuda(), r, 4, flags, seed=9, U_init=torch.from_numpy(U0).cuda())
    Uh, Vh = O.waltmin(N1, N2, rows, cols, vals32.astype(np.float64), qh, r, 4, ref.sA, U_init=U0)
    Uo, So, Vo = O.canonical(Uh, Vh)
    P, Po = _product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()), _product(Uo, So, Vo)
    tol = 1e-9 if fp64 else 5e-4
    assert np.linalg.norm(P - Po) <= tol * np.linalg.norm(Po)
    Ug = U.cpu().numpy()
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(r), atol=1e-10)
    s.close()


@pytest.mark.parametrize("r", [20, 28])
def test_waltmin_with_subspace_init_fp64(env, r):
    """The whole of Algorithm 2 with the GPU's subspace-iteration initial SVD (block order 48 and 64) against the
    oracle's LAPACK initial iterate, binary64 iterates."""
    torch, smp, pipeline, ref = env
    s, rows, cols, qh, vals32 = _setup(env, r)
    U, S, V = s.waltmin(torch.from_numpy(vals32).cuda(), r, 6, smp.SMP_FP64_ALS, seed=9)
    Uh, Vh = O.waltmin(N1, N2, rows, cols, vals32.astype(np.float64), qh, r, 6, ref.sA)
    Uo, So, Vo = O.canonical(Uh, Vh)
    P, Po = _product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()), _product(Uo, So, Vo)
    assert np.linalg.norm(P - Po) <= 1e-6 * np.linalg.norm(Po)
    s.close()


def test_waltmin_rank_above_data_rank_fp64(env):
    """r = 28 on data of latent rank 24: the normal equations of the noise directions are nearly singular, which the
    binary64 Gram (SMP_FP64_ALS) still solves; the factors match the oracle's."""
    torch, smp, pipeline, _ = env
    A, B = synth.lowrank_plus_noise(D, N1, N2, 24, 0.1, 0.5, seed=1201, dtype=np.float32)
    ref = O.sketch(A, B, K, 43, block_rows=700)
    s, rows, cols, qh, vals32 = _setup((torch, smp, pipeline, ref), 28)
    U0 = np.linalg.qr(np.random.default_rng(5).standard_normal((N1, 28)))[0]
    flags = smp.SMP_INIT_GIVEN | smp.SMP_FP64_ALS
    U, S, V = s.waltmin(torch.from_numpy(vals32).cuda(), 28, 4, flags, seed=9, U_init=torch.from_numpy(U0).cuda())
    Uh, Vh = O.waltmin(N1, N2, rows, cols, vals32.astype(np.float64), qh, 28, 4, ref.sA, U_init=U0)
    Uo, So, Vo = O.canonical(Uh, Vh)
    P, Po = _product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()), _product(Uo, So, Vo)
    assert np.linalg.norm(P - Po) <= 1e-8 * np.linalg.norm(Po)
    s.close()
