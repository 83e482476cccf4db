"""Parity of the BF16 tensor-core sketch engine (kind::f16, MN-major data operand, k up to 1,024 over two CTAs).

Small integers are exact in BF16 and their products and FP32 sums are exact, so the first tests compare bit for
bit (data layout, the MN-major descriptor, the sketch-row split at k > 512). The Philox tests compare against the
oracle run on the same stored BF16 values: Pi is rounded to BF16 (relative 2^-9), so the sketch columns agree to a
relative 1e-2; the column norms are of the stored values (squares exact in binary32, compensated sums), 1e-12.
"""
import numpy as np
import pytest

from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, csr_rows, omega_numpy, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    return torch, smp, pipeline


def _colrel(X, Y):
    num = np.linalg.norm(X - Y, axis=1)
    den = np.maximum(np.linalg.norm(Y, axis=1), 1e-300)
    return float((num / den).max())


def _bf16(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("k,n1,n2,nrows", [(300, 200, 136, 100), (1024, 256, 128, 64), (40, 40, 72, 16),
                                           (600, 136, 200, 333)])
def test_bf16_exact_on_integers(env, k, n1, n2, nrows):
    torch, smp, pipeline = env
    rng = np.random.default_rng(k + n1)
    A = rng.integers(-8, 9, size=(nrows, n1)).astype(np.float32)
    B = rng.integers(-8, 9, size=(nrows, n2)).astype(np.float32)
    ldp = (nrows + 3) // 4 * 4
    P = np.zeros((k, ldp), dtype=np.float32)
    P[:, :nrows] = rng.integers(-2, 3, size=(k, nrows))
    s = pipeline.Solver(n1, n2, k, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC)
    smp.smp_sketch_accumulate_pi(s.ctx, torch.from_numpy(P).cuda(), ldp, _bf16(torch, A), n1, _bf16(torch, B), n2, 0,
                                 nrows)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    Pi = P[:, :nrows].astype(np.int64)
    np.testing.assert_array_equal(st["At"].cpu().numpy(), (Pi @ A.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["Bt"].cpu().numpy(), (Pi @ B.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["sA"].cpu().numpy(), (A.astype(np.int64) ** 2).sum(0).astype(np.float64))
    np.testing.assert_array_equal(st["sB"].cpu().numpy(), (B.astype(np.int64) ** 2).sum(0).astype(np.float64))
    s.close()


@pytest.mark.parametrize("k", [100, 1024])
def test_bf16_philox_sketch_matches_oracle(env, k):
    """d = 3,000 in 1,000-row blocks out of order, n1 = 200, n2 = 136; the oracle sees the stored BF16 values."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(3000, 200, 136, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    Ab, Bb = _bf16(torch, A), _bf16(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)
    B64 = Bb.float().cpu().numpy().astype(np.float64)
    s = pipeline.Solver(200, 136, k, torch.bfloat16, seed=11, engine=smp.SMP_ENGINE_TC, max_rows=1000)
    s.sketch(Ab, Bb, 1000, order=[2000, 0, 1000])
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A64, B64, k, 11, block_rows=1000)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 1e-2
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 1e-2
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    s.close()


def test_bf16_k1024_matches_oracle(env):
    """The precision form's sketch size k = 1,024 (two CTAs per column tile) on one 2,048-row block, against the
    oracle run on the same stored BF16 values."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2048, 256, 128, 20, 0.05, 0.7, seed=7, dtype=np.float32)
    Ab, Bb = _bf16(torch, A), _bf16(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)
    B64 = Bb.float().cpu().numpy().astype(np.float64)
    s = pipeline.Solver(256, 128, 1024, torch.bfloat16, seed=21, engine=smp.SMP_ENGINE_TC, max_rows=2048)
    s.sketch(Ab, Bb, 2048)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A64, B64, 1024, 21, block_rows=2048)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 1e-2
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 1e-2
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    s.close()


def test_bf16_end_to_end_tiny(env):
    """Tiny workload stored in BF16 through the tensor-core engine: Omega bit-exact against the oracle on the same
    stored values (the norms are exact), spectral error within 3e-3 of the oracle's."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    Ab, Bb = _bf16(torch, A), _bf16(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)
    B64 = Bb.float().cpu().numpy().astype(np.float64)
    s = pipeline.Solver(200, 200, 100, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC)
    m = O.default_m(200, 200, 5)
    out = s.solve(Ab, Bb, 5, 10, m=m, sample_seed=2, walt_seed=3)
    ref = O.smp_pca(A64, B64, 5, 100, m, 10, seed=1, sample_seed=2)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A64.T @ B64
    e_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= 3e-3
    s.close()


def test_bf16_rejects_unaligned_leading_dimension(env):
    torch, smp, pipeline = env
    s = pipeline.Solver(30, 30, 64, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC)
    A = torch.zeros(10, 30, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_accumulate(s.ctx, A, 30, A, 30, 0, 10)
    assert e.value.status == smp.SMP_EUNSUPPORTED
    s.close()
