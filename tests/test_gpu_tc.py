"""Parity of the tensor-core (tcgen05, TF32) sketch engine.

Integer-valued data and Pi make every TF32 product and FP32 sum exact, so the first tests compare bit for bit and
any operand-layout mistake shows up as a mismatch. The Philox tests then compare against the oracle within the
TF32 rounding tolerance (relative 2e-3 per sketch column; column norms stay exact to 1e-13 because they are summed
from the FP32 inputs, not from the TF32 operands).
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


# the last two cases cover 10 and 8 column tiles over both matrices (a ragged tile on each)
@pytest.mark.parametrize("k,n1,n2,nrows", [(300, 200, 132, 100), (512, 256, 128, 64), (40, 36, 68, 16),
                                           (500, 132, 200, 333), (300, 640, 520, 200), (64, 512, 512, 48)])
def test_tc_exact_on_integers(env, k, n1, n2, nrows):
    torch, smp, pipeline = env
    rng = np.random.default_rng(k + n1)
    A = rng.integers(-8, 9, size=(nrows, n1)).astype(np.float32)
    B = rng.integers(-8, 9, size=(nrows, n2)).astype(np.float32)
    ldp = (nrows + 3) // 4 * 4
    P = np.zeros((k, ldp), dtype=np.float32)
    P[:, :nrows] = rng.integers(-2, 3, size=(k, nrows))
    s = pipeline.Solver(n1, n2, k, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC)
    smp.smp_sketch_accumulate_pi(s.ctx, torch.from_numpy(P).cuda(), ldp, torch.from_numpy(A).cuda(), n1,
                                 torch.from_numpy(B).cuda(), n2, 0, nrows)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    Pi = P[:, :nrows].astype(np.int64)
    np.testing.assert_array_equal(st["At"].cpu().numpy(), (Pi @ A.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["Bt"].cpu().numpy(), (Pi @ B.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["sA"].cpu().numpy(), (A.astype(np.int64) ** 2).sum(0).astype(np.float64))
    np.testing.assert_array_equal(st["sB"].cpu().numpy(), (B.astype(np.int64) ** 2).sum(0).astype(np.float64))
    s.close()


def test_tc_identity_pi(env):
    torch, smp, pipeline = env
    d, n1 = 64, 96
    rng = np.random.default_rng(3)
    A = rng.integers(-100, 101, size=(d, n1)).astype(np.float32)
    s = pipeline.Solver(n1, n1, d, torch.float32, seed=1, same_ab=True, engine=smp.SMP_ENGINE_TC)
    eye = torch.eye(d, dtype=torch.float32, device="cuda")
    smp.smp_sketch_accumulate_pi(s.ctx, eye, d, torch.from_numpy(A).cuda(), n1, None, 0, 0, d)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    np.testing.assert_array_equal(s.sketch_state()["At"].cpu().numpy(), A.T)
    s.close()


@pytest.mark.parametrize("same_ab", [False, True])
def test_tc_philox_sketch_matches_oracle(env, same_ab):
    """d = 2,000 in 700-row blocks (ragged), n1 = 200, n2 = 172, k = 100: Philox Pi generated by the tensor-core
    engine's Pi kernel, compared with the oracle's binary64 sketch."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 172, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    if same_ab:
        B = A
    n2 = 200 if same_ab else 172
    s = pipeline.Solver(200, n2, 100, torch.float32, seed=11, same_ab=same_ab, engine=smp.SMP_ENGINE_TC)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(B)).cuda(), 700,
             order=[1400, 0, 700])
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A, B, 100, 11, block_rows=700, same_ab=same_ab)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 2e-3
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 2e-3
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-13)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-13)
    s.close()


def test_tc_k500_matches_oracle(env):
    """The bench's sketch size k = 500 (two MMA boxes, 512 TMEM columns) on one 4,000-row block with ragged column
    tiles (n1 = 300, n2 = 260), against the oracle's binary64 sketch."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(4000, 300, 260, 20, 0.1, 0.5, seed=5, dtype=np.float32)
    s = pipeline.Solver(300, 260, 500, torch.float32, seed=21, engine=smp.SMP_ENGINE_TC, max_rows=4000)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 4000)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A, B, 500, 21, block_rows=4000)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 2e-3
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 2e-3
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    s.close()


def test_tc_end_to_end_tiny(env):
    """Tiny workload through the tensor-core engine: Omega bit-exact against the oracle (the norms are exact),
    spectral error within 1e-3 of the oracle's."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    s = pipeline.Solver(200, 200, 100, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC)
    m = O.default_m(200, 200, 5)
    out = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5, 10, m=m, sample_seed=2, walt_seed=3)
    ref = O.smp_pca(A, B, 5, 100, m, 10, seed=1, sample_seed=2)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A.astype(np.float64).T @ B.astype(np.float64)
    e_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= 1e-3
    s.close()


def test_tc_rejects_unaligned_leading_dimension(env):
    torch, smp, pipeline = env
    s = pipeline.Solver(30, 30, 64, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC)
    A = torch.zeros(10, 31, device="cuda")
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_accumulate(s.ctx, A, 31, A, 31, 0, 10)
    assert e.value.status == smp.SMP_EUNSUPPORTED
    s.close()
