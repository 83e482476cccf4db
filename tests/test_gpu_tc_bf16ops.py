"""Parity of SMP_ENGINE_TC_BF16: binary32 row blocks sketched on tcgen05 with BF16 operands (the inputs rounded to
BF16 on their way to the tensor cores, Pi generated in BF16, FP32 accumulation).

Small integers are exact in BF16 and their products and sums exact in binary32, so the first tests compare bit for
bit; any slip in the 32-row stage layout or the kind::f16 descriptors shows up as a mismatch. Against the oracle:
both operands carry a 2^-9 rounding, so sketch columns agree within 1e-2 relative (the BF16 engine's bound), the
column norms exactly as for the TF32 engine (they are summed from the binary32 inputs), and the end-to-end
spectral error within 3e-3 of the oracle's.
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


# the last case covers 10 column tiles over both matrices (a ragged tile on each)
@pytest.mark.parametrize("k,n1,n2,nrows", [(300, 200, 132, 100), (512, 256, 128, 64), (40, 36, 68, 16),
                                           (500, 132, 200, 333), (300, 640, 520, 200)])
def test_exact_on_integers(env, k, n1, n2, nrows):
    torch, smp, pipeline = env
    rng = np.random.default_rng(k + n1 + 7)
    A = rng.integers(-8, 9, size=(nrows, n1)).astype(np.float32)
    B = rng.integers(-8, 9, size=(nrows, n2)).astype(np.float32)
    ldp = (nrows + 3) // 4 * 4
    P = np.zeros((k, ldp), dtype=np.float32)
    P[:, :nrows] = rng.integers(-2, 3, size=(k, nrows))
    s = pipeline.Solver(n1, n2, k, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC_BF16)
    smp.smp_sketch_accumulate_pi(s.ctx, torch.from_numpy(P).cuda(), ldp, torch.from_numpy(A).cuda(), n1,
                                 torch.from_numpy(B).cuda(), n2, 0, nrows)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    Pi = P[:, :nrows].astype(np.int64)
    np.testing.assert_array_equal(st["At"].cpu().numpy(), (Pi @ A.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["Bt"].cpu().numpy(), (Pi @ B.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["sA"].cpu().numpy(), (A.astype(np.int64) ** 2).sum(0).astype(np.float64))
    s.close()


def test_identity_pi_multi_block(env):
    """Pi = I over three 64-row blocks (any order): At = A bit for bit for integers |x| <= 100 (exact in BF16)."""
    torch, smp, pipeline = env
    d, n1 = 192, 96
    rng = np.random.default_rng(4)
    A = rng.integers(-100, 101, size=(d, n1)).astype(np.float32)
    s = pipeline.Solver(n1, n1, d, torch.float32, seed=1, same_ab=True, engine=smp.SMP_ENGINE_TC_BF16, max_rows=64)
    eye = torch.eye(d, dtype=torch.float32, device="cuda")
    Ad = torch.from_numpy(A).cuda()
    for r0 in (128, 0, 64):
        smp.smp_sketch_accumulate_pi(s.ctx, eye[:, r0:].contiguous(), d - r0, Ad[r0:r0 + 64], n1, None, 0, r0, 64)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    np.testing.assert_array_equal(s.sketch_state()["At"].cpu().numpy(), A.T)
    s.close()


@pytest.mark.parametrize("same_ab", [False, True])
def test_philox_sketch_matches_oracle(env, same_ab):
    """d = 2,000 in 700-row blocks (ragged, out of order), n1 = 200, n2 = 172, k = 100."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 172, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    if same_ab:
        B = A
    n2 = 200 if same_ab else 172
    s = pipeline.Solver(200, n2, 100, torch.float32, seed=11, same_ab=same_ab, engine=smp.SMP_ENGINE_TC_BF16)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(B)).cuda(), 700,
             order=[1400, 0, 700])
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A, B, 100, 11, block_rows=700, same_ab=same_ab)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 1e-2
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 1e-2
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-13)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-13)
    s.close()


def test_k500_matches_oracle(env):
    """The scale workload's k = 500 (two MMA boxes) on one 4,000-row block with ragged column tiles, against the
    oracle's binary64 sketch (BF16 rounding of both operands: 1e-2 per column)."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(4000, 300, 260, 20, 0.1, 0.5, seed=5, dtype=np.float32)
    s = pipeline.Solver(300, 260, 500, torch.float32, seed=21, engine=smp.SMP_ENGINE_TC_BF16, max_rows=4000)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 4000)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A, B, 500, 21, block_rows=4000)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 1e-2
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 1e-2
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    s.close()


def test_end_to_end_tiny(env):
    """Tiny workload: Omega bit-exact against the oracle (exact norms), spectral error within 3e-3 of the oracle's."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    s = pipeline.Solver(200, 200, 100, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC_BF16)
    m = O.default_m(200, 200, 5)
    out = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5, 10, m=m, sample_seed=2, walt_seed=3)
    ref = O.smp_pca(A, B, 5, 100, m, 10, seed=1, sample_seed=2)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A.astype(np.float64).T @ B.astype(np.float64)
    e_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= 3e-3
    s.close()


def test_engine_argument_checks(env):
    torch, smp, pipeline = env
    with pytest.raises(smp.SmpError) as e:
        pipeline.Solver(64, 64, 16, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC_BF16)
    assert e.value.status == smp.SMP_EUNSUPPORTED
    s = pipeline.Solver(64, 64, 600, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC_BF16)
    A = torch.zeros(32, 64, device="cuda")
    with pytest.raises(smp.SmpError) as e:   # k > 512
        smp.smp_sketch_accumulate(s.ctx, A, 64, A, 64, 0, 32)
    assert e.value.status == smp.SMP_EUNSUPPORTED
    s.close()
