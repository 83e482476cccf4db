"""Parity of the FP8 E4M3 tensor-core sketch engine (kind::f8f6f4 from BF16 row blocks, one power-of-two scale per
block and matrix, FP32 accumulation).

Integers up to 15 in magnitude keep at most four significant bits, so they and their power-of-two multiples are
exact in E4M3, and the first tests compare bit for bit (conversion, the MN-major E4M3 atom layout, the scales, the
k > 512 split). The quantised-model test rebuilds what the engine computes from the oracle's Pi and the stored BF16
values rounded to E4M3 on the host (torch's CPU float8_e4m3fn, round to nearest even): At = s_A e4m3(sqrt(k) Pi)
e4m3(A / s_A) / sqrt(k), which the kernel must reproduce up to FP32 summation order and the rare element whose
FP32 and FP64 normals round to different E4M3 values. Against the exact oracle the E4M3 rounding of both operands
(3 mantissa bits) leaves a few per cent per sketch column.
"""
import numpy as np
import pytest

from oracle import philox as P
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


def _e4m3(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.float8_e4m3fn).float().numpy() \
        .astype(np.float64)


def _scale(X):
    """2^ceil(log2(max|X| / 448)), 1 for an all-zero block."""
    amax = float(np.abs(X).max()) if X.size else 0.0
    if amax == 0.0:
        return 1.0
    m, e = np.frexp(amax / 448.0)
    return float(np.ldexp(1.0, int(e) - 1 if m == 0.5 else int(e)))


@pytest.mark.parametrize("k,n1,n2,nrows,amp", [(300, 200, 136, 100, 8), (1024, 256, 128, 64, 15),
                                               (40, 40, 72, 16, 3), (600, 136, 200, 333, 12)])
def test_fp8_exact_on_integers(env, k, n1, n2, nrows, amp):
    torch, smp, pipeline = env
    rng = np.random.default_rng(k + n1)
    A = rng.integers(-amp, amp + 1, size=(nrows, n1)).astype(np.float32)
    B = rng.integers(-amp, amp + 1, size=(nrows, n2)).astype(np.float32)
    ldp = (nrows + 3) // 4 * 4
    Pm = np.zeros((k, ldp), dtype=np.float32)
    Pm[:, :nrows] = rng.integers(-2, 3, size=(k, nrows))
    s = pipeline.Solver(n1, n2, k, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC_FP8)
    smp.smp_sketch_accumulate_pi(s.ctx, torch.from_numpy(Pm).cuda(), ldp, _bf16(torch, A), n1, _bf16(torch, B), n2,
                                 0, nrows)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    Pi = Pm[:, :nrows].astype(np.int64)
    np.testing.assert_array_equal(st["At"].cpu().numpy(), (Pi @ A.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["Bt"].cpu().numpy(), (Pi @ B.astype(np.int64)).T.astype(np.float32))
    np.testing.assert_array_equal(st["sA"].cpu().numpy(), (A.astype(np.int64) ** 2).sum(0).astype(np.float64))
    np.testing.assert_array_equal(st["sB"].cpu().numpy(), (B.astype(np.int64) ** 2).sum(0).astype(np.float64))
    s.close()


def test_fp8_scales_follow_each_block(env):
    """Blocks of very different magnitude (2^-12 and 2^5 times small integers), each after a reset: each gets its
    own scale (a stale one would flush the small block to zero or saturate the large one), so all stay exact."""
    torch, smp, pipeline = env
    rng = np.random.default_rng(5)
    n1, n2, k, nrows = 136, 72, 96, 128
    s = pipeline.Solver(n1, n2, k, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC_FP8, max_rows=nrows)
    for mag in (2.0 ** -12, 2.0 ** 5, 2.0 ** -12):
        A = (rng.integers(-7, 8, size=(nrows, n1)) * mag).astype(np.float32)
        B = (rng.integers(-7, 8, size=(nrows, n2)) * mag).astype(np.float32)
        Pm = rng.integers(-2, 3, size=(k, nrows)).astype(np.float32)
        smp.smp_sketch_reset(s.ctx)
        smp.smp_sketch_accumulate_pi(s.ctx, torch.from_numpy(Pm).cuda(), nrows, _bf16(torch, A), n1,
                                     _bf16(torch, B), n2, 0, nrows)
        smp.smp_sketch_finalize(s.ctx)
        smp.smp_sync(s.ctx)
        st = s.sketch_state()
        np.testing.assert_array_equal(st["At"].cpu().numpy(), (Pm.astype(np.float64) @ A).T.astype(np.float32))
        np.testing.assert_array_equal(st["Bt"].cpu().numpy(), (Pm.astype(np.float64) @ B).T.astype(np.float32))
    s.close()


@pytest.mark.parametrize("k", [100, 700])
def test_fp8_matches_quantised_model(env, k):
    """d = 3,000 in 1,000-row blocks (out of order), n1 = 200, n2 = 136, Philox Pi."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(3000, 200, 136, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    Ab, Bb = _bf16(torch, A), _bf16(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)
    B64 = Bb.float().cpu().numpy().astype(np.float64)
    s = pipeline.Solver(200, 136, k, torch.bfloat16, seed=11, engine=smp.SMP_ENGINE_TC_FP8, max_rows=1000)
    s.sketch(Ab, Bb, 1000, order=[2000, 0, 1000])
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    At = np.zeros((k, 200))
    Bt = np.zeros((k, 136))
    for r0 in (0, 1000, 2000):
        Pq = _e4m3(torch, P.pi_block(11, k, r0, 1000) * np.sqrt(k))
        a, b = A64[r0:r0 + 1000], B64[r0:r0 + 1000]
        sa, sb = _scale(a), _scale(b)
        At += sa * (Pq @ _e4m3(torch, a / sa)) / np.sqrt(k)
        Bt += sb * (Pq @ _e4m3(torch, b / sb)) / np.sqrt(k)
    gA = st["At"].cpu().numpy().astype(np.float64)
    gB = st["Bt"].cpu().numpy().astype(np.float64)
    assert _colrel(gA, At.T) < 2e-3
    assert _colrel(gB, Bt.T) < 2e-3
    ref = O.sketch(A64, B64, k, 11, block_rows=1000)
    assert _colrel(gA, ref.At.T) < 8e-2
    assert _colrel(gB, ref.Bt.T) < 8e-2
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    s.close()


def test_fp8_same_ab(env):
    """A = B: one set of column tiles, the second scale unused."""
    torch, smp, pipeline = env
    rng = np.random.default_rng(9)
    n, k, nrows = 200, 64, 96
    A = rng.integers(-9, 10, size=(nrows, n)).astype(np.float32)
    Pm = rng.integers(-2, 3, size=(k, nrows)).astype(np.float32)
    s = pipeline.Solver(n, n, k, torch.bfloat16, seed=1, same_ab=True, engine=smp.SMP_ENGINE_TC_FP8)
    Ab = _bf16(torch, A)
    smp.smp_sketch_accumulate_pi(s.ctx, torch.from_numpy(Pm).cuda(), nrows, Ab, n, Ab, n, 0, nrows)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    np.testing.assert_array_equal(st["At"].cpu().numpy(),
                                  (Pm.astype(np.int64) @ A.astype(np.int64)).T.astype(np.float32))
    s.close()


def test_fp8_end_to_end_tiny(env):
    """Tiny workload through the FP8 engine: Omega bit-exact against the oracle on the same stored BF16 values (the
    norms come from the BF16 values, exactly); the spectral error stays within 2e-2 of the oracle's."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    Ab, Bb = _bf16(torch, A), _bf16(torch, B)
    A64 = Ab.float().cpu().numpy().astype(np.float64)
    B64 = Bb.float().cpu().numpy().astype(np.float64)
    s = pipeline.Solver(200, 200, 100, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_TC_FP8)
    m = O.default_m(200, 200, 5)
    out = s.solve(Ab, Bb, 5, 10, m=m, sample_seed=2, walt_seed=3)
    ref = O.smp_pca(A64, B64, 5, 100, m, 10, seed=1, sample_seed=2)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A64.T @ B64
    e_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= 2e-2, (e_gpu, e_ref)
    s.close()


def test_fp8_rejects_f32_contexts(env):
    torch, smp, pipeline = env
    with pytest.raises(smp.SmpError) as e:
        pipeline.Solver(30, 30, 64, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC_FP8)
    assert e.value.status == smp.SMP_EUNSUPPORTED
