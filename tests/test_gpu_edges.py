"""Edge cases of the path against the CPU oracle: degenerate shapes (single columns), ragged row blocks shorter than a
pipeline stage in any order, an all-zero column (reading: its sketch column is zero, so D = 0 and its estimates are
0; Eq. (1) then samples its entries through the other matrix's term only), the CUDA-core engine at the largest
sketch size the C ABI takes (k = 4,096), empty calls, and all-zero inputs (both Frobenius norms zero: an error)."""
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


def _sketch_against_oracle(env, A, B, k, engine, blocks, tol, max_rows=65536):
    torch, smp, pipeline = env
    n1, n2 = A.shape[1], B.shape[1]
    s = pipeline.Solver(n1, n2, k, torch.float32, seed=5, engine=engine, max_rows=max_rows)

    def padded(X):   # rows padded to 16 bytes, as the tensor-core engines require (lda % 4 == 0)
        ld = (X.shape[1] + 3) // 4 * 4
        P = np.zeros((X.shape[0], ld), dtype=np.float32)
        P[:, :X.shape[1]] = X
        return torch.from_numpy(P).cuda()

    Ad, Bd = padded(A), padded(B)
    smp.smp_sketch_reset(s.ctx)
    for r0, r1 in blocks:
        smp.smp_sketch_accumulate(s.ctx, Ad[r0:r1], Ad.stride(0), Bd[r0:r1], Bd.stride(0), r0, r1 - r0)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.SketchState(n1, n2, k, 5)
    for r0, r1 in blocks:
        ref.accumulate(A[r0:r1], B[r0:r1], r0)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < tol
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < tol
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    return s, ref


@pytest.mark.parametrize("engine,tol", [("simt", 1e-5), ("tc", 2e-3), ("tc_bf16", 1e-2)])
def test_single_columns_and_ragged_blocks(env, engine, tol):
    """n1 = n2 = 1 and blocks of 1, 7, 15, 17 and 13 rows (none a whole 16- or 32-row stage), out of order."""
    torch, smp, _ = env
    eng = {"simt": smp.SMP_ENGINE_SIMT, "tc": smp.SMP_ENGINE_TC, "tc_bf16": smp.SMP_ENGINE_TC_BF16}[engine]
    rng = np.random.default_rng(21)
    A = rng.standard_normal((53, 1)).astype(np.float32)
    B = rng.standard_normal((53, 1)).astype(np.float32)
    blocks = [(8, 15), (0, 1), (23, 40), (15, 23), (1, 8), (40, 53)]
    s, _ = _sketch_against_oracle(env, A, B, 24, eng, blocks, tol, max_rows=32)
    s.close()


@pytest.mark.parametrize("engine,tol", [("tc", 2e-3), ("simt", 1e-5)])
def test_zero_column(env, engine, tol):
    """Column 3 of A is all zero: its norm and sketch column are exactly 0, Omega (from the GPU's norms) is bit-exact
    against the oracle's sampler, and every estimate in row 3 is 0 while the others match the oracle's Eq. (2)."""
    torch, smp, _ = env
    eng = {"simt": smp.SMP_ENGINE_SIMT, "tc": smp.SMP_ENGINE_TC}[engine]
    A, B = synth.lowrank_plus_noise(900, 40, 36, 4, 0.1, 0.5, seed=31, dtype=np.float32)
    A[:, 3] = 0.0
    s, ref = _sketch_against_oracle(env, A, B, 48, eng, [(0, 500), (500, 900)], tol, max_rows=512)
    st = s.sketch_state()
    assert float(st["sA"][3]) == 0.0 and not st["At"][3].any()
    m = O.default_m(40, 36, 3)
    nnz = s.sample(m, 7)
    vals = s.estimate(nnz).cpu().numpy().astype(np.float64)
    om = omega_numpy(s)
    rows, cols, _ = O.sample_omega(st["sA"].cpu().numpy(), st["sB"].cpu().numpy(), m, 7)
    np.testing.assert_array_equal(om["col"], cols)
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    ref_vals = O.estimate(rows, cols, ref.At, ref.Bt, ref.sA, ref.sB)
    assert np.all(vals[rows == 3] == 0.0) and np.all(ref_vals[rows == 3] == 0.0)
    scale = np.sqrt(ref.sA[rows] * ref.sB[cols])
    assert float(np.max(np.abs(vals - ref_vals) / np.maximum(scale, 1e-300))) < 10 * tol
    s.close()


def test_simt_largest_sketch(env):
    """k = 4,096, the largest sketch size the C ABI takes, on the CUDA-core engine, against the oracle."""
    torch, smp, _ = env
    A, B = synth.lowrank_plus_noise(700, 24, 20, 4, 0.1, 0.5, seed=41, dtype=np.float32)
    s, _ = _sketch_against_oracle(env, A, B, 4096, smp.SMP_ENGINE_SIMT, [(0, 300), (300, 700)], 1e-5, max_rows=512)
    s.close()


def test_empty_calls_and_all_zero_inputs(env):
    """nrows = 0 is a no-op (the sketch of the other blocks is unchanged); a pass over all-zero inputs finalizes to
    zero norms and sampling it is SMP_EINVAL (both Frobenius norms zero), after which the context is still usable."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(300, 40, 36, 4, 0.1, 0.5, seed=51, dtype=np.float32)
    s = pipeline.Solver(40, 36, 32, torch.float32, seed=5, max_rows=512)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    smp.smp_sketch_reset(s.ctx)
    smp.smp_sketch_accumulate(s.ctx, Ad, 40, Bd, 36, 0, 300)
    smp.smp_sketch_accumulate(s.ctx, Ad, 40, Bd, 36, 300, 0)           # empty: nothing happens
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    ref = O.sketch(A, B, 32, 5, block_rows=300)
    assert _colrel(s.sketch_state()["At"].cpu().numpy().astype(np.float64), ref.At.T) < 2e-3
    Z = torch.zeros(300, 40, device="cuda")
    smp.smp_sketch_reset(s.ctx)
    smp.smp_sketch_accumulate(s.ctx, Z, 40, Z[:, :36].contiguous(), 36, 0, 300)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    assert not st["sA"].any() and not st["sB"].any()
    with pytest.raises(smp.SmpError) as e:
        s.sample(100.0, 2)
    assert e.value.status == smp.SMP_EINVAL
    smp.smp_sketch_reset(s.ctx)
    smp.smp_sketch_accumulate(s.ctx, Ad, 40, Bd, 36, 0, 300)
    smp.smp_sketch_finalize(s.ctx)
    nnz = s.sample(O.default_m(40, 36, 3), 2)
    assert nnz > 0
    s.close()
