"""Parity of LELA's two passes (smp_norms_accumulate, smp_exact_accumulate / smp_exact_values) and of LELA end to
end with the oracle (Section 4, Table 1's two-pass comparison method).

Exact entries on tensor cores: both operands are rounded to TF32 (2^-11 relative each) and summed in binary32
within a block, so |error| <= (2^-10 + rows * 2^-23) sum_t |A_ti B_tj| (rows: the block's row count); the CUDA-core
path in binary64 is held to 1e-12 of the same sum, in binary32 to rows * 2^-23 of it. Sizes span several tiles with
ragged tails: n1 = 700 (two 512-column chunks of A), n2 = 300 (three 128-column tiles of B), d = 5,000 rows in
2,048-row blocks (a 904-row last block).
"""
import numpy as np
import pytest

from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, csr_rows, omega_numpy, torch_cuda

pytestmark = pytest.mark.gpu

D, N1, N2, BLOCK = 5000, 700, 300, 2048


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    return torch, smp, pipeline


@pytest.fixture(scope="module")
def data():
    return synth.lowrank_plus_noise(D, N1, N2, 10, 0.1, 0.5, seed=77, dtype=np.float32)


def _abs_sums(A, B, rows, cols):
    """sum_t |A[t, i] B[t, j]| per entry (the scale of the rounding bounds)."""
    Aa, Ba = np.abs(A.astype(np.float64)), np.abs(B.astype(np.float64))
    return np.einsum("te,te->e", Aa[:, rows], Ba[:, cols])


def _lela_gpu(torch, s, A, B, m, sample_seed, block):
    Ad = torch.from_numpy(A).cuda()
    Bd = None if B is None else torch.from_numpy(B).cuda()
    s.norms(Ad, Bd, block)
    nnz = s.sample(m, seed=sample_seed)
    vals = s.exact(Ad, Bd, block)
    return nnz, vals.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype_name", ["f32", "bf16", "f64"])
def test_norms_pass_matches_oracle(env, data, dtype_name):
    """Pass 1 (norms only) equals the oracle's column norms of the same inputs (compensated sums)."""
    torch, smp, pipeline = env
    A, B = data
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[dtype_name]
    Ad = torch.from_numpy(A).to(tdt).cuda()
    Bd = torch.from_numpy(B).to(tdt).cuda()
    s = pipeline.Solver(N1, N2, 16, tdt, seed=1)
    s.norms(Ad, Bd, BLOCK)
    st = s.sketch_state()
    sA, sB = O.column_norms_sq(Ad.double().cpu().numpy(), Bd.double().cpu().numpy())
    np.testing.assert_allclose(st["sA"].cpu().numpy(), sA, rtol=1e-11)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), sB, rtol=1e-11)
    assert abs(st["F"][0] - O.frobenius_sq(sA)) <= 1e-11 * st["F"][0]
    s.close()


@pytest.mark.parametrize("engine", ["tc", "simt"])
def test_exact_entries_f32(env, data, engine):
    """Exact entries over the GPU's Omega against the oracle's definition, tensor-core and CUDA-core paths."""
    torch, smp, pipeline = env
    A, B = data
    eng = smp.SMP_ENGINE_TC if engine == "tc" else smp.SMP_ENGINE_SIMT
    s = pipeline.Solver(N1, N2, 16, torch.float32, seed=1, engine=eng, max_rows=BLOCK)
    m = O.default_m(N1, N2, 8)
    nnz, vals = _lela_gpu(torch, s, A, B, m, 5, BLOCK)
    om = omega_numpy(s)
    rows, cols = csr_rows(om["row_ptr"]), om["col"]
    assert nnz == rows.shape[0] > 0
    want = O.exact_entries(rows, cols, A, B)
    scale = _abs_sums(A, B, rows, cols)
    bound = (2.0 ** -10 + BLOCK * 2.0 ** -23) if engine == "tc" else BLOCK * 2.0 ** -23
    assert np.all(np.abs(vals - want) <= bound * scale)
    assert np.linalg.norm(vals - want) <= 1e-3 * np.linalg.norm(want)
    assert smp.smp_exact_coverage(s.ctx) == (D, D, 1)
    s.close()


def test_exact_entries_f64_simt(env, data):
    torch, smp, pipeline = env
    A, B = data
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    s = pipeline.Solver(N1, N2, 16, torch.float64, seed=1, max_rows=BLOCK)
    nnz, vals = _lela_gpu(torch, s, A64, B64, O.default_m(N1, N2, 8), 5, BLOCK)
    om = omega_numpy(s)
    rows, cols = csr_rows(om["row_ptr"]), om["col"]
    want = O.exact_entries(rows, cols, A64, B64)
    assert np.all(np.abs(vals - want) <= 1e-12 * _abs_sums(A64, B64, rows, cols))
    s.close()


def test_exact_entries_unaligned_rows_take_the_cuda_core_path(env, data):
    """lda = n1 + 1 = 299 (not a multiple of 4): SMP_ENGINE_AUTO runs the CUDA-core path, SMP_ENGINE_TC refuses."""
    torch, smp, pipeline = env
    A, B = data
    n1 = 298
    Apad = torch.zeros(D, n1 + 1, dtype=torch.float32)
    Apad[:, :n1] = torch.from_numpy(A[:, :n1])
    Ad, Bd = Apad.cuda(), torch.from_numpy(B).cuda()
    s = pipeline.Solver(n1, N2, 16, torch.float32, seed=1, max_rows=BLOCK)
    for r0 in range(0, D, BLOCK):
        r1 = min(D, r0 + BLOCK)
        smp.smp_norms_accumulate(s.ctx, Ad[r0:r1], n1 + 1, Bd[r0:r1], N2, r0, r1 - r0)
    smp.smp_sketch_finalize(s.ctx)
    nnz = s.sample(O.default_m(n1, N2, 5), seed=3)
    for r0 in range(0, D, BLOCK):
        r1 = min(D, r0 + BLOCK)
        smp.smp_exact_accumulate(s.ctx, Ad[r0:r1], n1 + 1, Bd[r0:r1], N2, r0, r1 - r0)
    vals = torch.empty(nnz, device="cuda")
    smp.smp_exact_values(s.ctx, vals)
    om = omega_numpy(s)
    rows, cols = csr_rows(om["row_ptr"]), om["col"]
    Ah = A[:, :n1]
    want = O.exact_entries(rows, cols, Ah, B)
    assert np.all(np.abs(vals.cpu().numpy() - want) <= BLOCK * 2.0 ** -23 * _abs_sums(Ah, B, rows, cols))
    s.close()
    t = pipeline.Solver(n1, N2, 16, torch.float32, seed=1, engine=smp.SMP_ENGINE_TC, max_rows=BLOCK)
    t.norms(torch.from_numpy(np.ascontiguousarray(A[:, :n1])).cuda(), Bd, BLOCK)
    t.sample(O.default_m(n1, N2, 5), seed=3)
    with pytest.raises(smp.SmpError) as e:
        smp.smp_exact_accumulate(t.ctx, Ad, n1 + 1, Bd, N2, 0, BLOCK)
    assert e.value.status == smp.SMP_EUNSUPPORTED
    t.close()


@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_lela_end_to_end_tiny(env, dtype_name):
    """The tiny workload's shape (d = 2,000, n = 200, r = 5, T = 10): Omega bit-exact against the oracle's LELA,
    the relative spectral error within 1e-3 of the oracle's (binary32 inputs) or 1e-6 (binary64)."""
    torch, smp, pipeline = env
    npdt = np.float32 if dtype_name == "f32" else np.float64
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=npdt)
    tdt = torch.float32 if dtype_name == "f32" else torch.float64
    s = pipeline.Solver(200, 200, 16, tdt, seed=1)
    m = O.default_m(200, 200, 5)
    out = s.lela(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5, 10, m=m, sample_seed=2, walt_seed=3)
    ref = O.lela(A, B, 5, m, 10, sample_seed=2)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A.astype(np.float64).T @ B.astype(np.float64)
    err_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    err_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(err_gpu - err_ref) <= (1e-3 if dtype_name == "f32" else 1e-6)
    assert err_gpu >= O.optimal_error(M, 5) - 1e-12
    s.close()


def test_lela_pca_case_on_tensor_cores(env):
    """A = B (PCA): the transposed block of A is both operands; Omega and the error against the oracle."""
    torch, smp, pipeline = env
    A, _ = synth.lowrank_plus_noise(3000, 260, 260, 6, 0.1, 0.5, seed=44, same_ab=True)
    s = pipeline.Solver(260, 260, 16, torch.float32, seed=5, same_ab=True, engine=smp.SMP_ENGINE_TC, max_rows=1024)
    m = O.default_m(260, 260, 4)
    out = s.lela(torch.from_numpy(A).cuda(), None, 4, 10, m=m, sample_seed=6, walt_seed=3, block_rows=1024)
    ref = O.lela(A, None, 4, m, 10, sample_seed=6, same_ab=True)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    rows, cols = ref["rows"], ref["cols"]
    vals = out["vals"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(vals - ref["vals"]) <= (2.0 ** -10 + 1024 * 2.0 ** -23) * _abs_sums(A, A, rows, cols))
    M = A.astype(np.float64).T @ A.astype(np.float64)
    err_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    err_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(err_gpu - err_ref) <= 1e-3
    s.close()


def test_exact_bitwise_reproducible(env, data):
    """Fixed-order split sums: two runs give the same bits; blocks in another order give the same Omega."""
    torch, smp, pipeline = env
    A, B = data
    outs = []
    for _ in range(2):
        s = pipeline.Solver(N1, N2, 16, torch.float32, seed=1, max_rows=BLOCK)
        outs.append(_lela_gpu(torch, s, A, B, O.default_m(N1, N2, 8), 5, BLOCK)[1])
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_call_order_errors(env, data):
    torch, smp, pipeline = env
    A, B = data
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    s = pipeline.Solver(N1, N2, 16, torch.float32, seed=1, max_rows=BLOCK)
    with pytest.raises(smp.SmpError) as e:     # no Omega yet
        smp.smp_exact_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 100)
    assert e.value.status == smp.SMP_ESTATE
    smp.smp_norms_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 100)
    with pytest.raises(smp.SmpError) as e:     # sketch rows after norms-only rows
        smp.smp_sketch_accumulate(s.ctx, Ad[100:], N1, Bd[100:], N2, 100, 100)
    assert e.value.status == smp.SMP_ESTATE
    smp.smp_norms_accumulate(s.ctx, Ad[100:], N1, Bd[100:], N2, 100, 100)
    smp.smp_sketch_finalize(s.ctx)
    s.sample(5000.0, seed=2)
    with pytest.raises(smp.SmpError) as e:     # no sketch to estimate from
        smp.smp_estimate(s.ctx, torch.empty(10, device="cuda"))
    assert e.value.status == smp.SMP_ESTATE
    with pytest.raises(smp.SmpError) as e:     # values before any exact rows
        smp.smp_exact_values(s.ctx, torch.empty(10, device="cuda"))
    assert e.value.status == smp.SMP_ESTATE
    smp.smp_exact_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 150)
    with pytest.raises(smp.SmpError) as e:     # overlaps rows 0..150
        smp.smp_exact_accumulate(s.ctx, Ad[100:], N1, Bd[100:], N2, 100, 100)
    assert e.value.status == smp.SMP_EINVAL
    assert smp.smp_exact_coverage(s.ctx) == (150, 150, 1)
    s.sample(5000.0, seed=3)                   # a new Omega starts the exact pass afresh
    assert smp.smp_exact_coverage(s.ctx) == (0, 0, 0)
    smp.smp_sketch_reset(s.ctx)                # and a reset frees the pass kind
    smp.smp_sketch_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 100)
    s.close()


def test_exact_entries_at_the_scale_shape(env):
    """The scale workload's launch configuration (n = 2,000, 65,536-row blocks, r = 10, m = 4 n r ln n) on four
    blocks: 128 sampled entries recomputed one by one in binary64 from the data."""
    torch, smp, pipeline = env
    n, R, nb, r = 2000, 65536, 4, 10
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(nb * R, n, n, 20, 0.1, 0.5, seed=9, device="cuda")
    s = pipeline.Solver(n, n, 16, torch.float32, seed=1, max_rows=R)
    s.norms(A, B, R)
    nnz = s.sample(O.default_m(n, n, r), seed=2)
    vals = s.exact(A, B, R).cpu().numpy().astype(np.float64)
    om = omega_numpy(s)
    rows, cols = csr_rows(om["row_ptr"]), om["col"]
    pick = np.random.default_rng(0).choice(nnz, 128, replace=False)
    Ai = A[:, torch.from_numpy(rows[pick]).cuda()].double().cpu().numpy()
    Bj = B[:, torch.from_numpy(cols[pick].astype(np.int64)).cuda()].double().cpu().numpy()
    want = np.einsum("te,te->e", Ai, Bj)
    scale = np.einsum("te,te->e", np.abs(Ai), np.abs(Bj))
    assert np.all(np.abs(vals[pick] - want) <= (2.0 ** -10 + R * 2.0 ** -23) * scale)
    assert np.linalg.norm(vals[pick] - want) <= 1e-3 * np.linalg.norm(want)
    s.close()


def test_table1_error_evaluator_matches_dense(env):
    """bench.py's implicit spectral-error evaluator (used where A^T A is too large to form) against dense SVDs of
    A^T A on a G D instance small enough to form (d = n = 1,500), with LELA's factors and a random rank-5 pair."""
    torch, smp, pipeline = env
    import bench
    from paper_1610_06656_gb300 import synth as sy
    n, r = 1500, 5
    A = sy.gd_torch(n, n, seed=3, device="cuda")
    s = pipeline.Solver(n, n, 16, torch.float32, seed=1, same_ab=True, max_rows=1024)
    out = s.lela(A, None, r, 10, block_rows=1024)
    s.close()
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    rnd = (torch.randn(n, r, generator=g, device="cuda", dtype=torch.float64),
           torch.rand(r, generator=g, device="cuda", dtype=torch.float64),
           torch.randn(n, r, generator=g, device="cuda", dtype=torch.float64))
    factors = [(out["U"], out["S"], out["V"]), rnd]
    errs, opt = bench.implicit_errors(torch, A, factors, r)
    M = A.double().T @ A.double()
    sv = torch.linalg.svdvals(M)
    assert abs(opt - float(sv[r] / sv[0])) <= 1e-4 * float(sv[r] / sv[0])
    for (U, S, V), e in zip(factors, errs):
        want = float(torch.linalg.matrix_norm(M - (U * S) @ V.T, ord=2) / sv[0])
        assert abs(e - want) <= 1e-3 * want
