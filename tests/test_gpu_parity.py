"""Stage and end-to-end parity of the CUDA path (through the C ABI) against the CPU oracle.

Sizes span several CTA tiles with ragged tails: d = 2,000 rows in 700-row blocks (32-row steps), n1 = 200 and
n2 = 170 columns (64-column tiles), k = 100 (64-row sketch chunks, not a multiple of 8).
"""
import math

import numpy as np
import pytest

from oracle import philox, smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, csr_rows, omega_numpy, philox_probe, torch_cuda

pytestmark = pytest.mark.gpu

D, N1, N2, K, R, T = 2000, 200, 170, 100, 5, 10
BLOCK = 700


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    return torch, smp, pipeline


@pytest.fixture(scope="module")
def data():
    A, B = synth.lowrank_plus_noise(D, N1, N2, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    return A, B


def _oracle_sketch(A, B, seed, same_ab=False, block=BLOCK):
    return O.sketch(A, B, K, seed, block_rows=block, same_ab=same_ab)


def _colrel(X, Y):
    """max over columns of ||X_c - Y_c|| / ||Y_c|| (columns = sketch columns, rows of the (n x k) arrays)."""
    num = np.linalg.norm(X - Y, axis=1)
    den = np.maximum(np.linalg.norm(Y, axis=1), 1e-300)
    return float((num / den).max())


# ------------------------------------------------------------------------------------------------ random streams
def test_philox_matches_curand(env):
    torch, _, _ = env
    rng = np.random.default_rng(5)
    n = 4096
    ctr = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64)
    key = rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64)
    ctr[:16] = 0
    key[:8] = 0
    key[8:16] = 0xFFFFFFFF
    c_d = torch.tensor(ctr.astype(np.uint32).view(np.int32), device="cuda")
    k_d = torch.tensor(key.astype(np.uint32).view(np.int32), device="cuda")
    mine = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    ref = torch.empty(n * 4, dtype=torch.int32, device="cuda")
    assert philox_probe().philox_pair(c_d.data_ptr(), k_d.data_ptr(), n, mine.data_ptr(), ref.data_ptr()) == 0
    ref_h = ref.cpu().numpy().view(np.uint32).reshape(n, 4)
    np.testing.assert_array_equal(mine.cpu().numpy().view(np.uint32).reshape(n, 4), ref_h)
    ora = np.stack(philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], 0, 0), axis=1)
    # the oracle with a per-row key: evaluate row by row for the keyed part
    for e in range(0, n, 97):
        o = philox.philox4x32_10_scalar(tuple(int(x) for x in ctr[e]), (int(key[e, 0]), int(key[e, 1])))
        assert o == tuple(int(x) for x in ref_h[e])
    zero_key = (key[:, 0] == 0) & (key[:, 1] == 0)
    np.testing.assert_array_equal(ora[zero_key].astype(np.uint32), ref_h[zero_key])


def test_gpu_pi_matches_oracle_pi(env):
    """Sketching an identity block returns Pi's columns: the GPU's Philox + Box-Muller stream equals the oracle's
    to binary32 rounding (including data-row indices above 2^32)."""
    torch, smp, pipeline = env
    k, n = 40, 96
    for row0 in (0, 123456, (1 << 32) - 37):
        s = pipeline.Solver(n, n, k, torch.float32, seed=77, same_ab=True, engine=smp.SMP_ENGINE_SIMT)
        eye = torch.eye(n, dtype=torch.float32, device="cuda")
        smp.smp_sketch_accumulate(s.ctx, eye, n, None, 0, row0, n)
        smp.smp_sketch_finalize(s.ctx)
        got = s.sketch_state()["At"].cpu().numpy().T            # k x n
        want = philox.pi_block(77, k, row0, n)
        assert np.abs(got - want).max() < 2e-5 / math.sqrt(k) * 10
        s.close()


# ------------------------------------------------------------------------------------------------ sketch
@pytest.mark.parametrize("same_ab", [False, True])
def test_sketch_simt_f32(env, data, same_ab):
    torch, smp, pipeline = env
    A, B = data
    if same_ab:
        B = A
    n2 = N1 if same_ab else N2
    s = pipeline.Solver(N1, n2, K, torch.float32, seed=11, same_ab=same_ab, engine=smp.SMP_ENGINE_SIMT)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(B)).cuda()
    order = [1400, 0, 700]                                       # blocks in any order, ragged last block
    s.sketch(Ad, Bd, BLOCK, order=order)
    st = s.sketch_state()
    ref = _oracle_sketch(A, B, 11, same_ab)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 2e-5
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 2e-5
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-13)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-13)
    assert st["F"][0] == pytest.approx(O.frobenius_sq(ref.sA), rel=1e-13)
    s.close()


def test_sketch_simt_f64(env, data):
    torch, smp, pipeline = env
    A, B = (x.astype(np.float64) for x in data)
    s = pipeline.Solver(N1, N2, K, torch.float64, seed=12, engine=smp.SMP_ENGINE_SIMT)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), BLOCK)
    st = s.sketch_state()
    ref = _oracle_sketch(A, B, 12)
    assert _colrel(st["At"].cpu().numpy(), ref.At.T) < 1e-12
    assert _colrel(st["Bt"].cpu().numpy(), ref.Bt.T) < 1e-12
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-14)
    s.close()


@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_long_sketch_above_1024(env, dtype_name):
    """k = 2,000 (Table 1's sketch size; above the tensor-core engines' limits): the CUDA-core sketch and the
    estimate's long-sketch kernel against the oracle, 400 rows in 150-row blocks, n1 = 70, n2 = 50."""
    torch, smp, pipeline = env
    npdt = np.float32 if dtype_name == "f32" else np.float64
    A, B = synth.lowrank_plus_noise(400, 70, 50, 5, 0.1, 0.5, seed=8, dtype=npdt)
    tdt = torch.float32 if dtype_name == "f32" else torch.float64
    k = 2000
    s = pipeline.Solver(70, 50, k, tdt, seed=13, max_rows=150)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 150)
    st = s.sketch_state()
    ref = O.sketch(A, B, k, 13, block_rows=150)
    tol = 2e-5 if dtype_name == "f32" else 1e-12
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < tol
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < tol
    m = O.default_m(70, 50, 3)
    nnz = s.sample(m, seed=4)
    vals = s.estimate(nnz).cpu().numpy().astype(np.float64)
    om = omega_numpy(s)
    rows, cols = csr_rows(om["row_ptr"]), om["col"]
    want = O.estimate(rows, cols, ref.At, ref.Bt, ref.sA, ref.sB)
    scale = np.sqrt(ref.sA[rows] * ref.sB[cols])
    assert np.max(np.abs(vals - want) / scale) < (2e-5 if dtype_name == "f32" else 1e-11)
    s.close()


def test_sketch_identity_pi_is_exact(env):
    """Pi = I (k = d) through the explicit-Pi hook: At = A bit for bit, so M~ = A^T B exactly."""
    torch, smp, pipeline = env
    d = 64
    A, B = synth.lowrank_plus_noise(d, 24, 30, 3, 0.1, 0.5, seed=3, dtype=np.float32)
    s = pipeline.Solver(24, 30, d, torch.float32, seed=1, engine=smp.SMP_ENGINE_SIMT)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    eye = torch.eye(d, dtype=torch.float32, device="cuda")
    smp.smp_sketch_accumulate_pi(s.ctx, eye, d, Ad, 24, Bd, 30, 0, d)
    smp.smp_sketch_finalize(s.ctx)
    st = s.sketch_state()
    np.testing.assert_array_equal(st["At"].cpu().numpy(), A.T)
    np.testing.assert_array_equal(st["Bt"].cpu().numpy(), B.T)
    nnz = s.sample(1e12, seed=2)
    assert nnz == 24 * 30
    vals = s.estimate(nnz).cpu().numpy()
    om = omega_numpy(s)
    rows, cols = np.repeat(np.arange(24), 30), np.tile(np.arange(30), 24)   # every entry, row-major
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    np.testing.assert_array_equal(om["col"], cols)
    M = A.astype(np.float64).T @ B.astype(np.float64)
    np.testing.assert_allclose(vals, M[rows, cols], rtol=2e-6, atol=1e-6 * np.abs(M).max())
    s.close()


def test_call_order_and_argument_errors(env, data):
    torch, smp, pipeline = env
    A, B = data
    s = pipeline.Solver(N1, N2, K, torch.float32, seed=1)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    smp.smp_sketch_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 0)            # empty block: no-op
    with pytest.raises(smp.SmpError) as e:
        smp.smp_estimate(s.ctx, torch.empty(1, device="cuda"))
    assert e.value.status == smp.SMP_ESTATE
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_accumulate(s.ctx, Ad, N1 - 1, Bd, N2, 0, 10)   # lda < n1
    assert e.value.status == smp.SMP_EINVAL
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 70000)    # nrows > max_rows
    assert e.value.status == smp.SMP_EINVAL
    smp.smp_sketch_finalize(s.ctx)
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_accumulate(s.ctx, Ad, N1, Bd, N2, 0, 10)
    assert e.value.status == smp.SMP_ESTATE
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_finalize(s.ctx)
    assert e.value.status == smp.SMP_ESTATE
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sample(s.ctx, -1.0, 2)
    assert e.value.status == smp.SMP_EINVAL
    s.close()
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_begin(10, 10, 0, 1)
    assert e.value.status == smp.SMP_EINVAL
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_begin(10, 12, 8, 1, same_ab=True)
    assert e.value.status == smp.SMP_EINVAL


# ------------------------------------------------------------------------------------------------ sampling
def _random_norms(n, seed, zero_some=False):
    rng = np.random.default_rng(seed)
    s = rng.gamma(0.6, 3.0, size=n) * (np.arange(1, n + 1) ** -0.7)
    if zero_some:
        s[rng.integers(0, n, size=max(1, n // 20))] = 0.0
    return s


def _oracle_csc(rows, cols, n2):
    order = np.lexsort((rows, cols))
    col_ptr = np.concatenate([[0], np.cumsum(np.bincount(cols, minlength=n2))])
    return col_ptr, rows[order], order


@pytest.mark.parametrize("n1,n2,m", [(200, 170, 5000.0), (333, 65, 40000.0), (64, 97, 12.5), (40, 50, 1e9)])
def test_sample_bit_exact_from_norms(env, n1, n2, m):
    torch, smp, pipeline = env
    sA, sB = _random_norms(n1, 1, zero_some=True), _random_norms(n2, 2)
    s = pipeline.Solver(n1, n2, 8, torch.float32, seed=1)
    nnz = smp.smp_sample_from_norms(s.ctx, torch.from_numpy(sA).cuda(), torch.from_numpy(sB).cuda(), m, 99)
    rows, cols, qh = O.sample_omega(sA, sB, m, 99)
    assert nnz == rows.shape[0]
    om = omega_numpy(s)
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    np.testing.assert_array_equal(om["col"], cols)
    np.testing.assert_array_equal(om["qhat"], qh)                  # bitwise: same IEEE ops in the same order
    col_ptr, csc_row, csc_pos = _oracle_csc(rows, cols, n2)
    np.testing.assert_array_equal(om["col_ptr"], col_ptr)
    np.testing.assert_array_equal(om["csc_row"], csc_row)
    np.testing.assert_array_equal(om["csc_pos"], csc_pos)
    s.close()


def test_sample_after_gpu_sketch(env, data):
    """Omega drawn from the GPU's own norms is the oracle's Omega for those norms (bit-exact), and (with
    compensated sums) the same as the oracle's Omega from its own binary64 norms."""
    torch, smp, pipeline = env
    A, B = data
    s = pipeline.Solver(N1, N2, K, torch.float32, seed=11, engine=smp.SMP_ENGINE_SIMT)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), BLOCK)
    m = O.default_m(N1, N2, R)
    nnz = s.sample(m, seed=7)
    st = s.sketch_state()
    om = omega_numpy(s)
    rows, cols, _ = O.sample_omega(st["sA"].cpu().numpy(), st["sB"].cpu().numpy(), m, 7)
    np.testing.assert_array_equal(om["col"], cols)
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    ref = _oracle_sketch(A, B, 11)
    rows2, cols2, _ = O.sample_omega(ref.sA, ref.sB, m, 7)
    assert nnz == rows2.shape[0]
    np.testing.assert_array_equal(om["col"], cols2)
    s.close()


# ------------------------------------------------------------------------------------------------ estimate
def test_estimate_matches_oracle(env, data):
    torch, smp, pipeline = env
    A, B = data
    ref = _oracle_sketch(A, B, 21)
    At32 = np.ascontiguousarray(ref.At.T.astype(np.float32))
    Bt32 = np.ascontiguousarray(ref.Bt.T.astype(np.float32))
    s = pipeline.Solver(N1, N2, K, torch.float32, seed=21)
    smp.smp_sketch_import(s.ctx, torch.from_numpy(At32).cuda(), torch.from_numpy(Bt32).cuda(),
                          torch.from_numpy(ref.sA).cuda(), torch.from_numpy(ref.sB).cuda())
    nnz = s.sample(O.default_m(N1, N2, R), seed=3)
    vals = s.estimate(nnz).cpu().numpy().astype(np.float64)
    # the oracle's own Omega (the GPU's equals it bit for bit) indexes the oracle's estimate
    rows, cols, _ = O.sample_omega(ref.sA, ref.sB, O.default_m(N1, N2, R), 3)
    om = omega_numpy(s)
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    np.testing.assert_array_equal(om["col"], cols)
    want = O.estimate(rows, cols, At32.T.astype(np.float64), Bt32.T.astype(np.float64), ref.sA, ref.sB)
    scale = np.sqrt(ref.sA[rows] * ref.sB[cols])
    assert np.max(np.abs(vals - want) / scale) < 2e-6
    s.close()


# ------------------------------------------------------------------------------------------------ WAltMin
def _waltmin_setup(env, data, seed=31):
    torch, smp, pipeline = env
    A, B = data
    ref = _oracle_sketch(A, B, seed)
    s = pipeline.Solver(N1, N2, K, torch.float32, seed=seed)
    At32 = np.ascontiguousarray(ref.At.T.astype(np.float32))
    Bt32 = np.ascontiguousarray(ref.Bt.T.astype(np.float32))
    smp.smp_sketch_import(s.ctx, torch.from_numpy(At32).cuda(), torch.from_numpy(Bt32).cuda(),
                          torch.from_numpy(ref.sA).cuda(), torch.from_numpy(ref.sB).cuda())
    m = O.default_m(N1, N2, R)
    s.sample(m, seed=5)
    # the oracle's own Omega (the GPU's equals it bit for bit) feeds the oracle's estimate and WAltMin
    rows, cols, qh = O.sample_omega(ref.sA, ref.sB, m, 5)
    og = omega_numpy(s)
    np.testing.assert_array_equal(csr_rows(og["row_ptr"]), rows)
    np.testing.assert_array_equal(og["col"], cols)
    om = dict(col=cols, qhat=qh)
    vals32 = O.estimate(rows, cols, At32.T.astype(np.float64), Bt32.T.astype(np.float64), ref.sA,
                        ref.sB).astype(np.float32)
    return s, ref, rows, om, vals32


def _product(U, S, V):
    return (U * S) @ V.T


@pytest.mark.parametrize("fp64", [True, False])
def test_waltmin_iterations_from_given_init(env, data, fp64):
    torch, smp, pipeline = env
    s, ref, rows, om, vals32 = _waltmin_setup(env, data)
    v64 = vals32.astype(np.float64)
    rng = np.random.default_rng(4)
    U0 = np.linalg.qr(rng.standard_normal((N1, R)))[0]
    flags = smp.SMP_INIT_GIVEN | (smp.SMP_FP64_ALS if fp64 else 0)
    U, S, V = s.waltmin(torch.from_numpy(vals32).cuda(), R, T, flags, seed=9, U_init=torch.from_numpy(U0).cuda())
    Uh, Vh = O.waltmin(N1, N2, rows, om["col"], v64, om["qhat"], R, T, ref.sA, U_init=U0)
    Uo, So, Vo = O.canonical(Uh, Vh)
    P, Po = _product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()), _product(Uo, So, Vo)
    tol = 1e-9 if fp64 else 2e-4
    assert np.linalg.norm(P - Po) <= tol * np.linalg.norm(Po)
    np.testing.assert_allclose(S.cpu().numpy(), So, rtol=tol * 10)
    # canonical form: orthonormal columns and the sign rule
    Ug = U.cpu().numpy()
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(R), atol=1e-10)
    for c in range(R):
        assert Ug[np.argmax(np.abs(Ug[:, c])), c] > 0
    s.close()


def test_waltmin_full_fp64(env, data):
    """Steps 2-10 with the subspace-iteration initial SVD against the oracle's LAPACK SVD initial iterate."""
    torch, smp, pipeline = env
    s, ref, rows, om, vals32 = _waltmin_setup(env, data)
    U, S, V = s.waltmin(torch.from_numpy(vals32).cuda(), R, T, smp.SMP_FP64_ALS, seed=9)
    Uh, Vh = O.waltmin(N1, N2, rows, om["col"], vals32.astype(np.float64), om["qhat"], R, T, ref.sA)
    Uo, So, Vo = O.canonical(Uh, Vh)
    P, Po = _product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()), _product(Uo, So, Vo)
    assert np.linalg.norm(P - Po) <= 1e-6 * np.linalg.norm(Po)
    s.close()


def test_waltmin_split_mode_fp64(env, data):
    torch, smp, pipeline = env
    s, ref, rows, om, vals32 = _waltmin_setup(env, data)
    rng = np.random.default_rng(8)
    U0 = np.linalg.qr(rng.standard_normal((N1, R)))[0]
    flags = smp.SMP_INIT_GIVEN | smp.SMP_FP64_ALS | smp.SMP_SPLIT_OMEGA
    T2 = 2
    U, S, V = s.waltmin(torch.from_numpy(vals32).cuda(), R, T2, flags, seed=17, U_init=torch.from_numpy(U0).cuda())
    Uh, Vh = O.waltmin(N1, N2, rows, om["col"], vals32.astype(np.float64), om["qhat"], R, T2, ref.sA,
                       split=O.SPLIT_OMEGA, split_seed=17, U_init=U0)
    Uo, So, Vo = O.canonical(Uh, Vh)
    P, Po = _product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()), _product(Uo, So, Vo)
    # each of the 2T+1 = 5 subsets leaves some rows with about r samples, so their r x r systems are nearly
    # singular (condition ~1e10): binary64 rounding-order differences grow to ~1e-6 there
    assert np.linalg.norm(P - Po) <= 1e-5 * np.linalg.norm(Po)
    s.close()


# ------------------------------------------------------------------------------------------------ end to end
@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_end_to_end_tiny(env, dtype_name):
    """The tiny workload (d = 2,000, n = 200, k = 100, r = 5, T = 10): Omega bit-exact against the oracle, and
    the relative spectral error of U S V^T within 1e-3 of the oracle's."""
    torch, smp, pipeline = env
    npdt = np.float32 if dtype_name == "f32" else np.float64
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=npdt)
    tdt = torch.float32 if dtype_name == "f32" else torch.float64
    s = pipeline.Solver(200, 200, 100, tdt, seed=1, engine=smp.SMP_ENGINE_SIMT)
    m = O.default_m(200, 200, 5)
    out = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5, 10, m=m, sample_seed=2, walt_seed=3)
    ref = O.smp_pca(A, B, 5, 100, m, 10, seed=1, sample_seed=2)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A.astype(np.float64).T @ B.astype(np.float64)
    err_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    err_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(err_gpu - err_ref) <= 1e-3
    assert err_gpu >= O.optimal_error(M, 5) - 1e-12
    s.close()


def test_end_to_end_pca_case(env):
    torch, smp, pipeline = env
    A, _ = synth.lowrank_plus_noise(3000, 120, 120, 6, 0.1, 0.5, seed=44, same_ab=True)
    s = pipeline.Solver(120, 120, 64, torch.float32, seed=5, same_ab=True, engine=smp.SMP_ENGINE_SIMT)
    m = O.default_m(120, 120, 4)
    out = s.solve(torch.from_numpy(A).cuda(), None, 4, 10, m=m, sample_seed=6, walt_seed=3)
    ref = O.smp_pca(A, None, 4, 64, m, 10, seed=5, sample_seed=6, same_ab=True)
    M = A.astype(np.float64).T @ A.astype(np.float64)
    err_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    err_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(err_gpu - err_ref) <= 1e-3
    s.close()


def test_full_sampling_identity_pi_recovers_svd(env):
    """Pi = I and q^ = 1 on an exactly rank-3 product: the output is the SVD of A^T B."""
    torch, smp, pipeline = env
    d = 64
    A, B = synth.lowrank_plus_noise(d, 20, 18, 3, 0.0, 0.3, seed=8, dtype=np.float32)
    s = pipeline.Solver(20, 18, d, torch.float32, seed=1, engine=smp.SMP_ENGINE_SIMT)
    eye = torch.eye(d, dtype=torch.float32, device="cuda")
    smp.smp_sketch_accumulate_pi(s.ctx, eye, d, torch.from_numpy(A).cuda(), 20, torch.from_numpy(B).cuda(), 18, 0, d)
    smp.smp_sketch_finalize(s.ctx)
    nnz = s.sample(1e12, seed=1)
    vals = s.estimate(nnz)
    U, S, V = s.waltmin(vals, 3, 15, smp.SMP_FP64_ALS, seed=2)
    M = A.astype(np.float64).T @ B.astype(np.float64)
    sv = np.linalg.svd(M, compute_uv=False)
    np.testing.assert_allclose(S.cpu().numpy(), sv[:3], rtol=1e-5)
    assert np.linalg.norm(_product(U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()) - M, 2) < 1e-5 * sv[0]
    s.close()


def test_bitwise_reproducible(env, data):
    torch, smp, pipeline = env
    A, B = data
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    outs = []
    s = pipeline.Solver(N1, N2, K, torch.float32, seed=3)
    for _ in range(2):
        o = s.solve(Ad, Bd, R, 4, sample_seed=4, walt_seed=5, block_rows=BLOCK)
        outs.append([o["vals"].cpu().numpy(), o["U"].cpu().numpy(), o["S"].cpu().numpy()])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    s.close()
