"""Parity of the row-wise multinomial sampler (smp_sample_multinomial, Appendix "Sampling") with the oracle: Omega
(CSR and CSC) and the stored q^ bit for bit, since both sides take every decision with the same binary64 operations
in the same order (the blocked prefix of beta included)."""
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


def _norms_solver(torch, pipeline, smp, sA, sB, k=8):
    n1, n2 = sA.shape[0], sB.shape[0]
    s = pipeline.Solver(n1, n2, k, torch.float32, seed=1)
    smp.smp_sketch_import(s.ctx, torch.zeros(n1, k, device="cuda"), torch.zeros(n2, k, device="cuda"),
                          torch.from_numpy(sA).cuda(), torch.from_numpy(sB).cuda())
    return s


@pytest.mark.parametrize("n1,n2,m,seed", [(200, 200, 21193.0, 2), (37, 2500, 9000.5, 7), (3000, 70, 40000.0, 9),
                                          (64, 64, 1e6, 3)])
def test_omega_bit_exact(env, n1, n2, m, seed):
    """Power-law norms (a few heavy rows take thousands of draws), n2 spanning several prefix blocks, ragged sizes,
    and m > n1 n2 (many repeated draws)."""
    torch, smp, pipeline = env
    rng = np.random.default_rng(n1 + n2)
    sA = rng.uniform(0.5, 1.5, n1) / (np.arange(n1) + 1.0)
    sB = rng.uniform(0.5, 1.5, n2) / np.sqrt(np.arange(n2) + 1.0)
    s = _norms_solver(torch, pipeline, smp, sA, sB)
    nnz = s.sample(m, seed, sampler="multinomial")
    rows, cols, qh, cnt = O.sample_omega_multinomial(sA, sB, m, seed)
    assert nnz == rows.shape[0]
    om = omega_numpy(s)
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
    np.testing.assert_array_equal(om["col"], cols)
    np.testing.assert_array_equal(om["qhat"], qh)
    order = np.lexsort((rows, cols))                              # CSC: by column, rows increasing
    np.testing.assert_array_equal(om["csc_row"], rows[order])
    np.testing.assert_array_equal(om["csc_pos"], order)
    s.close()


def test_end_to_end_tiny(env):
    """The tiny workload with multinomial Omega through the whole GPU path against the oracle's run (binary64
    context): Omega bit-exact, factors within 1e-6."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float64)
    s = pipeline.Solver(200, 200, 100, torch.float64, seed=1)
    m = O.default_m(200, 200, 5)
    out = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5, 10, m=m, sample_seed=2, walt_seed=3,
                  sampler="multinomial")
    ref = O.smp_pca(A, B, 5, 100, m, 10, seed=1, sample_seed=2, sampler="multinomial")
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A.T @ B
    e_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= 1e-6
    s.close()


def test_state_errors(env):
    torch, smp, pipeline = env
    s = pipeline.Solver(20, 20, 8, torch.float32, seed=1)
    with pytest.raises(smp.SmpError) as e:
        s.sample(100.0, 1, sampler="multinomial")
    assert e.value.status == smp.SMP_ESTATE
    s.close()


def test_rows_without_draws_and_single_column(env):
    """Tiny m: most rows round to zero draws (c_i = 0) and contribute no entries; n2 = 1: every draw is column 0."""
    torch, smp, pipeline = env
    rng = np.random.default_rng(21)
    for n1, n2, m in ((300, 40, 50.0), (50, 1, 400.0)):
        sA = rng.uniform(0.1, 2.0, n1) / (np.arange(n1) + 1.0) ** 2
        sB = rng.uniform(0.1, 2.0, n2)
        s = _norms_solver(torch, pipeline, smp, sA, sB)
        nnz = s.sample(m, 4, sampler="multinomial")
        rows, cols, qh, cnt = O.sample_omega_multinomial(sA, sB, m, 4)
        assert nnz == rows.shape[0]
        om = omega_numpy(s)
        np.testing.assert_array_equal(csr_rows(om["row_ptr"]), rows)
        np.testing.assert_array_equal(om["col"], cols)
        np.testing.assert_array_equal(om["qhat"], qh)
        s.close()
