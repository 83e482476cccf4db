"""Parity of the block SRHT sketch engine (SMP_ENGINE_SRHT: two-stage Walsh-Hadamard transform of every row
block, then the sampled rows) with the oracle's sketch_srht. Binary32 transforms of up to 2^16 terms against
binary64: sketch columns within relative 1e-5; column norms compensated, 1e-12; Omega bit-exact downstream."""
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
    return float((np.linalg.norm(X - Y, axis=1) / np.maximum(np.linalg.norm(Y, axis=1), 1e-300)).max())


@pytest.mark.parametrize("d,n1,n2,k,lg,order", [(3000, 200, 136, 100, 10, [2048, 0, 1024]),
                                                (3000, 200, 136, 700, 8, None),
                                                (70000, 40, 72, 64, 16, [65536, 0])])
def test_sketch_matches_oracle(env, d, n1, n2, k, lg, order):
    """Blocks of 2^lg rows (the last one partial), column tiles straddling the A/B boundary, k > 512, and 2^16-row
    blocks (256 chunks in the second stage)."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(d, n1, n2, 10, 0.1, 0.5, seed=1000 + d, dtype=np.float32)
    R = 1 << lg
    s = pipeline.Solver(n1, n2, k, torch.float32, seed=11, engine=smp.SMP_ENGINE_SRHT, max_rows=R)
    s.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), R, order=order)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch_srht(A.astype(np.float64), B.astype(np.float64), k, 11, lg)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 1e-5
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < 1e-5
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-12)
    s.close()


def test_same_ab(env):
    torch, smp, pipeline = env
    A, _ = synth.lowrank_plus_noise(1500, 130, 130, 8, 0.1, 0.5, seed=7, dtype=np.float32)
    s = pipeline.Solver(130, 130, 96, torch.float32, seed=5, same_ab=True, engine=smp.SMP_ENGINE_SRHT, max_rows=512)
    Ad = torch.from_numpy(A).cuda()
    s.sketch(Ad, Ad, 512)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch_srht(A.astype(np.float64), None, 96, 5, 9, same_ab=True)
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < 1e-5
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    s.close()


def test_end_to_end_tiny(env):
    """Tiny workload through the SRHT engine (256-row blocks): Omega bit-exact against the oracle, spectral error
    within 1e-4 of the oracle's."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(2000, 200, 200, 10, 0.1, 0.5, seed=1000, dtype=np.float32)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    s = pipeline.Solver(200, 200, 100, torch.float32, seed=1, engine=smp.SMP_ENGINE_SRHT, max_rows=256)
    m = O.default_m(200, 200, 5)
    out = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 5, 10, m=m, sample_seed=2, walt_seed=3,
                  block_rows=256)
    ref = O.smp_pca(A64, B64, 5, 100, m, 10, seed=1, sample_seed=2, srht_log2=8)
    om = omega_numpy(s)
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])
    M = A64.T @ B64
    e_gpu = O.spectral_error(M, out["U"].cpu().numpy(), out["S"].cpu().numpy(), out["V"].cpu().numpy())
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= 1e-4
    s.close()


def test_argument_errors(env):
    torch, smp, pipeline = env
    with pytest.raises(smp.SmpError) as e:
        pipeline.Solver(30, 30, 16, torch.bfloat16, seed=1, engine=smp.SMP_ENGINE_SRHT, max_rows=256)
    assert e.value.status == smp.SMP_EUNSUPPORTED
    with pytest.raises(smp.SmpError) as e:
        pipeline.Solver(30, 30, 16, torch.float32, seed=1, engine=smp.SMP_ENGINE_SRHT, max_rows=1000)
    assert e.value.status == smp.SMP_EINVAL
    s = pipeline.Solver(30, 30, 16, torch.float32, seed=1, engine=smp.SMP_ENGINE_SRHT, max_rows=256)
    X = torch.zeros(100, 30, device="cuda")
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_accumulate(s.ctx, X, 30, X, 30, 100, 100)
    assert e.value.status == smp.SMP_EINVAL
    s.close()
