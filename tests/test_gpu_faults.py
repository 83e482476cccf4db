"""Failure paths, made on the host (no GPU fault): duplicated or overlapping row blocks are rejected before
anything is launched, coverage reports what has been sketched, and injected device-allocation failures surface as
SMP_ENOMEM with the context still usable or destroyable."""
import numpy as np
import pytest

from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    return torch, smp, pipeline


def test_duplicate_and_overlapping_blocks(env):
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(3000, 64, 48, 5, 0.1, 0.5, seed=3, dtype=np.float32)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    s = pipeline.Solver(64, 48, 32, torch.float32, seed=1, max_rows=1000)
    smp.smp_sketch_reset(s.ctx)
    smp.smp_sketch_accumulate(s.ctx, Ad[1000:2000], 64, Bd[1000:2000], 48, 1000, 1000)
    assert smp.smp_sketch_coverage(s.ctx) == (1000, 0, 1)                     # row 0 still missing
    for r0, nr in ((1000, 1000), (1500, 10), (500, 600), (1999, 1)):           # duplicate / inside / straddling
        with pytest.raises(smp.SmpError) as e:
            smp.smp_sketch_accumulate(s.ctx, Ad[r0:r0 + nr], 64, Bd[r0:r0 + nr], 48, r0, nr)
        assert e.value.status == smp.SMP_EINVAL
    smp.smp_sketch_accumulate(s.ctx, Ad[0:1000], 64, Bd[0:1000], 48, 0, 1000)
    assert smp.smp_sketch_coverage(s.ctx) == (2000, 2000, 1)                  # merged into one range
    smp.smp_sketch_accumulate(s.ctx, Ad[2500:3000], 64, Bd[2500:3000], 48, 2500, 500)
    assert smp.smp_sketch_coverage(s.ctx) == (2500, 2000, 2)                  # a gap at 2000..2499
    smp.smp_sketch_accumulate(s.ctx, Ad[2000:2500], 64, Bd[2000:2500], 48, 2000, 500)
    assert smp.smp_sketch_coverage(s.ctx) == (3000, 3000, 1)
    smp.smp_sketch_finalize(s.ctx)
    smp.smp_sync(s.ctx)
    # the rejected blocks left the sketch untouched: it equals the oracle's over the 3,000 rows
    st = s.sketch_state()
    ref = O.sketch(A.astype(np.float64), B.astype(np.float64), 32, 1, block_rows=1000)
    rel = np.linalg.norm(st["At"].cpu().numpy() - ref.At.T) / np.linalg.norm(ref.At)
    assert rel < 2e-3
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    smp.smp_sketch_reset(s.ctx)
    assert smp.smp_sketch_coverage(s.ctx) == (0, 0, 0)
    s.close()


def test_injected_allocation_failures(env):
    torch, smp, pipeline = env
    try:
        smp.smp_debug_fail_allocs(1)                                          # the context's first allocation
        with pytest.raises(smp.SmpError) as e:
            pipeline.Solver(64, 48, 32, torch.float32, seed=1)
        assert e.value.status == smp.SMP_ENOMEM
        A, B = synth.lowrank_plus_noise(2000, 64, 48, 5, 0.1, 0.5, seed=4, dtype=np.float32)
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        s = pipeline.Solver(64, 48, 32, torch.float32, seed=1)
        s.sketch(Ad, Bd, 1000)
        smp.smp_debug_fail_allocs(1)                                          # the sampler's coin words
        with pytest.raises(smp.SmpError) as e:
            s.sample(2000.0, 2)
        assert e.value.status == smp.SMP_ENOMEM
        nnz = s.sample(2000.0, 2)                                             # retried: succeeds
        vals = s.estimate(nnz)
        smp.smp_debug_fail_allocs(1)                                          # WAltMin's scratch
        with pytest.raises(smp.SmpError) as e:
            s.waltmin(vals, 3, 4)
        assert e.value.status == smp.SMP_ENOMEM
        U, S, V = s.waltmin(vals, 3, 4)
        assert bool(torch.isfinite(S).all())
        s.close()
    finally:
        smp.smp_debug_fail_allocs(0)
