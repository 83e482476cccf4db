"""Failure paths, made on the host (no GPU fault): duplicated or overlapping row blocks are rejected before
anything is launched, coverage reports what has been sketched, injected device-allocation failures surface as
SMP_ENOMEM with the context still usable or destroyable, and a bounded device-side wait that runs out (a stage
whose loads are never issued, so nothing ever completes its barrier) ends the kernel with SMP_ETIMEOUT instead of a
hang, after which the same context sketches correctly again."""
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


@pytest.mark.parametrize("engine,n1,n2", [("tc", 200, 136), ("tc_bf16", 200, 136), ("tc", 512, 512),
                                          ("tc_bf16", 640, 520)])
def test_bounded_wait_runs_out(env, engine, n1, n2):
    """The tensor-core kernel with a 1 ms wait limit and the data loads of stage 3 never issued: its waits on that
    stage give up, the error word reports the timeout (SMP_ETIMEOUT from smp_sync), and a normal sketch on the same
    context afterwards matches the oracle; on 4 to 10 column tiles."""
    torch, smp, pipeline = env
    eng = {"tc": smp.SMP_ENGINE_TC, "tc_bf16": smp.SMP_ENGINE_TC_BF16}[engine]
    tol = 2e-3 if engine == "tc" else 1e-2
    A, B = synth.lowrank_plus_noise(1024, n1, n2, 5, 0.1, 0.5, seed=6, dtype=np.float32)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    s = pipeline.Solver(n1, n2, 64, torch.float32, seed=1, engine=eng, max_rows=1024)
    try:
        smp.smp_debug_tc_wait(1_000_000, 3)
        smp.smp_sketch_reset(s.ctx)
        smp.smp_sketch_accumulate(s.ctx, Ad, n1, Bd, n2, 0, 1024)
        with pytest.raises(smp.SmpError) as e:
            smp.smp_sync(s.ctx)
        assert e.value.status == smp.SMP_ETIMEOUT
        assert "wait" in smp.smp_last_error(s.ctx)
    finally:
        smp.smp_debug_tc_wait(0, -1)
    smp.smp_sync(s.ctx)                                                       # the error word was cleared
    s.sketch(Ad, Bd, 1024)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    ref = O.sketch(A, B, 64, 1, block_rows=1024)
    num = np.linalg.norm(st["At"].cpu().numpy() - ref.At.T, axis=1)
    assert float((num / np.linalg.norm(ref.At.T, axis=1)).max()) < tol
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-12)
    s.close()


def test_host_block_accumulate_matches_device_blocks(env):
    """smp_sketch_accumulate_host (row blocks in pinned and in pageable host memory, staged through the context's two
    device buffers) gives the same bits as smp_sketch_accumulate on the same blocks already on the device."""
    torch, smp, pipeline = env
    A, B = synth.lowrank_plus_noise(5000, 200, 136, 5, 0.1, 0.5, seed=8, dtype=np.float32)
    out = []
    for mode in ("device", "pinned", "pageable"):
        s = pipeline.Solver(200, 136, 96, torch.float32, seed=3, max_rows=2048)
        smp.smp_sketch_reset(s.ctx)
        Ah, Bh = torch.from_numpy(A), torch.from_numpy(B)
        if mode == "pinned":
            Ah, Bh = Ah.pin_memory(), Bh.pin_memory()
        for r0 in (2048, 0, 4096):
            r1 = min(5000, r0 + 2048)
            if mode == "device":
                smp.smp_sketch_accumulate(s.ctx, Ah[r0:r1].cuda(), 200, Bh[r0:r1].cuda(), 136, r0, r1 - r0)
                torch.cuda.synchronize()
            else:
                smp.smp_sketch_accumulate_host(s.ctx, Ah[r0:r1], 200, Bh[r0:r1], 136, r0, r1 - r0)
        smp.smp_sketch_finalize(s.ctx)
        smp.smp_sync(s.ctx)
        st = s.sketch_state()
        out.append({k: st[k].cpu() for k in ("At", "Bt", "sA", "sB")})
        s.close()
    for other in out[1:]:
        for k in ("At", "Bt", "sA", "sB"):
            assert torch.equal(out[0][k], other[k]), k
