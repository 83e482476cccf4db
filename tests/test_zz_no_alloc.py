"""The allocation-free sketch call (smp_sketch_noalloc) against the context-based path and the CPU oracle.

Some callers hold device buffers but may not allocate device memory (a plug-in whose host framework owns the
device-memory budget, or a latency-critical loop in which cudaMalloc would synchronise the device). For them the
library offers smp_sketch_noalloc, whose scratch is a fixed array compiled into the library. This test calls it
through the C ABI twice in a row (the second call reuses the array the first one left filled) and checks each
result against smp_sketch_begin / accumulate / finalize on the same CUDA-core engine (binary32 sums in another
split order: 2e-5 per column) and against the oracle's binary64 sketch (1e-5 per column, the CUDA-core engine's
tolerance), for binary32 and BF16 inputs; an empty row range must give zeros. The file is named to be collected
last.
"""
import numpy as np
import pytest

from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests.gpu_helpers import build_lib, torch_cuda

pytestmark = pytest.mark.gpu

N1, N2, K = 200, 170, 100


def _colrel(X, Y):
    num = np.linalg.norm(X - Y, axis=1)
    den = np.maximum(np.linalg.norm(Y, axis=1), 1e-300)
    return float((num / den).max())


def _context_sketch(torch, smp, pipeline, A, B, seed, row0):
    s = pipeline.Solver(N1, N2, K, A.dtype, seed=seed, engine=smp.SMP_ENGINE_SIMT, max_rows=A.shape[0])
    smp.smp_sketch_accumulate(s.ctx, A, N1, B, N2, row0, A.shape[0])
    smp.smp_sketch_finalize(s.ctx)
    st = s.sketch_state()
    out = {k: st[k].cpu().numpy() for k in ("At", "Bt", "sA", "sB")}
    s.close()
    return out


def _oracle_sketch(A, B, seed, row0):
    """The oracle's single pass over rows [row0, row0 + rows) (Pi's columns selected by the global row index)."""
    A64 = A.float().cpu().numpy().astype(np.float64)
    B64 = B.float().cpu().numpy().astype(np.float64)
    st = O.SketchState(N1, N2, K, seed)
    st.accumulate(A64, B64, row0)
    return st


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_noalloc_sketch_matches_context_path_and_oracle_twice(dtype):
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    tdt, sdt = (torch.float32, smp.SMP_F32) if dtype == "f32" else (torch.bfloat16, smp.SMP_BF16)
    cases = [(2000, 1000, 11, 0), (1500, 77, 12, 123456)]      # (rows, data seed, Pi seed, row0)
    At = torch.empty(N1, K, dtype=torch.float32, device="cuda")
    Bt = torch.empty(N2, K, dtype=torch.float32, device="cuda")
    sA = torch.empty(N1, dtype=torch.float64, device="cuda")
    sB = torch.empty(N2, dtype=torch.float64, device="cuda")
    for rows, dseed, seed, row0 in cases:
        A, B = synth.lowrank_plus_noise(rows, N1, N2, 10, 0.1, 0.5, seed=dseed, dtype=np.float32)
        Ad, Bd = torch.from_numpy(A).cuda().to(tdt), torch.from_numpy(B).cuda().to(tdt)
        smp.smp_sketch_noalloc(Ad, N1, Bd, N2, N1, N2, K, sdt, seed, row0, rows, At, Bt, sA, sB)
        torch.cuda.synchronize()
        gA, gB = At.cpu().numpy().astype(np.float64), Bt.cpu().numpy().astype(np.float64)
        ref = _context_sketch(torch, smp, pipeline, Ad, Bd, seed, row0)
        assert _colrel(gA, ref["At"].astype(np.float64)) < 2e-5
        assert _colrel(gB, ref["Bt"].astype(np.float64)) < 2e-5
        np.testing.assert_allclose(sA.cpu().numpy(), ref["sA"], rtol=1e-13)
        np.testing.assert_allclose(sB.cpu().numpy(), ref["sB"], rtol=1e-13)
        orc = _oracle_sketch(Ad, Bd, seed, row0)
        assert _colrel(gA, orc.At.T) < 1e-5
        assert _colrel(gB, orc.Bt.T) < 1e-5
        np.testing.assert_allclose(sA.cpu().numpy(), orc.sA, rtol=1e-12)
        np.testing.assert_allclose(sB.cpu().numpy(), orc.sB, rtol=1e-12)


def test_noalloc_empty_range_gives_zeros():
    """nrows = 0 after a call that filled the scratch: the outputs are zero (the used partials are cleared)."""
    torch = torch_cuda()
    smp = build_lib()
    A, B = synth.lowrank_plus_noise(512, N1, N2, 10, 0.1, 0.5, seed=3, dtype=np.float32)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    At = torch.empty(N1, K, dtype=torch.float32, device="cuda")
    Bt = torch.empty(N2, K, dtype=torch.float32, device="cuda")
    sA = torch.empty(N1, dtype=torch.float64, device="cuda")
    sB = torch.empty(N2, dtype=torch.float64, device="cuda")
    smp.smp_sketch_noalloc(Ad, N1, Bd, N2, N1, N2, K, smp.SMP_F32, 5, 0, 512, At, Bt, sA, sB)
    smp.smp_sketch_noalloc(Ad, N1, Bd, N2, N1, N2, K, smp.SMP_F32, 5, 0, 0, At, Bt, sA, sB)
    torch.cuda.synchronize()
    assert not At.any() and not Bt.any() and not sA.any() and not sB.any()


def test_noalloc_rejects_shapes_beyond_its_scratch():
    torch = torch_cuda()
    smp = build_lib()
    # small real buffers; the size checks reject the calls before anything is launched or dereferenced
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(smp.SmpError) as e:
        smp.smp_sketch_noalloc(buf, 20000, buf, 20000, 20000, 20000, 1024, smp.SMP_F32, 1, 0, 10, buf, buf, buf, buf)
    assert e.value.status == smp.SMP_EINVAL
    assert "scratch" in smp.smp_last_error()
    with pytest.raises(smp.SmpError) as e:   # n1 beyond 2^30: rejected before any size arithmetic
        smp.smp_sketch_noalloc(buf, 1 << 31, buf, 16, 1 << 31, 16, 16, smp.SMP_F32, 1, 0, 10, buf, buf, buf, buf)
    assert e.value.status == smp.SMP_EINVAL
