"""The serving form on the GPU: a job's factors are the same bits alone, in a mix of interleaved jobs and through
the plain pipeline, and within the stated tolerance of the CPU oracle's; admission by budget, cancellation and
collection. The batched form: one instance bit-equal to the plain pipeline and within tolerance of the oracle."""
import numpy as np
import pytest
import torch

from oracle import smp as O
from paper_1610_06656_gb300 import serve, synth
from tests.gpu_helpers import build_lib, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(300_000, 512, 512, 20, 0.1, 0.5, seed=1004, device="cuda",
                                                   dtype=torch.bfloat16)
    return smp, pipeline, A.contiguous(), B.contiguous()


def _factors(n, r):
    return (torch.empty(n, r, dtype=torch.float64, device="cuda"), torch.empty(r, dtype=torch.float64, device="cuda"),
            torch.empty(n, r, dtype=torch.float64, device="cuda"))


def _oracle_check(spec, A, B, factors, tol, block_rows):
    """The job's window through the CPU oracle (binary64, on the stored values, the job's seeds): Omega's size must
    match and the spectral error of the served factors must be within tol of the oracle's."""
    a = A[spec.row_offset:spec.row_offset + spec.d, :spec.n].float().cpu().numpy().astype(np.float64)
    b = B[spec.row_offset:spec.row_offset + spec.d, :spec.n].float().cpu().numpy().astype(np.float64)
    ref = O.smp_pca(a, b, spec.r, spec.k, spec.m, spec.T, seed=2 * spec.seed + 1, sample_seed=2 * spec.seed + 2,
                    block_rows=block_rows)
    M = a.T @ b
    U, S, V = (x.cpu().numpy() for x in factors)
    e_gpu = O.spectral_error(M, U, S, V)
    e_ref = O.spectral_error(M, ref["U"], ref["S"], ref["V"])
    assert abs(e_gpu - e_ref) <= tol, (e_gpu, e_ref)
    return ref


def _jobs(count, seed):
    return serve.poisson_jobs(count, 2000.0, seed, pool_rows=300_000, n_range=(64, 512), d_range=(10_000, 120_000))


def test_alone_mixed_and_plain_agree(env):
    smp, pipeline, A, B = env
    jobs = _jobs(12, seed=7)
    probe = jobs[5]
    sv = smp.smp_serve_create(8 << 30, solve_workers=3)
    try:
        alone = {probe.idx: _factors(probe.n, probe.r)}
        recs, _ = serve.run(sv, [probe], A, B, smp.SMP_BF16, keep=alone)
        assert len(recs) == 1
        mixed = {probe.idx: _factors(probe.n, probe.r)}
        recs, _ = serve.run(sv, jobs, A, B, smp.SMP_BF16, keep=mixed)
        assert sorted(r["idx"] for r in recs) == list(range(12))
        assert all(r["latency_ms"] > 0 for r in recs)
    finally:
        smp.smp_serve_destroy(sv)
    for a, b in zip(alone[probe.idx], mixed[probe.idx]):
        assert torch.equal(a, b)
    # the served job against the oracle on its stored BF16 values: BF16 sketch tolerance
    _oracle_check(probe, A, B, mixed[probe.idx], 3e-3, 32768)
    # the same job through the plain pipeline (one context on torch's stream): the same bits again
    s = pipeline.Solver(probe.n, probe.n, probe.k, torch.bfloat16, seed=2 * probe.seed + 1, max_rows=32768)
    a = A[probe.row_offset:probe.row_offset + probe.d, :probe.n]
    b = B[probe.row_offset:probe.row_offset + probe.d, :probe.n]
    out = s.solve(a, b, probe.r, probe.T, m=probe.m, sample_seed=2 * probe.seed + 2, walt_seed=2 * probe.seed + 3,
                  block_rows=32768)
    for got, key in zip(alone[probe.idx], ("U", "S", "V")):
        assert torch.equal(got, out[key])
    s.close()


def test_admission_by_budget(env):
    smp, pipeline, A, B = env
    j = _jobs(1, seed=3)[0]
    need = smp.smp_serve_job_bytes(j.params(smp.SMP_BF16))
    sv = smp.smp_serve_create(int(need * 1.5), solve_workers=1)
    try:
        first = smp.smp_serve_admit(sv, j.params(smp.SMP_BF16))
        assert first is not None
        assert smp.smp_serve_admit(sv, j.params(smp.SMP_BF16)) is None          # SMP_EBUSY
        used, live = smp.smp_serve_stats(sv)
        assert used == need and live == 1
        smp.smp_serve_cancel(sv, first)
        assert smp.smp_serve_stats(sv) == (0, 0)
        second = smp.smp_serve_admit(sv, j.params(smp.SMP_BF16))
        assert second is not None
        for r0, nr in serve.block_plan(j.d, 32768):
            a = A[j.row_offset + r0:j.row_offset + r0 + nr, :j.n]
            b = B[j.row_offset + r0:j.row_offset + r0 + nr, :j.n]
            smp.smp_serve_block(sv, second, a, A.stride(0), b, B.stride(0), r0, nr)
        smp.smp_serve_close(sv, second)
        with pytest.raises(smp.SmpError) as e:                                   # closed: no more blocks
            smp.smp_serve_block(sv, second, a, A.stride(0), b, B.stride(0), 0, 16)
        assert e.value.status == smp.SMP_ESTATE
        nnz, lat = smp.smp_serve_collect(sv, second)
        assert nnz > 0 and lat > 0
        assert smp.smp_serve_stats(sv) == (0, 0)
    finally:
        smp.smp_serve_destroy(sv)


def test_cancel_streaming_and_queued_jobs(env):
    smp, pipeline, A, B = env
    jobs = _jobs(3, seed=11)
    sv = smp.smp_serve_create(8 << 30, solve_workers=1)
    try:
        ids = [smp.smp_serve_admit(sv, j.params(smp.SMP_BF16)) for j in jobs]
        j0 = jobs[0]
        a = A[j0.row_offset:j0.row_offset + 1024, :j0.n]
        b = B[j0.row_offset:j0.row_offset + 1024, :j0.n]
        smp.smp_serve_block(sv, ids[0], a, A.stride(0), b, B.stride(0), 0, 1024)
        smp.smp_serve_cancel(sv, ids[0])                                         # streaming
        for jid, j in zip(ids[1:], jobs[1:]):
            for r0, nr in serve.block_plan(j.d, 32768):
                smp.smp_serve_block(sv, jid, A[j.row_offset + r0:j.row_offset + r0 + nr, :j.n], A.stride(0),
                                    B[j.row_offset + r0:j.row_offset + r0 + nr, :j.n], B.stride(0), r0, nr)
            smp.smp_serve_close(sv, jid)
        smp.smp_serve_cancel(sv, ids[2])                                         # queued or solving
        nnz, lat = smp.smp_serve_collect(sv, ids[1])
        assert nnz > 0
        with pytest.raises(smp.SmpError):
            smp.smp_serve_poll(sv, ids[2])                                       # gone
        assert smp.smp_serve_stats(sv) == (0, 0)
    finally:
        smp.smp_serve_destroy(sv)


def test_batch_matches_single_instance(env):
    """Eight uneven instances solved together with autotuned engines: one of them equals, bit for bit, the same
    instance through the plain pipeline with the engine the tuner chose."""
    smp, pipeline, A, B = env
    from paper_1610_06656_gb300 import batch
    A32, B32 = A.float(), B.float()
    specs = batch.instances(8, seed=13, pool_rows=300_000, n_range=(64, 512), d_range=(10_000, 150_000))
    tuner = batch.EngineTuner(batch.probe_timer(A32, B32))
    probe = specs[3]
    keep = {probe.idx: _factors(probe.n, probe.r)}
    sv = smp.smp_serve_create(16 << 30, solve_workers=4)
    try:
        recs, wall = batch.run(sv, specs, A32, B32, smp.SMP_F32, tuner, block_rows=65536, keep=keep)
    finally:
        smp.smp_serve_destroy(sv)
    assert sorted(r["idx"] for r in recs) == list(range(8)) and wall > 0
    s = pipeline.Solver(probe.n, probe.n, probe.k, torch.float32, seed=2 * probe.seed + 1, engine=probe.engine,
                        max_rows=65536)
    out = s.solve(A32[probe.row_offset:probe.row_offset + probe.d, :probe.n],
                  B32[probe.row_offset:probe.row_offset + probe.d, :probe.n], probe.r, probe.T, m=probe.m,
                  sample_seed=2 * probe.seed + 2, walt_seed=2 * probe.seed + 3, block_rows=65536)
    for got, key in zip(keep[probe.idx], ("U", "S", "V")):
        assert torch.equal(got, out[key])
    s.close()
    # the batched instance against the oracle: the tuner's engine for FP32 inputs is the TF32 one (1e-3)
    _oracle_check(probe, A32, B32, keep[probe.idx], 1e-3, 65536)


def test_collect_timeout_and_destroy_with_live_jobs(env):
    """A zero timeout on a job whose chain cannot have finished returns SMP_ETIMEOUT and keeps the job; destroying
    the server with streaming, queued and finished jobs releases them all."""
    smp, pipeline, A, B = env
    jobs = _jobs(3, seed=17)
    sv = smp.smp_serve_create(8 << 30, solve_workers=1)
    try:
        ids = [smp.smp_serve_admit(sv, j.params(smp.SMP_BF16)) for j in jobs]
        for jid, j in zip(ids[:2], jobs[:2]):
            for r0, nr in serve.block_plan(j.d, 32768):
                smp.smp_serve_block(sv, jid, A[j.row_offset + r0:j.row_offset + r0 + nr, :j.n], A.stride(0),
                                    B[j.row_offset + r0:j.row_offset + r0 + nr, :j.n], B.stride(0), r0, nr)
        smp.smp_serve_close(sv, ids[0])              # both closed back to back: job 1 queues behind job 0's chain
        smp.smp_serve_close(sv, ids[1])
        with pytest.raises(smp.SmpError) as e:       # one worker, two chains of milliseconds each: not done yet
            smp.smp_serve_collect(sv, ids[1], timeout_s=0.0)
        assert e.value.status == smp.SMP_ETIMEOUT
        assert smp.smp_serve_stats(sv)[1] == 3
        with pytest.raises(smp.SmpError) as e:        # streaming job: nothing to collect yet
            smp.smp_serve_collect(sv, ids[2])
        assert e.value.status == smp.SMP_ESTATE
    finally:
        smp.smp_serve_destroy(sv)
