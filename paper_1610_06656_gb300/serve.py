"""Serving form on top of libsmp's server (include/smp.h, smp_serve_*): Poisson job arrivals, interleaved row
blocks, admission by the server's memory budget, latency from a job's last block to its factors.

The scheduling here is host logic only (which job pushes which block when); every computation runs in libsmp.
Job inputs are windows of a shared pool of synthetic rows (A and B drawn from one low-rank-plus-noise model with
the pool's full width), so no input is generated inside a timed region.
"""
import collections
import math
import time

import numpy as np

from . import smp as S


class JobSpec:
    """One request: sizes, seeds, arrival time (seconds from the start) and its window of the input pool."""

    def __init__(self, idx, arrival, n, d, r, k, T, m, row_offset, seed, engine=None):
        self.idx, self.arrival, self.n, self.d, self.r, self.k, self.T = idx, arrival, n, d, r, k, T
        self.m, self.row_offset, self.seed, self.engine = m, row_offset, seed, engine

    def params(self, dtype, engine=S.SMP_ENGINE_AUTO, block_rows=32768):
        """Job parameters; the job's own engine (set by an autotuner) wins over the run's."""
        eng = engine if self.engine is None else self.engine
        return S.job_params(self.n, self.n, self.k, self.r, self.T, self.m, seed=2 * self.seed + 1,
                            sample_seed=2 * self.seed + 2, walt_seed=2 * self.seed + 3, dtype=dtype, engine=eng,
                            max_rows=block_rows)


def poisson_jobs(count, rate, seed, pool_rows, n_range=(64, 2048), d_range=(10_000, 500_000), ranks=(5, 10, 20),
                 T=10, n_multiple=8):
    """count jobs with exponential inter-arrival times (rate per second); n and d uniform in their ranges (n rounded
    down to a multiple of n_multiple), r uniform over ranks, k = 8 r, m = 4 n r ln n; row windows inside the pool."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.integers(n_range[0], n_range[1] + 1)) // n_multiple * n_multiple
        n = max(n, n_multiple)
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        r = int(rng.choice(ranks))
        r = min(r, n)
        off = int(rng.integers(0, max(1, pool_rows - d)))
        jobs.append(JobSpec(i, t, n, d, r, 8 * r, T, 4.0 * n * r * math.log(n), off, seed * 100003 + i))
    return jobs


def block_plan(d, block_rows):
    """Row blocks (row0, nrows) of one job, in order."""
    return [(r0, min(block_rows, d - r0)) for r0 in range(0, d, block_rows)]


class RoundRobin:
    """Interleaves the blocks of the active jobs: each pass gives every active job its next block."""

    def __init__(self):
        self.active = collections.OrderedDict()   # job id -> (spec, remaining blocks deque)

    def add(self, jid, spec, blocks):
        self.active[jid] = (spec, collections.deque(blocks))

    def next_pass(self):
        """[(job id, spec, (row0, nrows), is_last)] for one pass; finished jobs leave the rotation."""
        out = []
        for jid in list(self.active):
            spec, q = self.active[jid]
            blk = q.popleft()
            last = not q
            out.append((jid, spec, blk, last))
            if last:
                del self.active[jid]
        return out

    def __len__(self):
        return len(self.active)


def run(server, jobs, pool_A, pool_B, dtype, block_rows=32768, engine=S.SMP_ENGINE_AUTO, keep=None,
        time_limit=600.0):
    """Drive the server through the jobs (arrival times honoured). Returns per-job records
    {idx, latency_ms, nnz, done_at} in completion order and the wall time from the first arrival to the last
    completion. keep: optional {idx: (U, S, V) device tensors} to receive those jobs' factors."""
    pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
    rr = RoundRobin()
    closed = {}
    records = []
    lda = pool_A.stride(0)
    t0 = time.perf_counter()
    while pending or len(rr) or closed:
        now = time.perf_counter() - t0
        if now > time_limit:
            raise RuntimeError("serving run exceeded %.0f s" % time_limit)
        while pending and pending[0].arrival <= now:
            spec = pending[0]
            jid = S.smp_serve_admit(server, spec.params(dtype, engine, block_rows))
            if jid is None:        # over budget: retry after collections free memory
                break
            pending.popleft()
            rr.add(jid, spec, block_plan(spec.d, block_rows))
        for jid, spec, (r0, nr), last in rr.next_pass():
            a = pool_A[spec.row_offset + r0: spec.row_offset + r0 + nr, :spec.n]
            b = pool_B[spec.row_offset + r0: spec.row_offset + r0 + nr, :spec.n]
            S.smp_serve_block(server, jid, a, lda, b, lda, r0, nr)
            if last:
                S.smp_serve_close(server, jid)
                closed[jid] = spec
        for jid in list(closed):
            if S.smp_serve_poll(server, jid):
                spec = closed.pop(jid)
                U = Sv = V = None
                if keep is not None and spec.idx in keep:
                    U, Sv, V = keep[spec.idx]
                nnz, lat = S.smp_serve_collect(server, jid, U, Sv, V)
                records.append(dict(idx=spec.idx, latency_ms=lat, nnz=nnz, done_at=time.perf_counter() - t0))
        if not len(rr):
            wait = (pending[0].arrival - (time.perf_counter() - t0)) if pending else 0.0
            time.sleep(min(max(wait, 0.0), 0.0005) if closed or pending else 0.0)
    first = min(j.arrival for j in jobs) if jobs else 0.0
    wall = (max(r["done_at"] for r in records) - first) if records else 0.0
    return records, wall


def run_staged(server, jobs, pool_A, pool_B, dtype, block_rows=32768, engine=S.SMP_ENGINE_AUTO, keep=None,
               time_limit=600.0, sync=None):
    """Batched schedule, stage by stage: admit as many jobs as the budget takes (a wave), push every block of the
    wave (all sketches run concurrently), wait until the device has finished them (sync()), then close the whole
    wave so the server's workers run the solve chains without sketch kernels queued in front of them on the
    device's hardware queues; collect, then the next wave. Returns records and wall time like run()."""
    pending = collections.deque(jobs)
    records = []
    lda = pool_A.stride(0)
    t0 = time.perf_counter()
    phases = {"sketch_s": 0.0, "solve_s": 0.0, "waves": 0}
    while pending:
        if time.perf_counter() - t0 > time_limit:
            raise RuntimeError("batched run exceeded %.0f s" % time_limit)
        wave = []
        while pending:
            jid = S.smp_serve_admit(server, pending[0].params(dtype, engine, block_rows))
            if jid is None:
                break
            wave.append((jid, pending.popleft()))
        if not wave:
            raise RuntimeError("a single job does not fit the server's memory budget")
        phases["waves"] += 1
        tw = time.perf_counter()
        plans = [block_plan(spec.d, block_rows) for _, spec in wave]
        for p in range(max(len(pl) for pl in plans)):
            for (jid, spec), pl in zip(wave, plans):
                if p < len(pl):
                    r0, nr = pl[p]
                    a = pool_A[spec.row_offset + r0: spec.row_offset + r0 + nr, :spec.n]
                    b = pool_B[spec.row_offset + r0: spec.row_offset + r0 + nr, :spec.n]
                    S.smp_serve_block(server, jid, a, lda, b, lda, r0, nr)
        if sync is not None:
            sync()
        ts = time.perf_counter()
        phases["sketch_s"] += ts - tw
        for jid, _ in wave:
            S.smp_serve_close(server, jid)
        for jid, spec in wave:
            U = Sv = V = None
            if keep is not None and spec.idx in keep:
                U, Sv, V = keep[spec.idx]
            nnz, lat = S.smp_serve_collect(server, jid, U, Sv, V)
            records.append(dict(idx=spec.idx, latency_ms=lat, nnz=nnz, done_at=time.perf_counter() - t0))
        phases["solve_s"] += time.perf_counter() - ts
    wall = max(r["done_at"] for r in records) if records else 0.0
    run_staged.last_phases = phases
    return records, wall

