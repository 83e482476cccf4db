"""Host-side logic of the serving form: the admission charge (libsmp's smp_serve_job_bytes, a host function) and
the request generator / block interleaving of paper_1610_06656_gb300.serve. No GPU."""
import math

import numpy as np
import pytest

from paper_1610_06656_gb300 import build, serve
from paper_1610_06656_gb300 import smp as S


@pytest.fixture(scope="module")
def lib():
    S.load(build.build())
    return S


def test_job_bytes_grows_with_every_size(lib):
    base = dict(n1=1000, n2=800, k=80, r=10, T=10, m=50000.0, seed=1, sample_seed=2, walt_seed=3)
    b0 = lib.smp_serve_job_bytes(lib.job_params(**base))
    for key, val in (("n1", 2000), ("n2", 1600), ("k", 160), ("r", 20), ("m", 200000.0)):
        kw = dict(base)
        kw[key] = val
        assert lib.smp_serve_job_bytes(lib.job_params(**kw)) > b0, key
    # the sketch partials alone: 9 x (n1 + n2) x ldk x 4 bytes
    assert b0 > 9 * 1800 * 80 * 4


def test_job_bytes_rejects_bad_params(lib):
    with pytest.raises(lib.SmpError) as e:
        lib.smp_serve_job_bytes(lib.job_params(n1=0, n2=10, k=8, r=1, T=1, m=10.0, seed=1, sample_seed=2,
                                               walt_seed=3))
    assert e.value.status == lib.SMP_EINVAL


def test_poisson_arrivals_and_sizes():
    jobs = serve.poisson_jobs(4000, 200.0, seed=3, pool_rows=1_000_000)
    gaps = np.diff([0.0] + [j.arrival for j in jobs])
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.05                 # mean inter-arrival 1 / rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05             # exponential: coefficient of variation 1
    for j in jobs[:200]:
        assert 64 <= j.n <= 2048 and j.n % 8 == 0 and 10_000 <= j.d <= 500_000
        assert j.k == 8 * j.r and j.r in (5, 10, 20)
        assert j.row_offset + j.d <= 1_000_000
        assert j.m == pytest.approx(4 * j.n * j.r * math.log(j.n))


def test_round_robin_interleaves_and_retires():
    rr = serve.RoundRobin()
    rr.add(1, "a", serve.block_plan(70000, 32768))     # 3 blocks, last partial
    rr.add(2, "b", serve.block_plan(10000, 32768))     # 1 block
    p1 = rr.next_pass()
    assert [(j, b, last) for j, _, b, last in p1] == [(1, (0, 32768), False), (2, (0, 10000), True)]
    rr.add(3, "c", serve.block_plan(32768, 32768))
    p2 = rr.next_pass()
    assert [(j, b, last) for j, _, b, last in p2] == [(1, (32768, 32768), False), (3, (0, 32768), True)]
    p3 = rr.next_pass()
    assert [(j, b, last) for j, _, b, last in p3] == [(1, (65536, 4464), True)]
    assert len(rr) == 0


def test_batch_instances_and_tuner_cache(tmp_path):
    from paper_1610_06656_gb300 import batch
    specs = batch.instances(256, seed=4, pool_rows=1_000_000)
    assert len(specs) == 256 and all(s.arrival == 0.0 and s.k == 8 * s.r for s in specs)
    calls = []

    def fake(n, k, dtype, engine):          # the tensor-core engine wins from n = 512 up; SIMT cannot run k = 160;
        calls.append((n, k, engine))        # FP8 takes BF16 inputs only and wins on them from n = 1,024 up
        if engine == S.SMP_ENGINE_SIMT:
            return None if k == 160 else 1.0
        if engine == S.SMP_ENGINE_TC_FP8:
            return None if dtype != S.SMP_BF16 else (0.3 if n >= 1024 else 3.0)
        return 0.5 if n >= 512 else 2.0

    path = str(tmp_path / "tune.json")
    t = batch.EngineTuner(fake, cache_path=path)
    assert t.choose(100, 40, S.SMP_F32) == S.SMP_ENGINE_SIMT
    assert t.choose(120, 40, S.SMP_F32) == S.SMP_ENGINE_SIMT            # same bucket (128): cached
    assert t.choose(1000, 40, S.SMP_F32) == S.SMP_ENGINE_TC
    assert t.choose(100, 160, S.SMP_F32) == S.SMP_ENGINE_TC             # SIMT unavailable
    assert t.trials == 9 and len(calls) == 9                            # three candidates per shape key
    assert t.choose(1000, 40, S.SMP_BF16) == S.SMP_ENGINE_TC_FP8
    assert t.choose(200, 40, S.SMP_BF16) == S.SMP_ENGINE_SIMT           # bucket 256: FP8 and TF32 slower
    t2 = batch.EngineTuner(fake, cache_path=path)                       # reloaded from the file: no new trials
    assert t2.choose(1000, 40, S.SMP_F32) == S.SMP_ENGINE_TC and t2.trials == 0
    assert batch.n_bucket(64) == 64 and batch.n_bucket(65) == 128 and batch.n_bucket(2048) == 2048


class _FakeServer:
    """Stands in for libsmp's server calls: admits while a byte budget lasts, records the call order."""

    def __init__(self, budget):
        self.budget, self.used, self.next, self.log, self.live = budget, 0, 1, [], {}

    def admit(self, jp):
        need = int(jp.sketch.n1) * 1000
        if self.used + need > self.budget:
            return None
        jid, self.next = self.next, self.next + 1
        self.used += need
        self.live[jid] = need
        self.log.append(("admit", jid))
        return jid

    def block(self, jid, row0, nrows):
        self.log.append(("block", jid, row0, nrows))

    def close(self, jid):
        self.log.append(("close", jid))

    def collect(self, jid):
        self.used -= self.live.pop(jid)
        self.log.append(("collect", jid))
        return 7, 1.5


def test_staged_schedule_waves_and_order(monkeypatch):
    """run_staged: a wave is what the budget admits; every block of the wave is pushed (round-robin by block index)
    before the device sync, every job of the wave is closed after it, and the next wave starts after collection."""
    fake = _FakeServer(budget=2500 * 1000)
    monkeypatch.setattr(S, "smp_serve_admit", lambda sv, jp: fake.admit(jp))
    monkeypatch.setattr(S, "smp_serve_block", lambda sv, jid, a, lda, b, ldb, r0, nr: fake.block(jid, r0, nr))
    monkeypatch.setattr(S, "smp_serve_close", lambda sv, jid: fake.close(jid))
    monkeypatch.setattr(S, "smp_serve_collect", lambda sv, jid, U=None, Sv=None, V=None: fake.collect(jid))
    syncs = []
    fake_sync = lambda: (syncs.append(len(fake.log)), fake.log.append(("sync",)))   # noqa: E731

    class Pool:
        def __init__(self):
            self.shape = (1_000_000, 2048)

        def stride(self, i):
            return 2048

        def __getitem__(self, idx):
            return None

    jobs = [serve.JobSpec(i, 0.0, n, d, 5, 40, 10, 1000.0, 0, i)
            for i, (n, d) in enumerate([(1000, 70000), (1000, 10000), (1000, 40000), (800, 32768)])]
    recs, wall = serve.run_staged(None, jobs, Pool(), Pool(), S.SMP_F32, block_rows=32768, sync=fake_sync)
    assert [r["idx"] for r in recs] == [0, 1, 2, 3] and all(r["nnz"] == 7 for r in recs)
    ev = fake.log
    # wave 1: jobs 1, 2 (2,000 of the 2,500 budget; job 3 would exceed it); wave 2: jobs 3, 4
    assert [e for e in ev if e[0] == "admit"] == [("admit", 1), ("admit", 2), ("admit", 3), ("admit", 4)]
    s1, s2 = [i for i, e in enumerate(ev) if e[0] == "sync"]
    w1 = ev[:s1]
    assert [e for e in w1 if e[0] == "block"] == [("block", 1, 0, 32768), ("block", 2, 0, 10000),
                                                 ("block", 1, 32768, 32768), ("block", 1, 65536, 4464)]
    assert all(e[0] in ("admit", "block") for e in w1) and ("admit", 3) not in w1
    w1_after = ev[s1 + 1:s2]
    assert w1_after[:2] == [("close", 1), ("close", 2)] and ("collect", 2) in w1_after
    assert w1_after.index(("collect", 2)) < w1_after.index(("admit", 3))
    assert ev[-2:] == [("collect", 3), ("collect", 4)]
    assert fake.used == 0
