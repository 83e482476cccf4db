"""Batched form: many independent SMP-PCA instances of uneven n, d and r solved together on one GPU.

Every instance is a job of libsmp's server (include/smp.h, smp_serve_*) admitted at time zero: the instances'
row blocks sketch concurrently on their own streams and their solve chains overlap on the server's worker threads,
so small instances fill the device next to large ones. The sketch engine of each instance comes from an autotuner
that times one probe block of every candidate engine per (dtype, k, n bucket) through the C-ABI and keeps the
fastest. Inputs are windows of a resident pool of synthetic rows, so the instances' data never has to be
generated while the batch runs.
"""
import json
import math
import os

import numpy as np

from . import serve
from . import smp as S


def instances(count, seed, pool_rows, n_range=(64, 2048), d_range=(10_000, 500_000), ranks=(5, 10, 20), T=10,
              n_multiple=8):
    """count instances with n, d uniform in their ranges (n a multiple of n_multiple), r uniform over ranks,
    k = 8 r, m = 4 n r ln n, each a window of the pool."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = max(n_multiple, int(rng.integers(n_range[0], n_range[1] + 1)) // n_multiple * n_multiple)
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        r = min(int(rng.choice(ranks)), n)
        off = int(rng.integers(0, max(1, pool_rows - d)))
        out.append(serve.JobSpec(i, 0.0, n, d, r, 8 * r, T, 4.0 * n * r * math.log(n), off, seed * 100003 + i))
    return out


def n_bucket(n):
    """Next power of two >= n (the autotuner's shape key)."""
    return 1 << max(0, int(math.ceil(math.log2(max(1, n)))))


class EngineTuner:
    """Per (dtype, k, n bucket): time every candidate engine (CUDA cores, TF32 / BF16 tensor cores, FP8 E4M3 for
    BF16 inputs) with time_fn(n, k, dtype, engine) -> ms per block (None when the engine cannot run the shape) and
    keep the fastest. Results are cached in memory and, with
    cache_path, in a JSON file reused by later runs."""

    def __init__(self, time_fn, candidates=(S.SMP_ENGINE_SIMT, S.SMP_ENGINE_TC, S.SMP_ENGINE_TC_FP8),
                 cache_path=None):
        self.time_fn, self.candidates, self.cache_path = time_fn, tuple(candidates), cache_path
        self.cache = {}
        self.trials = 0
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = {tuple(json.loads(k)): v for k, v in json.load(f).items()}

    def key(self, n, k, dtype):
        return (int(dtype), int(k), n_bucket(n))

    def choose(self, n, k, dtype):
        key = self.key(n, k, dtype)
        if key not in self.cache:
            best, best_ms, timings = None, None, {}
            for eng in self.candidates:
                ms = self.time_fn(key[2], k, dtype, eng)
                self.trials += 1
                timings[int(eng)] = ms
                if ms is not None and (best_ms is None or ms < best_ms):
                    best, best_ms = int(eng), ms
            if best is None:
                raise RuntimeError("no sketch engine can run n=%d k=%d" % (n, k))
            self.cache[key] = {"engine": best, "ms": timings}
            if self.cache_path:
                with open(self.cache_path, "w") as f:
                    json.dump({json.dumps(list(k2)): v for k2, v in self.cache.items()}, f)
        return self.cache[key]["engine"]


def probe_timer(pool_A, pool_B, rows=32768, reps=3):
    """time_fn for EngineTuner: one context per probe, one warm block, then reps blocks timed with CUDA events."""
    import torch
    from . import pipeline

    def time_fn(n, k, dtype, engine):
        tdt = {S.SMP_F32: torch.float32, S.SMP_BF16: torch.bfloat16}[dtype]
        n = min(n, pool_A.shape[1])
        try:
            s = pipeline.Solver(n, n, k, tdt, seed=1, engine=engine, max_rows=rows)
        except S.SmpError:
            return None
        try:
            a, b = pool_A[:rows, :n], pool_B[:rows, :n]
            S.smp_sketch_accumulate(s.ctx, a, pool_A.stride(0), b, pool_B.stride(0), 0, rows)
            S.smp_sync(s.ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(reps):
                S.smp_sketch_accumulate(s.ctx, a, pool_A.stride(0), b, pool_B.stride(0), (i + 1) * rows, rows)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        except S.SmpError:
            return None
        finally:
            s.close()

    return time_fn


def run(server, specs, pool_A, pool_B, dtype, tuner, block_rows=65536, keep=None, staged=True):
    """Tune each instance's engine, then solve all instances together (every arrival at time zero). staged: the
    sketches of a budget-sized wave first, then its solve chains (serve.run_staged); otherwise the streaming
    server loop. Returns the server's per-instance records and the wall time from start to the last completion.
    keep: optional {idx: (U, S, V) device tensors} to receive those instances' factors."""
    for sp in specs:
        sp.engine = tuner.choose(sp.n, sp.k, dtype)
        sp.arrival = 0.0
    if staged:
        import torch
        return serve.run_staged(server, specs, pool_A, pool_B, dtype, block_rows=block_rows, keep=keep,
                                sync=torch.cuda.synchronize)
    return serve.run(server, specs, pool_A, pool_B, dtype, block_rows=block_rows, keep=keep)
