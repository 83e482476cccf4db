"""Test infrastructure: the CPU oracle's single pass at the benchmark's sizes.

Only the oracle's own functions compute here: `oracle.philox.pi_block` draws each row block's Pi (binary64, the
specified Philox stream) and `oracle.smp.SketchState.accumulate` adds the block's contribution, exactly as
`oracle.smp.sketch` does; this module only schedules them. Pi's Philox blocks are the oracle's slowest step
(single-threaded numpy), so a pool of *spawned* worker processes draws them (spawned, not forked: the parent has
already initialised CUDA) while the parent folds the blocks in, one at a time, in row order; the row blocks
themselves are fetched one at a time through a callback, so the d x n inputs never need to sit on the host whole.
"""
import multiprocessing as mp
import os

import numpy as np

from oracle import philox
from oracle import smp as O


def _pi_job(job):
    seed, k, row0, nrows = job
    return philox.pi_block(seed, k, row0, nrows)


def host_workers():
    return max(1, min(12, len(os.sched_getaffinity(0)) - 2))


class PiPool:
    """Spawned worker processes drawing the oracle's Pi blocks (Philox + Box-Muller, binary64)."""

    def __init__(self, workers=None):
        self.pool = mp.get_context("spawn").Pool(workers or host_workers())

    def blocks(self, seed, k, starts, nrows_of):
        """Pi[:, r0:r0 + nrows] for each r0 in starts, in order (drawn ahead by the workers)."""
        return self.pool.imap(_pi_job, [(seed, k, r0, nrows_of(r0)) for r0 in starts])

    def close(self):
        self.pool.close()
        self.pool.join()


def sketch_stream(fetch, d, n1, n2, k, seed, block_rows, same_ab=False, pool=None):
    """The oracle's single pass over rows [0, d) in blocks of block_rows rows: fetch(r0, r1) -> (A_blk, B_blk) as
    host arrays (B_blk ignored when same_ab). Returns the oracle's SketchState."""
    st = O.SketchState(n1, n2, k, seed, same_ab)
    starts = list(range(0, d, block_rows))
    own = pool is None
    pool = pool or PiPool()
    try:
        for r0, P in zip(starts, pool.blocks(seed, k, starts, lambda r: min(d, r + block_rows) - r)):
            r1 = min(d, r0 + block_rows)
            A_blk, B_blk = fetch(r0, r1)
            A64 = np.asarray(A_blk, dtype=np.float64)
            B64 = None if same_ab else np.asarray(B_blk, dtype=np.float64)
            st.accumulate(A64, B64, r0, pi_blk=P)
    finally:
        if own:
            pool.close()
    return st


def solve_from_state(st, m, r, T, sample_seed):
    """Steps 3-5 of Algorithm 1 on the oracle's finalized single pass (as oracle.smp.smp_pca does after sketch())."""
    rows, cols, qhat = O.sample_omega(st.sA, st.sB, m, sample_seed)
    vals = O.estimate(rows, cols, st.At, st.Bt, st.sA, st.sB)
    Uh, Vh = O.waltmin(st.n1, st.n2, rows, cols, vals, qhat, r, T, st.sA)
    U, S, V = O.canonical(Uh, Vh)
    return dict(rows=rows, cols=cols, qhat=qhat, vals=vals, U=U, S=S, V=V)
