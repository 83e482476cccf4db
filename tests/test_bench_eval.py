"""bench.py's spectral-error evaluators on CPU tensors against dense numpy SVDs (evaluation code, no GPU): the
blockwise one used on the scale workloads and the implicit one used where A^T A is too large to form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from paper_1610_06656_gb300 import synth  # noqa: E402


def _dense(M, U, S, V):
    return np.linalg.norm(M - (U * S) @ V.T, 2) / np.linalg.norm(M, 2)


def test_blockwise_error_matches_dense():
    A, B = synth.lowrank_plus_noise(700, 60, 50, 5, 0.1, 0.5, seed=3, dtype=np.float32)
    rng = np.random.default_rng(1)
    U, V = rng.standard_normal((60, 4)), rng.standard_normal((50, 4))
    S = np.abs(rng.standard_normal(4)) * 50
    errs, opt = bench.spectral_error(torch, torch.from_numpy(A), torch.from_numpy(B),
                                     [(torch.from_numpy(U), torch.from_numpy(S), torch.from_numpy(V))], block=256)
    M = A.astype(np.float64).T @ B.astype(np.float64)
    sv = np.linalg.svd(M, compute_uv=False)
    assert abs(opt - sv[4] / sv[0]) < 1e-6
    assert abs(errs[0] - _dense(M, U, S, V)) < 1e-6 * max(1.0, errs[0])


def test_implicit_error_matches_dense_on_gd():
    n, r = 400, 5
    A = synth.gd(n, n, seed=11).astype(np.float32)
    M = A.astype(np.float64).T @ A.astype(np.float64)
    w, Q = np.linalg.eigh(M)
    top = np.argsort(w)[::-1][:r]
    near = (Q[:, top], w[top] * (1 + 1e-3), Q[:, top])            # close to the optimum: a small residual
    rng = np.random.default_rng(2)
    far = (rng.standard_normal((n, r)), np.abs(rng.standard_normal(r)), rng.standard_normal((n, r)))
    factors = [tuple(torch.from_numpy(np.ascontiguousarray(x)) for x in f) for f in (near, far)]
    errs, opt = bench.implicit_errors(torch, torch.from_numpy(A), factors, r)
    sv = np.sort(np.abs(w))[::-1]
    assert abs(opt - sv[r] / sv[0]) <= 1e-4 * sv[r] / sv[0]
    for f, e in zip((near, far), errs):
        want = _dense(M, *f)
        assert abs(e - want) <= 1e-3 * want
