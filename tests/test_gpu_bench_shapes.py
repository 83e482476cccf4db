"""Parity against the CPU binary64 oracle at the benchmark's shapes and launch configuration.

bench.py times contexts of max_rows = 65,536 fed one 65,536-row block per smp_sketch_accumulate call. These tests
run exactly that configuration and compare with the oracle (never with another GPU engine):

1. One full 65,536-row block per tensor-core engine. Scale shape (n1 = n2 = 2,000, k = 500: two N = 256 Pi boxes,
   512 TMEM columns): the TF32 engine within 2e-3 per sketch column, the BF16-operand engine within 1e-2.
   Precision shape (n1 = n2 = 4,096, k = 1,024: the sketch rows split over two CTAs): BF16 within 1e-2; FP8 within
   2e-3 of the quantised model (the oracle's Pi and the block rounded to E4M3 on the host) and within 8e-2 of the
   exact oracle. Column norms: compensated binary32 sums of the unrounded inputs (TwoSum plus the FMA residual, the
   low parts summed in binary32) over R rows carry a relative error of at most about R u^2 (u = 2^-24); with
   R <= 16,384 rows per accumulator (a 65,536-row block in 4 row splits) that is 6e-11: 1e-10 for every engine.
2. The scale workload end to end at full size (d = 1,000,000 in 16 blocks, the last one ragged), and its A = B
   (PCA) case: Omega bit-exact against the oracle run on the same bytes (so the compensated norms summed over 16
   blocks and the row splits flip no coin), every sketch column within 2e-3, relative spectral error within 1e-3
   of the oracle's.
3. The precision workload on its d = 200,000 row prefix (BF16 stored): Omega bit-exact; the spectral error of the
   BF16 path within 3e-3 and of the FP8 path within 1e-2 of the oracle's.

The tolerances per engine are the ones their operand rounding gives (TF32: unit roundoff 2^-11 on both operands;
BF16: 2^-9; E4M3: 2^-4 per operand, i.e. a few per cent per column against the exact product). The spectral
errors of both sides are evaluated against the same binary64 A^T B (blockwise binary32 products without TF32,
summed in binary64, on the GPU through torch: evaluation only). The oracle's Pi blocks are drawn by spawned worker
processes (tests/oracle_stream.py); only oracle functions compute them.
"""
import numpy as np
import pytest

from oracle import philox as P
from oracle import smp as O
from paper_1610_06656_gb300 import synth
from tests import oracle_stream as OS
from tests.gpu_helpers import build_lib, csr_rows, omega_numpy, torch_cuda

pytestmark = pytest.mark.gpu

BLOCK = 65536
SCALE = dict(d=1_000_000, n=2000, L=20, sigma=0.1, alpha=0.5, k=500, r=10, T=10, seed=1001)
PREC = dict(d=200_000, n=4096, L=32, sigma=0.05, alpha=0.7, k=1024, r=20, T=15, seed=1002)


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    smp = build_lib()
    from paper_1610_06656_gb300 import pipeline
    return torch, smp, pipeline


@pytest.fixture(scope="module")
def pool():
    p = OS.PiPool()
    yield p
    p.close()


def _colrel(X, Y):
    num = np.linalg.norm(X - Y, axis=1)
    den = np.maximum(np.linalg.norm(Y, axis=1), 1e-300)
    return float((num / den).max())


def _host(t):
    return t.float().cpu().numpy()


def _product(torch, A, B):
    """A^T B in binary64 from binary32 block products (TF32 off): the evaluation reference of both sides."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    M = torch.zeros(A.shape[1], B.shape[1], dtype=torch.float64, device=A.device)
    for r0 in range(0, A.shape[0], BLOCK):
        M += (A[r0:r0 + BLOCK].float().T @ B[r0:r0 + BLOCK].float()).double()
    torch.backends.cuda.matmul.allow_tf32 = prev
    return M


def _errors(torch, M, factors):
    """||M - U S V^T||_2 / ||M||_2 for each (U, S, V) (numpy or torch, binary64) and the Eckart-Young optimum."""
    sv = torch.linalg.svdvals(M)
    out = []
    for U, S, V in factors:
        U, S, V = (torch.as_tensor(np.asarray(x) if not torch.is_tensor(x) else x, dtype=torch.float64,
                                   device=M.device) for x in (U, S, V))
        out.append(float(torch.linalg.matrix_norm(M - (U * S) @ V.T, ord=2) / sv[0]))
    return out, sv


# ------------------------------------------------------------------------------------------------------ one block
@pytest.fixture(scope="module")
def scale_block(env, pool):
    """The scale workload's first 65,536-row block on the device and the oracle's single pass over it."""
    torch, _, _ = env
    w = SCALE
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(BLOCK, w["n"], w["n"], w["L"], w["sigma"], w["alpha"],
                                                  seed=w["seed"], device="cuda")
    torch.cuda.synchronize()
    ref = OS.sketch_stream(lambda r0, r1: (_host(A[r0:r1]), _host(B[r0:r1])), BLOCK, w["n"], w["n"], w["k"], 1,
                           BLOCK, pool=pool)
    return A, B, ref


@pytest.mark.parametrize("engine,tol", [("tc", 2e-3), ("tc_bf16", 1e-2)])
def test_scale_block_matches_oracle(env, scale_block, engine, tol):
    torch, smp, pipeline = env
    A, B, ref = scale_block
    w = SCALE
    eng = {"tc": smp.SMP_ENGINE_TC, "tc_bf16": smp.SMP_ENGINE_TC_BF16}[engine]
    s = pipeline.Solver(w["n"], w["n"], w["k"], torch.float32, seed=1, engine=eng, max_rows=BLOCK)
    s.sketch(A, B, BLOCK)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    assert _colrel(st["At"].cpu().numpy().astype(np.float64), ref.At.T) < tol
    assert _colrel(st["Bt"].cpu().numpy().astype(np.float64), ref.Bt.T) < tol
    np.testing.assert_allclose(st["sA"].cpu().numpy(), ref.sA, rtol=1e-10)
    np.testing.assert_allclose(st["sB"].cpu().numpy(), ref.sB, rtol=1e-10)
    s.close()


@pytest.fixture(scope="module")
def precision_block(env, pool):
    """The precision workload's first 65,536-row block (BF16 stored) and the oracle's pass over the stored values."""
    torch, _, _ = env
    w = PREC
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(BLOCK, w["n"], w["n"], w["L"], w["sigma"], w["alpha"],
                                                  seed=w["seed"], device="cuda", dtype=torch.bfloat16)
    torch.cuda.synchronize()
    ref = OS.sketch_stream(lambda r0, r1: (_host(A[r0:r1]), _host(B[r0:r1])), BLOCK, w["n"], w["n"], w["k"], 1,
                           BLOCK, pool=pool)
    return A, B, ref


def _sketch_bf16(env, A, B, engine):
    torch, smp, pipeline = env
    w = PREC
    s = pipeline.Solver(w["n"], w["n"], w["k"], torch.bfloat16, seed=1, engine=engine, max_rows=BLOCK)
    s.sketch(A, B, BLOCK)
    smp.smp_sync(s.ctx)
    st = s.sketch_state()
    out = {key: st[key].cpu().numpy().astype(np.float64) for key in ("At", "Bt", "sA", "sB")}
    s.close()
    return out


def test_precision_block_bf16_matches_oracle(env, precision_block):
    torch, smp, _ = env
    A, B, ref = precision_block
    g = _sketch_bf16(env, A, B, smp.SMP_ENGINE_TC)
    assert _colrel(g["At"], ref.At.T) < 1e-2
    assert _colrel(g["Bt"], ref.Bt.T) < 1e-2
    np.testing.assert_allclose(g["sA"], ref.sA, rtol=1e-10)
    np.testing.assert_allclose(g["sB"], ref.sB, rtol=1e-10)


def _e4m3(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.float8_e4m3fn).float().numpy() \
        .astype(np.float64)


def _pow2_scale(X):
    """2^ceil(log2(max|X| / 448)), the engine's per-block scale (1 for an all-zero block)."""
    amax = float(np.abs(X).max()) if X.size else 0.0
    if amax == 0.0:
        return 1.0
    mant, e = np.frexp(amax / 448.0)
    return float(np.ldexp(1.0, int(e) - 1 if mant == 0.5 else int(e)))


def test_precision_block_fp8_matches_oracle(env, precision_block):
    torch, smp, _ = env
    A, B, ref = precision_block
    w = PREC
    g = _sketch_bf16(env, A, B, smp.SMP_ENGINE_TC_FP8)
    # the quantised model: s e4m3(sqrt(k) Pi) e4m3(X / s) / sqrt(k), one power-of-two s per block and matrix
    Pq = _e4m3(torch, P.pi_block(1, w["k"], 0, BLOCK) * np.sqrt(w["k"]))
    for key, X in (("At", A), ("Bt", B)):
        Xh = _host(X).astype(np.float64)
        s = _pow2_scale(Xh)
        model = np.zeros((w["k"], Xh.shape[1]))
        for r0 in range(0, BLOCK, 8192):
            model += Pq[:, r0:r0 + 8192] @ _e4m3(torch, Xh[r0:r0 + 8192] / s)
        model *= s / np.sqrt(w["k"])
        assert _colrel(g[key], model.T) < 2e-3, key
    assert _colrel(g["At"], ref.At.T) < 8e-2
    assert _colrel(g["Bt"], ref.Bt.T) < 8e-2
    np.testing.assert_allclose(g["sA"], ref.sA, rtol=1e-10)
    np.testing.assert_allclose(g["sB"], ref.sB, rtol=1e-10)


# ------------------------------------------------------------------------------------------- full-size workloads
@pytest.fixture(scope="module")
def scale_data(env):
    torch, _, _ = env
    w = SCALE
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(w["d"], w["n"], w["n"], w["L"], w["sigma"], w["alpha"],
                                                  seed=w["seed"], device="cuda")
    torch.cuda.synchronize()
    yield A, B
    del A, B
    torch.cuda.empty_cache()


@pytest.mark.parametrize("same_ab", [False, True])
def test_scale_workload_end_to_end(env, pool, scale_data, same_ab):
    """d = 1,000,000, n1 = n2 = 2,000, k = 500, r = 10, T = 10, m = 4 n r ln n, TF32 tensor-core sketch (the
    bench's engine and launch configuration), 16 blocks of 65,536 rows."""
    torch, smp, pipeline = env
    w = SCALE
    A, B = scale_data
    Bd = A if same_ab else B
    m = O.default_m(w["n"], w["n"], w["r"])
    s = pipeline.Solver(w["n"], w["n"], w["k"], torch.float32, seed=1, same_ab=same_ab, max_rows=BLOCK)
    out = s.solve(A, None if same_ab else B, w["r"], w["T"], m=m, sample_seed=2, walt_seed=3, block_rows=BLOCK)
    torch.cuda.synchronize()
    om = omega_numpy(s)
    st = s.sketch_state()
    gA = st["At"].cpu().numpy().astype(np.float64)
    gB = st["Bt"].cpu().numpy().astype(np.float64)
    gsA, gsB = st["sA"].cpu().numpy(), st["sB"].cpu().numpy()
    s.close()

    ref_st = OS.sketch_stream(lambda r0, r1: (_host(A[r0:r1]), None if same_ab else _host(B[r0:r1])), w["d"],
                              w["n"], w["n"], w["k"], 1, BLOCK, same_ab=same_ab, pool=pool)
    ref = OS.solve_from_state(ref_st, m, w["r"], w["T"], 2)

    np.testing.assert_allclose(gsA, ref_st.sA, rtol=1e-10)
    np.testing.assert_allclose(gsB, ref_st.sB, rtol=1e-10)
    assert _colrel(gA, ref_st.At.T) < 2e-3
    assert _colrel(gB, ref_st.Bt.T) < 2e-3
    assert om["nnz"] == ref["rows"].shape[0]
    np.testing.assert_array_equal(om["col"], ref["cols"])
    np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])

    M = _product(torch, A, Bd)
    (e_gpu, e_ref), sv = _errors(torch, M, [(out["U"], out["S"], out["V"]), (ref["U"], ref["S"], ref["V"])])
    opt = float(sv[w["r"]] / sv[0])
    assert abs(e_gpu - e_ref) <= 1e-3, (e_gpu, e_ref)
    assert e_gpu >= opt - 1e-9 and e_ref >= opt - 1e-9


def test_precision_prefix_end_to_end(env, pool):
    """The precision workload (n1 = n2 = 4,096, k = 1,024, r = 20, T = 15, BF16 stored, latent rank 32, noise 0.05,
    column exponent 0.7) on a d = 200,000 row prefix: the BF16 and FP8 tensor-core paths against the oracle run on
    the same stored values."""
    torch, smp, pipeline = env
    w = PREC
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(w["d"], w["n"], w["n"], w["L"], w["sigma"], w["alpha"],
                                                  seed=w["seed"], device="cuda", dtype=torch.bfloat16)
    torch.cuda.synchronize()
    m = O.default_m(w["n"], w["n"], w["r"])
    res = {}
    for name, eng in (("bf16", smp.SMP_ENGINE_TC), ("fp8", smp.SMP_ENGINE_TC_FP8)):
        s = pipeline.Solver(w["n"], w["n"], w["k"], torch.bfloat16, seed=1, engine=eng, max_rows=BLOCK)
        out = s.solve(A, B, w["r"], w["T"], m=m, sample_seed=2, walt_seed=3, block_rows=BLOCK)
        torch.cuda.synchronize()
        res[name] = (out, omega_numpy(s))
        s.close()

    ref_st = OS.sketch_stream(lambda r0, r1: (_host(A[r0:r1]), _host(B[r0:r1])), w["d"], w["n"], w["n"], w["k"], 1,
                              BLOCK, pool=pool)
    ref = OS.solve_from_state(ref_st, m, w["r"], w["T"], 2)
    for name, (_, om) in res.items():
        assert om["nnz"] == ref["rows"].shape[0], name
        np.testing.assert_array_equal(om["col"], ref["cols"])
        np.testing.assert_array_equal(csr_rows(om["row_ptr"]), ref["rows"])

    M = _product(torch, A, B)
    fac = [(o["U"], o["S"], o["V"]) for o, _ in (res["bf16"], res["fp8"])] + [(ref["U"], ref["S"], ref["V"])]
    (e_bf16, e_fp8, e_ref), sv = _errors(torch, M, fac)
    opt = float(sv[w["r"]] / sv[0])
    assert abs(e_bf16 - e_ref) <= 3e-3, (e_bf16, e_ref)
    assert abs(e_fp8 - e_ref) <= 1e-2, (e_fp8, e_ref)
    assert min(e_bf16, e_fp8, e_ref) >= opt - 1e-9
