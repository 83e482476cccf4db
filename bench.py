#!/usr/bin/env python
"""Throughput of SMP-PCA (Algorithm 1) on one GB300 per rank, through libsmp's C ABI.

Workload (default "scale"): A, B in R^{1,000,000 x 2,000} FP32 (16 GB, resident in HBM, larger than L2 so no
flush is needed), low rank 20 + noise 0.1, column scales (j+1)^-0.5; k = 500, r = 10, T = 10,
m = 4 n r ln n; rows stream through smp_sketch_accumulate in 65,536-row blocks. One step = one full solve:
sketch (16 blocks) + finalize + sample + estimate + WAltMin + canonical form.

Prints one JSON line (rank 0). value = solves per second over all ranks (each rank solves its own instance:
weak scaling, no data-path collective). `roofline` describes the sketch kernel (the dominant one), `e2e` the same
metric through smp_sketch_accumulate_host with the inputs in pinned host memory, `cpu_baseline` and `oracle` the
CPU oracle's whole solve of the same workload (its time, Omega bit for bit, its spectral error). On one GPU the
line also carries the `precision`, `batched` and `serving` forms, each measured on its own workload outside the
timed region with its own clocks and oracle comparison (--no-forms leaves them out).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--engine auto|simt|tc]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sketch GB/s vs HBM peak; end-to-end solves/s & p99 at fixed spectral error"
WORKLOADS = {
    "scale": dict(d=1_000_000, n1=2000, n2=2000, L=20, sigma=0.1, alpha=0.5, k=500, r=10, T=10, block=65536),
    "tiny": dict(d=2000, n1=200, n2=200, L=10, sigma=0.1, alpha=0.5, k=100, r=5, T=10, block=65536),
    # one 65,536-row block of the scale shape (1 GB of inputs): the case the ncu captures of the sketch kernel use
    "block": dict(d=65536, n1=2000, n2=2000, L=20, sigma=0.1, alpha=0.5, k=500, r=10, T=10, block=65536),
    # one 65,536-row block at the largest width and smallest sketch of the batched form (n = 2,048, r = 5, k = 40):
    # the sketch instantiation for k <= 160 (32-row stages), HBM-bound
    "block_batch": dict(d=65536, n1=2048, n2=2048, L=20, sigma=0.1, alpha=0.5, k=40, r=5, T=10, block=65536),
    # serving form: Poisson arrivals, job sizes of the batched config (n in [64, 2048], d in [1e4, 5e5],
    # r in {5, 10, 20}, k = 8 r), BF16 inputs windowed from a resident pool, 32,768-row blocks, 120 GB budget
    "serve": dict(rate=200.0, jobs=800, warm_jobs=40, block=32768, pool_rows=1_000_000, width=2048, L=20,
                  sigma=0.1, alpha=0.5, budget=120e9, workers=6, T=10),
    # precision form: BF16-stored inputs, sketch in BF16 and in FP8 E4M3 (tensor cores) against the FP32 path
    # (k = 1,024 exceeds the TF32 engine's 512, so FP32 runs on the CUDA-core engine) on the same stored values
    "precision": dict(d=4_000_000, n1=4096, n2=4096, L=32, sigma=0.05, alpha=0.7, k=1024, r=20, T=15, block=65536,
                      steps=4, warm=1),
    # one 65,536-row block of the precision shape (1 GB of BF16 inputs): the case the ncu captures use
    "precision_block": dict(d=65536, n1=4096, n2=4096, L=32, sigma=0.05, alpha=0.7, k=1024, r=20, T=15,
                            block=65536, steps=1, warm=1),
    # Table 1's synthetic row (Section 4): d = n = 100,000, A = B = G D (G Gaussian, D_ii = 1 / i), k = 2,000, the
    # default r = 5, T = 10, m = 4 n r ln n; SMP-PCA against LELA and the optimum, with the paper's printed errors
    "table1": dict(d=100_000, n1=100_000, n2=100_000, k=2000, r=5, T=10, block=16384,
                   paper={"optimal": 0.0271, "lela": 0.0274, "smp_pca": 0.0280}),
    # batched form: 256 FP32 instances (n in [64, 2048], d in [1e4, 5e5], r in {5, 10, 20}, k = 8 r) solved
    # together, sketch engine per (k, n bucket) from the autotuner
    "batch": dict(instances=256, warm=16, block=65536, pool_rows=1_000_000, width=2048, L=20, sigma=0.1, alpha=0.5,
                  budget=200e9, workers=32, T=10),
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (every rank gets it): a step's time is the slowest rank's."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# rows of the scale workload's single pass the CPU oracle is timed on (about 10 s of host work on the GPU machine)
CPU_SAMPLE_ROWS = 65536


def cpu_oracle_sample(w, seed_in, rows=CPU_SAMPLE_ROWS):
    """Time the CPU oracle on a bounded sample of the workload: the single pass over `rows` of the d rows (scaled
    by d / rows: the pass is linear in d) plus sampling, estimation and WAltMin at full n (independent of d)."""
    import numpy as np

    from oracle import smp as O
    from paper_1610_06656_gb300 import synth
    A, B = synth.lowrank_plus_noise(rows, w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"], seed=seed_in,
                                    dtype=np.float32)
    m = O.default_m(w["n1"], w["n2"], w["r"])
    t0 = time.perf_counter()
    st = O.sketch(A, B, w["k"], 1, block_rows=min(rows, w["block"]))
    t1 = time.perf_counter()
    rws, cls, qh = O.sample_omega(st.sA, st.sB, m, 2)
    vals = O.estimate(rws, cls, st.At, st.Bt, st.sA, st.sB)
    Uh, Vh = O.waltmin(w["n1"], w["n2"], rws, cls, vals, qh, w["r"], w["T"], st.sA)
    O.canonical(Uh, Vh)
    t2 = time.perf_counter()
    per_solve = (t1 - t0) * (w["d"] / rows) + (t2 - t1)
    return per_solve, t2 - t0


def run_reference(args, w):
    """The reference arm: the CPU oracle as it stands, on the machine's host cores. Each step is a bounded sample of the
    workload (the single pass over CPU_SAMPLE_ROWS of the d rows plus sampling, estimate and WAltMin at full n);
    `value` extrapolates the sample to a whole solve (the pass is linear in d) and says so."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    rows = CPU_SAMPLE_ROWS if args.workload == "scale" else w["d"]
    for _ in range(args.warmup):
        cpu_oracle_sample(w, 1001, rows)
    per, walls = [], []
    for _ in range(args.steps):
        p, wall = cpu_oracle_sample(w, 1001, rows)
        per.append(p)
        walls.append(wall)
    value = len(per) / sum(per)
    extrapolated = rows < w["d"]
    sample = ("single pass over %d of %d rows + sampling, estimate, WAltMin at n = %d; solve time = pass time x "
              "d / rows + the rest" % (rows, w["d"], w["n1"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "extrapolated": extrapolated,
            "extrapolation": ("value = 1 / (sample pass time x %d / %d + sampling, estimate and WAltMin time); "
                              "ms_per_step is the measured wall time of one sample step" % (w["d"], rows))
            if extrapolated else None,
            "extrapolated_ms_per_solve": 1e3 * sum(per) / len(per),
            "config": {"workload": args.workload, **{k: w[k] for k in ("d", "n1", "n2", "k", "r", "T")},
                       "block_rows": w["block"], "oracle": "CPU binary64 (numpy/LAPACK)"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def OS_workers():
    from tests import oracle_stream as OS
    return OS.host_workers()


def oracle_full_solve(w, fetch, m, same_ab=False):
    """The CPU oracle's whole solve of a workload whose row blocks fetch(r0, r1) returns as host arrays: the single
    pass with Pi's Philox blocks drawn by spawned worker processes (tests/oracle_stream.py schedules the oracle's own
    functions), then sampling, estimate, WAltMin and the canonical form. Returns (result dict, wall seconds)."""
    from tests import oracle_stream as OS
    pool = OS.PiPool()
    try:
        t0 = time.perf_counter()
        st = OS.sketch_stream(fetch, w["d"], w["n1"], w["n2"], w["k"], 1, w["block"], same_ab=same_ab, pool=pool)
        ref = OS.solve_from_state(st, m, w["r"], w["T"], 2)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
    ref["sA"], ref["sB"] = st.sA, st.sB
    return ref, wall


def spectral_error(torch, A, B, factors, block=65536):
    """||A^T B - U S V^T||_2 / ||A^T B||_2 for each (U, S, V) in factors, with A^T B accumulated blockwise (FP32
    products, no TF32, summed in binary64), and the Eckart-Young optimum. Evaluation only: torch / cuSOLVER compute
    the norms, not the path."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    M = torch.zeros(A.shape[1], B.shape[1], dtype=torch.float64, device=A.device)
    for r0 in range(0, A.shape[0], block):
        M += (A[r0:r0 + block].float().T @ B[r0:r0 + block].float()).double()
    torch.backends.cuda.matmul.allow_tf32 = prev
    sv = torch.linalg.svdvals(M)
    r = factors[0][0].shape[1]
    opt = float(sv[r] / sv[0]) if sv.shape[0] > r else 0.0
    errs = [float(torch.linalg.matrix_norm(M - (U * S) @ V.T, ord=2) / sv[0]) for U, S, V in factors]
    return errs, opt


def main():
    # the batched and serving forms run many jobs on streams of their own: let more of them reach the device at once
    # (process-local; it must be set before the CUDA context exists)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=sorted(WORKLOADS))
    ap.add_argument("--engine", default="auto", choices=["auto", "simt", "tc", "tc_bf16", "srht"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true")
    ap.add_argument("--workers", type=int, default=0, help="solve worker threads of the batched / serving forms")
    ap.add_argument("--batch-dtype", default="f32", choices=["f32", "bf16"], help="stored inputs of the batched form")
    ap.add_argument("--serve-dtype", default="bf16", choices=["f32", "bf16"], help="stored inputs of the serving form")
    ap.add_argument("--rate", type=float, default=0.0, help="serving form: offered jobs/s instead of 200")
    ap.add_argument("--size", type=int, default=0, help="table1 workload: d = n = SIZE instead of 100,000")
    ap.add_argument("--no-baseline", action="store_true",
                    help="skip the SVD(A~^T B~) and multinomial-sampling comparisons")
    ap.add_argument("--no-forms", action="store_true",
                    help="scale workload: leave the precision / batched / serving sub-objects out of the line")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.workload == "serve":
        return run_serving(args, w)
    if args.workload == "batch":
        return run_batched(args, w)
    if args.workload in ("precision", "precision_block"):
        return run_precision(args, w)
    if args.workload == "table1":
        return run_table1(args, w)

    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1610_06656_gb300 import build, pipeline, smp, synth
    smp.load(build.build() if rank == 0 or world == 1 else build.LIB_PATH)
    if world > 1:
        dist.barrier()
    engine = {"auto": smp.SMP_ENGINE_AUTO, "simt": smp.SMP_ENGINE_SIMT, "tc": smp.SMP_ENGINE_TC,
              "tc_bf16": smp.SMP_ENGINE_TC_BF16, "srht": smp.SMP_ENGINE_SRHT}[args.engine]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(w["d"], w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"],
                                                  seed=1001 + rank, device=dev)
    torch.cuda.synchronize()
    # two contexts on streams of their own: consecutive solves alternate between them, so that the sketch of solve
    # i + 1 (tensor-bound) runs while solve i's WAltMin (small dependent launches and host checks) finishes
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    solvers = [pipeline.Solver(w["n1"], w["n2"], w["k"], torch.float32, seed=1 + rank, engine=engine,
                               max_rows=w["block"], stream=st.cuda_stream) for st in streams]
    solver = solvers[0]
    m = pipeline.default_m(w["n1"], w["n2"], w["r"])

    def sketch_timed(i, evs, svs, sts):
        sv, st = svs[i % 2], sts[i % 2]
        smp.smp_sketch_reset(sv.ctx)
        for r0 in range(0, w["d"], w["block"]):
            r1 = min(w["d"], r0 + w["block"])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            smp.smp_sketch_accumulate(sv.ctx, A[r0:r1], w["n1"], B[r0:r1], w["n2"], r0, r1 - r0)
            e1.record(st)
            evs.append((e0, e1, r1 - r0))
        smp.smp_sketch_finalize(sv.ctx)

    def run_steps(count, evs, step_events, svs=solvers, sts=streams):
        """count solves, pipelined: solve i's sketch was issued before solve i - 1's WAltMin."""
        out = None
        marks = {}

        def issue(i):
            s0 = torch.cuda.Event(enable_timing=True)
            s0.record(sts[i % 2])
            marks[i] = s0
            sketch_timed(i, evs, svs, sts)

        issue(0)
        for i in range(count):
            sv, st = svs[i % 2], sts[i % 2]
            nnz = sv.sample(m, 2 + rank)
            with torch.cuda.stream(st):
                vals = sv.estimate(nnz)
            if i + 1 < count:
                issue(i + 1)
            with torch.cuda.stream(st):
                out = sv.waltmin(vals, w["r"], w["T"], 0, 3 + rank), nnz
            s1 = torch.cuda.Event(enable_timing=True)
            s1.record(st)
            step_events.append((marks.pop(i), s1))
        return out

    run_steps(args.warmup, [], [])
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = smp.smp_launch_count()
    sk_events, step_events = [], []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for st in streams:
        st.wait_event(t_start)
    (U, S, V), nnz = run_steps(args.steps, sk_events, step_events)
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        stream.wait_event(ev)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = smp.smp_launch_count() - launches0
    clk = clocks.stop()
    om_last = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the last timed solve's Omega, for the oracle leg
        om_last = {key: (v.cpu().numpy() if hasattr(v, "cpu") else v)
                   for key, v in solvers[(args.steps - 1) % 2].omega().items()}
    elapsed = t_start.elapsed_time(t_end) / 1e3
    if world > 1:
        elapsed = max_over_ranks(elapsed, dist, dev)
    step_ms = sorted(a.elapsed_time(b) for a, b in step_events)
    sk_ms = [a.elapsed_time(b) for a, b, _ in sk_events]
    sk_rows = [n for _, _, n in sk_events]
    value = world * args.steps / elapsed

    peaks, peak_kind = measured_peaks()
    ntot = w["n1"] + w["n2"]
    sk_bytes = sum(sk_rows) * ntot * 4 / len(sk_rows)          # algorithmic bytes per launch: A and B rows read once
    sk_flops = 2.0 * w["k"] * sum(sk_rows) * ntot / len(sk_rows)
    sk_avg_s = sum(sk_ms) / len(sk_ms) / 1e3
    b16ops = engine == smp.SMP_ENGINE_TC_BF16
    tc_used = engine in (smp.SMP_ENGINE_TC, smp.SMP_ENGINE_TC_BF16) or (engine == smp.SMP_ENGINE_AUTO and tc_active(w))
    srht = engine == smp.SMP_ENGINE_SRHT
    kind = "srht" if srht else "tc_bf16" if b16ops else "tc" if tc_used else "simt"
    roof = sketch_roofline(kind, sk_bytes, sk_flops, sk_avg_s, peaks, peak_kind)
    roof["traffic"] = sketch_traffic(sum(sk_rows) / len(sk_rows), w) if tc_used and not b16ops else None
    roof["kernel"] = ("smp_sketch_accumulate: block SRHT (srht_fused_kernel)" if srht else
                      "smp_sketch_accumulate: sketch_tc_kernel<BF16 operands> (tcgen05 kind::f16), Pi of the next "
                      "block generated on a side stream meanwhile" if b16ops else
                      "smp_sketch_accumulate: sketch_tc_kernel (tcgen05), Pi of the next block generated on a side "
                      "stream meanwhile" if tc_used else "sketch_simt_kernel")
    roof["hbm_gbs"] = sk_bytes / sk_avg_s / 1e9
    roof["hbm_frac"] = roof["hbm_gbs"] / peaks["hbm_gbs"]
    roof["launch_ms"] = sk_avg_s * 1e3
    roof["bytes_per_launch"] = sk_bytes

    # the same pipelined solves with BF16 tensor-core operands for the binary32 inputs (SMP_ENGINE_TC_BF16), outside
    # the timed region above: solves/s, sketch rate against the BF16 peak, and (below) the spectral error
    alt = None
    if rank == 0 and not args.no_baseline and tc_used and not b16ops and not srht:
        a_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
        a_solvers = [pipeline.Solver(w["n1"], w["n2"], w["k"], torch.float32, seed=1 + rank,
                                     engine=smp.SMP_ENGINE_TC_BF16, max_rows=w["block"], stream=st.cuda_stream)
                     for st in a_streams]
        run_steps(args.warmup, [], [], a_solvers, a_streams)
        torch.cuda.synchronize()
        a_sk, a_steps = [], []
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for st in a_streams:
            st.wait_event(a0)
        (Ua, Sa, Va), _ = run_steps(args.steps, a_sk, a_steps, a_solvers, a_streams)
        for st in a_streams:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        a1.record(stream)
        torch.cuda.synchronize()
        a_launch = sum(x.elapsed_time(y) for x, y, _ in a_sk) / len(a_sk) / 1e3
        alt = {"name": "SMP_ENGINE_TC_BF16: the same inputs with BF16 tensor-core operands "
                       "(sketch_tc_kernel<BF16 operands>, kind::f16)",
               "solves_per_s": args.steps / (a0.elapsed_time(a1) / 1e3),
               "p50_ms": statistics.median(sorted(x.elapsed_time(y) for x, y in a_steps)),
               "sketch_launch_ms": a_launch * 1e3, "sketch_tflops": sk_flops / a_launch / 1e12,
               "sketch_frac_of_bf16_peak": sk_flops / a_launch / 1e12 / peaks["bf16_tflops"],
               "sketch_hbm_frac": sk_bytes / a_launch / 1e9 / peaks["hbm_gbs"], "spectral_err": None}
        for sv in a_solvers:
            sv.close()

    # the paper's comparison, SVD(A~^T B~) by power iteration on the last step's sketches (outside the timed
    # region; smp_sketch_svd synchronises, so host wall time is its duration)
    base = None
    if rank == 0 and not args.no_baseline:
        solver.sketch_svd(w["r"], seed=4)
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            Ub, Sb, Vb = solver.sketch_svd(w["r"], seed=4)
        base = {"name": "SVD(A~^T B~) by block power iteration (smp_sketch_svd)",
                "ms": 1e3 * (time.perf_counter() - t0) / reps, "spectral_err": None}

    # the Appendix's row-wise multinomial sampler against the Bernoulli coins on the same sketches: sampling time
    # (both synchronise: host wall time), |Omega|, and the error of a full WAltMin on the multinomial Omega
    mn = None
    if rank == 0 and not args.no_baseline:
        def timed(fn, reps=3):
            fn()
            t0 = time.perf_counter()
            for _ in range(reps):
                out = fn()
            return out, 1e3 * (time.perf_counter() - t0) / reps
        nnz_b, ms_b = timed(lambda: solver.sample(m, 2 + rank))
        nnz_m, ms_m = timed(lambda: solver.sample(m, 2 + rank, "multinomial"))
        Um, Sm, Vm = solver.waltmin(solver.estimate(nnz_m), w["r"], w["T"], 0, 3 + rank)
        mn = {"name": "row-wise multinomial sampling (smp_sample_multinomial)", "sample_ms": ms_m,
              "bernoulli_sample_ms": ms_b, "nnz": int(nnz_m), "bernoulli_nnz": int(nnz_b), "spectral_err": None}

    # LELA, the two-pass method of Table 1, on the same data: pass 1 norms only, the same Omega sampling, pass 2 the
    # exact entries on tensor cores, the same WAltMin (outside the timed region; per-block CUDA events on the passes,
    # host wall time around whole solves, which synchronise)
    lela = None
    if rank == 0 and not args.no_baseline:
        ls = pipeline.Solver(w["n1"], w["n2"], 16, torch.float32, seed=1 + rank, max_rows=w["block"])

        def lela_solve(evn=None, evx=None):
            smp.smp_sketch_reset(ls.ctx)
            for r0 in range(0, w["d"], w["block"]):
                r1 = min(w["d"], r0 + w["block"])
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(stream)
                smp.smp_norms_accumulate(ls.ctx, A[r0:r1], w["n1"], B[r0:r1], w["n2"], r0, r1 - r0)
                ev[1].record(stream)
                if evn is not None:
                    evn.append(ev)
            smp.smp_sketch_finalize(ls.ctx)
            nnz_l = ls.sample(m, 2 + rank)
            for r0 in range(0, w["d"], w["block"]):
                r1 = min(w["d"], r0 + w["block"])
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(stream)
                smp.smp_exact_accumulate(ls.ctx, A[r0:r1], w["n1"], B[r0:r1], w["n2"], r0, r1 - r0)
                ev[1].record(stream)
                if evx is not None:
                    evx.append((ev[0], ev[1], r1 - r0))
            vals_l = torch.empty(max(nnz_l, 1), dtype=torch.float32, device=dev)
            smp.smp_exact_values(ls.ctx, vals_l)
            return ls.waltmin(vals_l[:nnz_l], w["r"], w["T"], 0, 3 + rank), nnz_l

        lela_solve()
        torch.cuda.synchronize()
        evn, evx, reps = [], [], 2
        t0 = time.perf_counter()
        for _ in range(reps):
            (Ul, Sl, Vl), nnz_l = lela_solve(evn, evx)
        torch.cuda.synchronize()
        l_ms = 1e3 * (time.perf_counter() - t0) / reps
        n_ms = sum(a.elapsed_time(b) for a, b in evn) / reps
        x_ms = [a.elapsed_time(b) for a, b, _ in evx]
        x_rows = sum(n for _, _, n in evx) / len(evx)
        x_flops = 2.0 * w["n1"] * w["n2"] * x_rows             # the dense tile product per launch
        tf32_peak = peaks["bf16_tflops"] * (1.1 / 2.25)
        x_avg = sum(x_ms) / len(x_ms) / 1e3
        lela = {"name": "LELA two-pass (smp_norms_accumulate; smp_exact_accumulate: transpose_tf32_kernel + "
                        "exact_tc_kernel)", "solves_per_s": 1e3 / l_ms, "ms": l_ms, "nnz": int(nnz_l),
                "norms_pass_ms": n_ms, "norms_pass_gbs": w["d"] * ntot * 4 / (n_ms / 1e3) / 1e9,
                "exact_pass_ms": sum(x_ms) / reps, "exact_launch_ms": x_avg * 1e3,
                "exact_tflops": x_flops / x_avg / 1e12, "exact_tf32_frac": x_flops / x_avg / 1e12 / tf32_peak,
                "exact_useful_tflops": 2.0 * nnz_l * x_rows / x_avg / 1e12, "spectral_err": None}
        ls.close()

    # the CPU oracle's whole solve of the same workload (same bytes, same seeds): the CPU baseline (timed, every row,
    # no extrapolation) and the parity of the timed solve (Omega bit for bit, spectral error)
    ref, cpu, orc = None, None, None
    if om_last is not None:
        ref, o_wall = oracle_full_solve(w, lambda r0, r1: (A[r0:r1].cpu().numpy(), B[r0:r1].cpu().numpy()), m)
        rows_gpu = np.repeat(np.arange(w["n1"]), np.diff(om_last["row_ptr"]))
        omega_equal = bool(om_last["nnz"] == ref["rows"].shape[0] and np.array_equal(om_last["col"], ref["cols"])
                           and np.array_equal(rows_gpu, ref["rows"]))
        workers = OS_workers()
        cpu = {"value": 1.0 / o_wall, "unit": "solves/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": "one whole solve of the workload (all %d rows, no extrapolation): the oracle's single pass "
                         "with its Pi blocks drawn by %d spawned processes and its products on the main process's "
                         "BLAS, then sampling, estimate, WAltMin and the canonical form; %.1f s"
                         % (w["d"], workers, o_wall)}
        orc = {"omega_equal": omega_equal, "nnz": int(ref["rows"].shape[0]), "spectral_err": None,
               "err_diff": None, "tolerance": 1e-3, "wall_s": o_wall}

    err, opt_err = None, None
    if not args.no_error and rank == 0:
        extra = ([(Ub, Sb, Vb)] if base else []) + ([(Um, Sm, Vm)] if mn else []) + ([(Ul, Sl, Vl)] if lela else []) \
            + ([(Ua, Sa, Va)] if alt else [])
        if ref is not None:
            extra.append(tuple(torch.from_numpy(np.ascontiguousarray(ref[x])).to(dev) for x in ("U", "S", "V")))
        errs, opt_err = spectral_error(torch, A, B, [(U, S, V)] + extra)
        err = errs[0]
        rest = errs[1:]
        for entry in (base, mn, lela, alt):
            if entry:
                entry["spectral_err"] = rest.pop(0)
        if orc is not None:
            orc["spectral_err"] = rest.pop(0)
            orc["err_diff"] = abs(err - orc["spectral_err"])

    # ---- end to end: host-resident inputs copied in every step (pinned, double-buffered row blocks)
    e2e = None
    if args.e2e_steps > 0:
        with torch.cuda.stream(streams[0]):
            e2e = run_e2e(torch, smp, solver, A, B, w, m, rank, args.e2e_steps, streams[0], world, dev)


    in_gb = w["d"] * (w["n1"] + w["n2"]) * 4 / 1e9
    l2_note = ("inputs (%.1f GB) larger than L2; no flush" % in_gb) if in_gb > 0.129 else "inputs fit in L2"
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16 operands (f32 inputs)" if b16ops else ("tf32" if tc_used else "f32"),
                "data": "synthetic (low rank 20 + noise 0.1, column scales (j+1)^-0.5, torch RNG seeded per rank)",
                "config": {"workload": args.workload, **{k: w[k] for k in ("d", "n1", "n2", "k", "r", "T")},
                           "block_rows": w["block"], "m": m, "nnz": int(nnz), "parallelism": "replicas",
                           "pipelining": "2 contexts on 2 streams: solve i + 1's sketch overlaps solve i's WAltMin",
                           "l2": l2_note, "engine": args.engine},
                "p50_ms": statistics.median(step_ms), "p99_ms": step_ms[min(len(step_ms) - 1,
                                                                            int(math.ceil(0.99 * len(step_ms))) - 1)],
                "sketch_gbs": roof["hbm_gbs"], "spectral_err": err, "optimal_err": opt_err,
                "oracle_err": orc["spectral_err"] if orc else None,
                "omega_equal": orc["omega_equal"] if orc else None, "oracle": orc,
                "baseline_sketch_svd": base, "sampler_multinomial": mn, "lela": lela, "engine_bf16_operands": alt,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk}
    for sv in solvers:
        sv.close()
    if rank == 0 and world == 1 and args.workload == "scale" and not args.no_forms:
        # the three forms of the method on their own workloads, each outside the timed region above and with its
        # own clocks, launch count and oracle comparison: precision (BF16 / FP8 / FP32 sketches), batched (256
        # uneven instances), serving (Poisson arrivals)
        del A, B
        torch.cuda.empty_cache()
        line["precision"] = run_precision(args, WORKLOADS["precision"], embed=True)
        line["batched"] = run_batched(args, WORKLOADS["batch"], embed=True)
        line["serving"] = run_serving(args, WORKLOADS["serve"], embed=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def implicit_errors(torch, A, factors, r, iters=40, block=16, seed=0):
    """For the implicit symmetric product M = A^T A (never formed): ||M - U S V^T||_2 / ||M||_2 for each (U, S, V)
    and the Eckart-Young optimum sigma_{r+1} / sigma_1, by block subspace iteration with a Rayleigh-Ritz step (torch
    FP32 products without TF32, binary64 Ritz problems). Evaluation only."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    g = torch.Generator(device=A.device)
    g.manual_seed(seed)
    n = A.shape[1]

    def mul(X):
        return A.T @ (A @ X)

    def top_eigs(op, b):
        X = torch.linalg.qr(torch.randn(n, b, generator=g, device=A.device))[0]
        for _ in range(iters):
            X = torch.linalg.qr(op(X))[0]
        H = (X.T @ op(X)).double()
        return torch.linalg.eigvalsh(0.5 * (H + H.T)).flip(0)

    ev = top_eigs(mul, block)
    s1 = float(ev[0])
    opt = float(ev[r] / ev[0])
    errs = []
    for U, S, V in factors:
        Uf, Vf, Sf = U.float(), V.float(), S.float()

        def rtr(X, Uf=Uf, Vf=Vf, Sf=Sf):   # R^T R X with R = M - U S V^T (M symmetric)
            Y = mul(X) - Uf @ (Sf[:, None] * (Vf.T @ X))
            return mul(Y) - Vf @ (Sf[:, None] * (Uf.T @ Y))

        errs.append(float(torch.sqrt(torch.clamp(top_eigs(rtr, 8)[0], min=0.0))) / s1)
    torch.backends.cuda.matmul.allow_tf32 = prev
    return errs, opt


def run_table1(args, w):
    """Table 1's synthetic row (Section 4): SMP-PCA (one pass: Gaussian sketch with k = 2,000, above the tensor-core
    engines' limits, so on the CUDA cores) and LELA (two passes: norms, then the exact entries on tensor cores) on
    the same A = B = G D, their relative spectral errors and the optimum next to the paper's printed values, and
    each solve's wall time (both end in a synchronising WAltMin)."""
    import torch
    from paper_1610_06656_gb300 import build, pipeline, smp, synth
    smp.load(build.build())
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.size:
        w = dict(w, d=args.size, n1=args.size, n2=args.size)
    n = w["n1"]
    A = synth.gd_torch(w["d"], n, seed=2016, device=dev)
    torch.cuda.synchronize()
    m = pipeline.default_m(n, n, w["r"])
    out = {}
    for name, k in (("smp_pca", w["k"]), ("lela", 16)):
        s = pipeline.Solver(n, n, k, torch.float32, seed=1, same_ab=True, max_rows=w["block"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "smp_pca":
            res = s.solve(A, None, w["r"], w["T"], m=m, sample_seed=2, walt_seed=3, block_rows=w["block"])
        else:
            res = s.lela(A, None, w["r"], w["T"], m=m, sample_seed=2, walt_seed=3, block_rows=w["block"])
        torch.cuda.synchronize()
        out[name] = dict(ms=1e3 * (time.perf_counter() - t0), nnz=int(res["nnz"]),
                         factors=(res["U"], res["S"], res["V"]))
        s.close()
    errs, opt = implicit_errors(torch, A, [out["smp_pca"]["factors"], out["lela"]["factors"]], w["r"])
    line = {"metric": "relative spectral error, Table 1 synthetic row", "value": errs[0],
            "unit": "||A^T B - U S V^T||_2 / ||A^T B||_2", "higher_is_better": False, "n_gpus": 1,
            "vs_baseline": None, "dtype": "f32 (SMP-PCA sketch on CUDA cores), tf32 (LELA exact entries)",
            "data": "synthetic A = B = G D, G standard Gaussian (torch RNG, seed 2016), D_ii = 1 / i",
            "config": {"workload": "table1", "d": w["d"], "n": n, "k": w["k"], "r": w["r"], "T": w["T"],
                       "m": m, "block_rows": w["block"]},
            "smp_pca": {"spectral_err": errs[0], "solve_ms": out["smp_pca"]["ms"], "nnz": out["smp_pca"]["nnz"]},
            "lela": {"spectral_err": errs[1], "solve_ms": out["lela"]["ms"], "nnz": out["lela"]["nnz"]},
            "optimal_err": opt, "paper_table1": w["paper"]}
    print(json.dumps(line), flush=True)


def oracle_job_check(torch, spec, pool_A, pool_B, factors, block_rows, tol):
    """One job / instance of the serving or batched form against the CPU oracle run on its window of the pool (the
    stored values, the job's seeds): spectral errors of both against the same A^T B and the size of Omega."""
    import numpy as np
    from oracle import smp as O
    a = pool_A[spec.row_offset:spec.row_offset + spec.d, :spec.n]
    b = pool_B[spec.row_offset:spec.row_offset + spec.d, :spec.n]
    a64 = a.float().cpu().numpy().astype(np.float64)
    b64 = b.float().cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    ref = O.smp_pca(a64, b64, spec.r, spec.k, spec.m, spec.T, seed=2 * spec.seed + 1, sample_seed=2 * spec.seed + 2,
                    block_rows=block_rows)
    wall = time.perf_counter() - t0
    dev = pool_A.device
    fac = [factors, tuple(torch.from_numpy(np.ascontiguousarray(ref[x])).to(dev) for x in ("U", "S", "V"))]
    (e_gpu, e_ref), opt = spectral_error(torch, a, b, fac)
    return {"job": {"n": spec.n, "d": spec.d, "r": spec.r, "k": spec.k}, "spectral_err": e_gpu, "oracle_err": e_ref,
            "err_diff": abs(e_gpu - e_ref), "tolerance": tol, "optimal_err": opt, "oracle_nnz": int(ref["rows"].shape[0]),
            "oracle_wall_s": wall}


def run_serving(args, w, embed=False):
    """The serving form (one GPU): Poisson job arrivals at w["rate"] per second through libsmp's server; reports
    completed solves per second over the run and the latency from each job's last block to its factors. One job is
    also solved by the CPU oracle on its window of the pool and compared."""
    # many jobs run on streams of their own: let more of them reach the device concurrently (process-local)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_1610_06656_gb300 import build, serve, smp, synth
    smp.load(build.build())
    torch.cuda.set_device(0)
    f32 = args.serve_dtype == "f32"
    tdt, sdt, esz = (torch.float32, smp.SMP_F32, 4) if f32 else (torch.bfloat16, smp.SMP_BF16, 2)
    if args.rate:
        w = dict(w, rate=args.rate)
    pool_A, pool_B, _, _, _ = synth.lowrank_plus_noise_torch(w["pool_rows"], w["width"], w["width"], w["L"],
                                                             w["sigma"], w["alpha"], seed=1005, device="cuda",
                                                             dtype=tdt)
    torch.cuda.synchronize()
    pool_bytes = 2 * pool_A.numel() * esz
    workers = args.workers or w["workers"]
    server = smp.smp_serve_create(int(w["budget"] - pool_bytes), solve_workers=workers)
    try:
        warm = serve.poisson_jobs(w["warm_jobs"], w["rate"], seed=99, pool_rows=w["pool_rows"], T=w["T"])
        serve.run(server, warm, pool_A, pool_B, sdt, block_rows=w["block"])
        jobs = serve.poisson_jobs(w["jobs"], w["rate"], seed=5, pool_rows=w["pool_rows"], T=w["T"])
        probe = min(jobs[:50], key=lambda j: j.d * j.n)          # a small early job, for the oracle comparison
        keep = {probe.idx: (torch.empty(probe.n, probe.r, dtype=torch.float64, device="cuda"),
                            torch.empty(probe.r, dtype=torch.float64, device="cuda"),
                            torch.empty(probe.n, probe.r, dtype=torch.float64, device="cuda"))}
        clocks = ClockSampler(0)
        clocks.start()
        launches0 = smp.smp_launch_count()
        records, wall = serve.run(server, jobs, pool_A, pool_B, sdt, block_rows=w["block"], keep=keep)
        launches = smp.smp_launch_count() - launches0
        clk = clocks.stop()
    finally:
        smp.smp_serve_destroy(server)
    lat = sorted(r["latency_ms"] for r in records)
    streamed = sum(j.d * 2 * j.n * esz for j in jobs)
    line = {"metric": "serving: completed solves/s under Poisson arrivals; p50/p99 latency from a job's last "
                      "block to its factors", "value": len(records) / wall, "unit": "solves/s", "n_gpus": 1,
            "steps": len(records), "warmup": w["warm_jobs"], "ms_per_step": 1e3 * wall / max(1, len(records)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.serve_dtype,
            "data": "synthetic (low rank 20 + noise 0.1, column scales (j+1)^-0.5), job inputs are windows of a "
                    "resident %d x %d %s pool pair" % (w["pool_rows"], w["width"], "FP32" if f32 else "BF16"),
            "config": {"workload": "serve", "arrival_rate_per_s": w["rate"], "jobs": w["jobs"],
                       "n": "uniform [64, 2048]", "d": "uniform [10000, 500000]", "r": [5, 10, 20], "k": "8 r",
                       "T": w["T"], "block_rows": w["block"], "budget_bytes": w["budget"],
                       "pool_bytes_charged": pool_bytes, "solve_workers": workers},
            "p50_ms": statistics.median(lat), "p99_ms": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
            "mean_latency_ms": sum(lat) / len(lat), "wall_s": wall, "input_gb_streamed": streamed / 1e9,
            "input_gbs": streamed / wall / 1e9, "gpu_launches": int(launches), "clocks": clk,
            "roofline": None, "cpu_baseline": None, "e2e": None}
    if not args.no_cpu_baseline:
        line["oracle"] = oracle_job_check(torch, probe, pool_A, pool_B, keep[probe.idx], w["block"],
                                          1e-3 if f32 else 3e-3)
    del pool_A, pool_B
    torch.cuda.empty_cache()
    if embed:
        return line
    print(json.dumps(line), flush=True)


def run_precision(args, w, embed=False):
    """The precision form (one GPU): solves/s and spectral error of SMP-PCA with the sketch in BF16, in FP8 E4M3
    (tensor cores) and in FP32 (CUDA cores) on the same BF16-stored inputs; WAltMin's solves in binary64. Then the
    BF16 and FP8 paths and the CPU oracle on the d = 200,000 row prefix of the same inputs: Omega and the spectral
    errors compared."""
    import numpy as np
    import torch
    from paper_1610_06656_gb300 import build, pipeline, smp, synth
    smp.load(build.build())
    torch.cuda.set_device(0)
    A, B, _, _, _ = synth.lowrank_plus_noise_torch(w["d"], w["n1"], w["n2"], w["L"], w["sigma"], w["alpha"],
                                                  seed=1002, device="cuda", dtype=torch.bfloat16)
    torch.cuda.synchronize()
    m = pipeline.default_m(w["n1"], w["n2"], w["r"])
    stream = torch.cuda.current_stream()
    results = {}
    peaks, peak_kind = measured_peaks()
    # (name, stored dtype, engine, timed solves): the FP32 CUDA-core path takes ~2.3 s a solve, so it is timed on 2
    forms = (("bf16", torch.bfloat16, smp.SMP_ENGINE_TC, w["steps"]),
             ("fp8_e4m3", torch.bfloat16, smp.SMP_ENGINE_TC_FP8, w["steps"]),
             ("fp32", torch.float32, smp.SMP_ENGINE_SIMT, min(2, w["steps"])))
    factors = []
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = smp.smp_launch_count()
    for name, tdt, eng, steps in forms:
        Xa, Xb = (A, B) if tdt == torch.bfloat16 else (A.float(), B.float())
        # two contexts on two streams, consecutive solves alternating: solve i + 1's sketch runs while solve i's
        # WAltMin finishes (as in the scale bench)
        sts = [torch.cuda.Stream() for _ in range(2)]
        svs = [pipeline.Solver(w["n1"], w["n2"], w["k"], tdt, seed=1, engine=eng, max_rows=w["block"],
                               stream=st.cuda_stream) for st in sts]
        sk_ev = []

        def run(count):
            out = None

            def issue(i):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(sts[i % 2])
                svs[i % 2].sketch(Xa, Xb, w["block"])
                e1.record(sts[i % 2])
                sk_ev.append((e0, e1))

            issue(0)
            for i in range(count):
                sv, st = svs[i % 2], sts[i % 2]
                nnz = sv.sample(m, 2)
                with torch.cuda.stream(st):
                    vals = sv.estimate(nnz)
                if i + 1 < count:
                    issue(i + 1)
                with torch.cuda.stream(st):
                    out = sv.waltmin(vals, w["r"], w["T"], 0, 3), nnz
            return out

        run(w["warm"])
        torch.cuda.synchronize()
        sk_ev.clear()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for st in sts:
            st.wait_event(t0)
        (U, S, V), nnz = run(steps)
        for st in sts:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        t1.record(stream)
        torch.cuda.synchronize()
        sk_ms = [a.elapsed_time(b) for a, b in sk_ev]
        ms = t0.elapsed_time(t1) / steps
        in_bytes = w["d"] * (w["n1"] + w["n2"]) * 2
        flops = 2.0 * w["k"] * w["d"] * (w["n1"] + w["n2"])
        sk_s = sum(sk_ms) / len(sk_ms) / 1e3
        results[name] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "timed_solves": steps,
                         "sketch_ms": sk_s * 1e3, "sketch_tflops": flops / sk_s / 1e12,
                         "sketch_gbs": in_bytes / sk_s / 1e9, "nnz": int(nnz)}
        factors.append((U.clone(), S.clone(), V.clone()))
        for sv in svs:
            sv.close()
        del Xa, Xb
        torch.cuda.empty_cache()
    launches = smp.smp_launch_count() - launches0
    clk = clocks.stop()
    bf = results["bf16"]
    roof = {"bound": "tensor", "achieved": bf["sketch_tflops"], "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
            "frac": bf["sketch_tflops"] / peaks["bf16_tflops"], "traffic": None,
            "peak_kind": "%s bf16 burst" % peak_kind,
            "kernel": "BF16 sketch of a whole solve (sketch_bf16_kernel + pi_gen_kernel, 62 blocks), CUDA events "
                      "around the 62 smp_sketch_accumulate calls",
            "hbm_frac": bf["sketch_gbs"] / peaks["hbm_gbs"]}
    opt = None
    if not args.no_error:
        errs, opt = spectral_error(torch, A, B, factors)
        for (name, _, _, _), e in zip(forms, errs):
            results[name]["spectral_err"] = e
    prefix = None
    if not args.no_cpu_baseline:
        d0 = min(200_000, w["d"])
        Ap, Bp = A[:d0], B[:d0]
        res, fac = {}, []
        for name, eng in (("bf16", smp.SMP_ENGINE_TC), ("fp8_e4m3", smp.SMP_ENGINE_TC_FP8)):
            sv = pipeline.Solver(w["n1"], w["n2"], w["k"], torch.bfloat16, seed=1, engine=eng, max_rows=w["block"])
            out = sv.solve(Ap, Bp, w["r"], w["T"], m=m, sample_seed=2, walt_seed=3, block_rows=w["block"])
            torch.cuda.synchronize()
            om = {key: (v.cpu().numpy() if hasattr(v, "cpu") else v) for key, v in sv.omega().items()}
            sv.close()
            res[name] = om
            fac.append((out["U"], out["S"], out["V"]))
        ref, o_wall = oracle_full_solve(dict(w, d=d0), lambda r0, r1: (Ap[r0:r1].float().cpu().numpy(),
                                                                       Bp[r0:r1].float().cpu().numpy()), m)
        fac.append(tuple(torch.from_numpy(np.ascontiguousarray(ref[x])).to(A.device) for x in ("U", "S", "V")))
        errs, popt = spectral_error(torch, Ap, Bp, fac)
        prefix = {"d": d0, "oracle_err": errs[2], "optimal_err": popt, "oracle_wall_s": o_wall,
                  "oracle_nnz": int(ref["rows"].shape[0])}
        for (name, om), e, tol in zip(res.items(), errs[:2], (3e-3, 1e-2)):
            rows_gpu = np.repeat(np.arange(w["n1"]), np.diff(om["row_ptr"]))
            prefix[name] = {"spectral_err": e, "err_diff": abs(e - errs[2]), "tolerance": tol,
                            "omega_equal": bool(om["nnz"] == ref["rows"].shape[0] and
                                                np.array_equal(om["col"], ref["cols"]) and
                                                np.array_equal(rows_gpu, ref["rows"]))}
    line = {"metric": "precision form: solves/s and spectral error per sketch precision (same BF16-stored inputs)",
            "value": results["bf16"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": w["steps"],
            "warmup": w["warm"], "ms_per_step": results["bf16"]["ms_per_solve"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (low rank 32 + noise 0.05, column scales (j+1)^-0.7), stored in BF16",
            "config": {"workload": "precision", **{k: w[k] for k in ("d", "n1", "n2", "k", "r", "T")},
                       "block_rows": w["block"], "m": m,
                       "l2": "inputs (%.1f GB) larger than L2; no flush" % (w["d"] * (w["n1"] + w["n2"]) * 2 / 1e9)},
            "forms": results, "optimal_err": opt, "oracle_prefix": prefix, "bf16_peak_tflops": peaks["bf16_tflops"],
            "roofline": roof, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk}
    del A, B
    torch.cuda.empty_cache()
    if embed:
        return line
    print(json.dumps(line), flush=True)


def run_batched(args, w, embed=False):
    """The batched form (one GPU): w["instances"] independent FP32 instances solved together through libsmp's
    server, each instance's sketch engine chosen by the autotuner; reports instances solved per second and the
    input bandwidth the whole batch sustained."""
    # many jobs run on streams of their own: let more of them reach the device concurrently (process-local)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_1610_06656_gb300 import batch, build, serve, smp, synth
    smp.load(build.build())
    torch.cuda.set_device(0)
    bf16 = args.batch_dtype == "bf16"
    tdt, sdt, esz = (torch.bfloat16, smp.SMP_BF16, 2) if bf16 else (torch.float32, smp.SMP_F32, 4)
    pool_A, pool_B, _, _, _ = synth.lowrank_plus_noise_torch(w["pool_rows"], w["width"], w["width"], w["L"],
                                                             w["sigma"], w["alpha"], seed=1004, device="cuda",
                                                             dtype=tdt)
    torch.cuda.synchronize()
    pool_bytes = 2 * pool_A.numel() * esz
    tuner = batch.EngineTuner(batch.probe_timer(pool_A, pool_B))
    t_tune = time.perf_counter()
    specs = batch.instances(w["instances"], seed=4, pool_rows=w["pool_rows"], T=w["T"])
    for sp in specs:
        tuner.choose(sp.n, sp.k, sdt)
    t_tune = time.perf_counter() - t_tune
    workers = args.workers or w["workers"]
    server = smp.smp_serve_create(int(w["budget"] - pool_bytes), solve_workers=workers)
    try:
        batch.run(server, batch.instances(w["warm"], seed=98, pool_rows=w["pool_rows"], T=w["T"]), pool_A, pool_B,
                  sdt, tuner, block_rows=w["block"])
        probe = min(specs[:50], key=lambda j: j.d * j.n)        # a small instance, for the oracle comparison
        keep = {probe.idx: (torch.empty(probe.n, probe.r, dtype=torch.float64, device="cuda"),
                            torch.empty(probe.r, dtype=torch.float64, device="cuda"),
                            torch.empty(probe.n, probe.r, dtype=torch.float64, device="cuda"))}
        clocks = ClockSampler(0)
        clocks.start()
        launches0 = smp.smp_launch_count()
        records, wall = batch.run(server, specs, pool_A, pool_B, sdt, tuner, block_rows=w["block"], keep=keep)
        launches = smp.smp_launch_count() - launches0
        clk = clocks.stop()
    finally:
        smp.smp_serve_destroy(server)
    peaks, peak_kind = measured_peaks()
    streamed = sum(sp.d * 2 * sp.n * esz for sp in specs)
    engines = {}
    names = {smp.SMP_ENGINE_SIMT: "simt", smp.SMP_ENGINE_TC: "tc", smp.SMP_ENGINE_TC_FP8: "tc_fp8"}
    for sp in specs:
        engines[names.get(sp.engine, str(sp.engine))] = engines.get(names.get(sp.engine, str(sp.engine)), 0) + 1
    lat = sorted(r["latency_ms"] for r in records)
    line = {"metric": "batched: instances solved per second (256 uneven instances together)",
            "value": len(records) / wall, "unit": "solves/s", "n_gpus": 1, "steps": len(records), "warmup": w["warm"],
            "ms_per_step": 1e3 * wall / max(1, len(records)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ("bf16" if bf16 else "tf32/f32") + " per instance (autotuned)",
            "data": "synthetic (low rank 20 + noise 0.1, column scales (j+1)^-0.5); instance inputs are windows of a "
                    "resident %d x %d %s pool pair" % (w["pool_rows"], w["width"], "BF16" if bf16 else "FP32"),
            "config": {"workload": "batch", "schedule": "staged: a budget-sized wave's sketches, then its solve chains",
                       "instances": w["instances"], "n": "uniform [64, 2048]",
                       "d": "uniform [10000, 500000]", "r": [5, 10, 20], "k": "8 r", "T": w["T"],
                       "block_rows": w["block"], "solve_workers": workers, "engines": engines,
                       "autotune_s": t_tune, "autotune_trials": tuner.trials},
            "wall_s": wall, "phases": getattr(serve.run_staged, "last_phases", None),
            "input_gb": streamed / 1e9, "input_gbs": streamed / wall / 1e9,
            "hbm_frac": streamed / wall / 1e9 / peaks["hbm_gbs"], "hbm_peak_kind": peak_kind,
            "p50_ms": statistics.median(lat), "p99_ms": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
            "gpu_launches": int(launches), "clocks": clk, "roofline": None, "cpu_baseline": None, "e2e": None}
    if not args.no_cpu_baseline:
        line["oracle"] = oracle_job_check(torch, probe, pool_A, pool_B, keep[probe.idx], w["block"],
                                          3e-3 if bf16 else 1e-3)
    del pool_A, pool_B
    torch.cuda.empty_cache()
    if embed:
        return line
    print(json.dumps(line), flush=True)


def sketch_roofline(kind, sk_bytes, sk_flops, sk_avg_s, peaks, peak_kind):
    """The sketch kernel's roofline object: kind "srht" (HBM), "tc_bf16" (BF16 tensor peak), "tc" (the TF32 peak,
    derived from the measured BF16 one, or HBM when the sketch's k / 2 flop per input byte is below the TF32 ridge),
    "simt" (FP32 FMA issue rate). sk_bytes / sk_flops: algorithmic bytes / flops per launch; sk_avg_s: mean launch
    time."""
    tf32_peak = peaks["bf16_tflops"] * (1.1 / 2.25)
    hbm = {"bound": "hbm", "achieved": sk_bytes / sk_avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "peak_kind": "%s HBM copy" % peak_kind}
    if kind == "srht":
        roof = hbm
    elif kind == "tc_bf16":
        roof = {"bound": "tensor", "achieved": sk_flops / sk_avg_s / 1e12, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "peak_kind": "%s bf16 burst" % peak_kind}
    elif kind == "tc" and sk_flops / sk_bytes * peaks["hbm_gbs"] / 1e3 < tf32_peak:
        roof = hbm
    elif kind == "tc":
        roof = {"bound": "tensor", "achieved": sk_flops / sk_avg_s / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
                "peak_kind": "%s bf16 burst x nominal tf32/bf16 ratio 1.1/2.25" % peak_kind}
    else:
        clk_mhz = peaks.get("sm_max_mhz", 2070.0)
        alu_peak = 152 * 128 * 2 * clk_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": sk_flops / sk_avg_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                "peak_kind": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x %.0f MHz" % clk_mhz}
    roof["frac"] = roof["achieved"] / roof["peak"]
    return roof


def sketch_traffic(rows_per_launch, w):
    """DRAM bytes (read + write) per sketch launch from the committed ncu capture of sketch_tc_kernel of the same
    instantiation and width (k <= 160: the n = 2,048, k = 40 block; otherwise the n = 2,000, k = 500 block), scaled
    to the rows one launch of this run processes; None when the kernel source has changed since the capture or no
    capture matches the shape."""
    import hashlib
    name = "sketch_tc_small_block.md" if w["k"] <= 160 else "sketch_tc_full_scale.md"
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            line = next(ln for ln in f if ln.startswith("bench: "))
        kv = dict(tok.split("=") for tok in line.split()[1:])
        with open(os.path.join(ROOT, "paper_1610_06656_gb300", "csrc", "sketch_tc.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, StopIteration, ValueError):
        return None
    if kv.get("sha") != sha or int(kv.get("ntot", -1)) != w["n1"] + w["n2"]:
        return None
    return float(kv["traffic_bytes"]) * rows_per_launch / float(kv["rows"])


def tc_active(w):
    """AUTO runs the tensor-core engine for binary32 blocks with k <= 512 and 16-byte aligned rows (n1, n2 multiples
    of 4 here: the bench's blocks are whole rows of contiguous tensors)."""
    return w["k"] <= 512 and w["n1"] % 4 == 0 and w["n2"] % 4 == 0


def run_e2e(torch, smp, solver, A, B, w, m, rank, steps, stream, world, dev):
    """The same solve through the C ABI with the inputs in pinned HOST memory: every step hands each 65,536-row
    block to smp_sketch_accumulate_host (the library copies it into one of its two device staging buffers on its
    copy stream while the previous block is sketched) and reads U, S, V back to pinned host memory. Also reports the
    effective host-to-device rate and this box's pinned copy rate measured alone, so the e2e time can be read as
    input bytes / link rate."""
    blk = w["block"]
    Ah = torch.empty(A.shape, dtype=A.dtype, pin_memory=True)
    Bh = torch.empty(B.shape, dtype=B.dtype, pin_memory=True)
    Ah.copy_(A)
    Bh.copy_(B)
    outU = torch.empty(w["n1"], w["r"], dtype=torch.float64, pin_memory=True)
    outS = torch.empty(w["r"], dtype=torch.float64, pin_memory=True)
    outV = torch.empty(w["n2"], w["r"], dtype=torch.float64, pin_memory=True)

    def one():
        smp.smp_sketch_reset(solver.ctx)
        for r0 in range(0, w["d"], blk):
            r1 = min(w["d"], r0 + blk)
            smp.smp_sketch_accumulate_host(solver.ctx, Ah[r0:r1], w["n1"], Bh[r0:r1], w["n2"], r0, r1 - r0)
        smp.smp_sketch_finalize(solver.ctx)
        nnz = solver.sample(m, 2 + rank)
        vals = solver.estimate(nnz)
        U, S, V = solver.waltmin(vals, w["r"], w["T"], 0, 3 + rank)
        outU.copy_(U, non_blocking=True)
        outS.copy_(S, non_blocking=True)
        outV.copy_(V, non_blocking=True)
        stream.synchronize()

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        el = max_over_ranks(el, dist, dev)
    h2d = (A.numel() * A.element_size() + B.numel() * B.element_size())
    d2h = (outU.numel() + outS.numel() + outV.numel()) * 8
    # the link alone: one pinned block pair copied host-to-device, CUDA events on a copy stream
    cs = torch.cuda.Stream(device=dev)
    dA = torch.empty(blk, w["n1"], dtype=A.dtype, device=dev)
    dB = torch.empty(blk, w["n2"], dtype=B.dtype, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(cs):
        dA.copy_(Ah[:blk], non_blocking=True)
        e0.record(cs)
        for _ in range(4):
            dA.copy_(Ah[:blk], non_blocking=True)
            dB.copy_(Bh[:blk], non_blocking=True)
        e1.record(cs)
    cs.synchronize()
    link = 4 * (dA.numel() + dB.numel()) * A.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9
    # and the whole input range once, block by block, with nothing else running
    with torch.cuda.stream(cs):
        e0.record(cs)
        for r0 in range(0, w["d"], blk):
            r1 = min(w["d"], r0 + blk)
            dA[:r1 - r0].copy_(Ah[r0:r1], non_blocking=True)
            dB[:r1 - r0].copy_(Bh[r0:r1], non_blocking=True)
        e1.record(cs)
    cs.synchronize()
    link_full = h2d / (e0.elapsed_time(e1) / 1e3) / 1e9
    del Ah, Bh, dA, dB
    return {"value": world * steps / el, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": 1e3 * el / steps, "api": "smp_sketch_accumulate_host (pinned host blocks)",
            "h2d_gbs_effective": h2d / (el / steps) / 1e9, "h2d_link_gbs_measured": link,
            "h2d_link_gbs_whole_range": link_full, "bound_ms_by_link": 1e3 * h2d / (link_full * 1e9)}


if __name__ == "__main__":
    main()
