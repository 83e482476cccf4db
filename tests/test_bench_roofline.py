"""bench.py's roofline bookkeeping on CPU: which peak a sketch is measured against (the TF32 tensor peak above the
TF32 ridge, HBM below it, BF16 for BF16 operands, HBM for the SRHT, the FP32 FMA rate for the CUDA-core engine) and
when the committed ncu capture's DRAM traffic applies (same kernel source hash and same width, scaled by rows)."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}


def _launch(k, ntot, rows=65536):
    return rows * ntot * 4.0, 2.0 * k * rows * ntot   # algorithmic bytes, flops


def test_tf32_sketch_above_the_ridge_is_tensor_bound():
    b, f = _launch(500, 4000)
    roof = bench.sketch_roofline("tc", b, f, 0.5e-3, PEAKS, "measured")
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["peak"] == pytest.approx(1900.0 * 1.1 / 2.25)
    assert roof["achieved"] == pytest.approx(f / 0.5e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])


@pytest.mark.parametrize("k", [40, 80, 160])
def test_tf32_sketch_below_the_ridge_is_hbm_bound(k):
    b, f = _launch(k, 4096)   # k / 2 flop per byte: 20-80, the TF32 ridge here is ~136
    roof = bench.sketch_roofline("tc", b, f, 0.32e-3, PEAKS, "measured")
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(b / 0.32e-3 / 1e9)
    assert roof["frac"] == pytest.approx(b / 0.32e-3 / 1e9 / 6800.0)


def test_other_engines():
    b, f = _launch(500, 4000)
    assert bench.sketch_roofline("tc_bf16", b, f, 1e-3, PEAKS, "m")["peak"] == 1900.0
    assert bench.sketch_roofline("srht", b, f, 1e-3, PEAKS, "m")["bound"] == "hbm"
    simt = bench.sketch_roofline("simt", b, f, 1e-3, PEAKS, "m")
    assert simt["bound"] == "alu" and simt["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)


def test_sketch_traffic_applies_only_to_the_captured_source_and_width(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_1610_06656_gb300", "csrc", "sketch_tc.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "sketch_tc_full_scale.md").write_text("x\nbench: traffic_bytes=1000 rows=100 ntot=4000 sha=%s\n" % sha)
    (prof / "sketch_tc_small_block.md").write_text("bench: traffic_bytes=500 rows=100 ntot=4096 sha=0000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_1610_06656_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_1610_06656_gb300" / "csrc" / "sketch_tc.cu").write_bytes(open(src, "rb").read())
    assert bench.sketch_traffic(200, {"k": 500, "n1": 2000, "n2": 2000}) == pytest.approx(2000.0)
    assert bench.sketch_traffic(200, {"k": 500, "n1": 2048, "n2": 2048}) is None        # another width
    assert bench.sketch_traffic(200, {"k": 40, "n1": 2048, "n2": 2048}) is None         # another source hash


def test_auto_engine_is_the_tensor_core_one_for_the_bench_shapes():
    assert bench.tc_active(bench.WORKLOADS["scale"]) and bench.tc_active(bench.WORKLOADS["block_batch"])
    assert not bench.tc_active(dict(bench.WORKLOADS["scale"], k=1024))
