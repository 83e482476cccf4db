"""Shared helpers of the GPU parity tests: build/load libsmp, move Omega and the sketch to numpy."""
import ctypes
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    return torch


def build_lib():
    from paper_1610_06656_gb300 import build, smp
    smp.load(build.build())
    return smp


def omega_numpy(solver):
    om = solver.omega()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in om.items()}


def csr_rows(row_ptr):
    return np.repeat(np.arange(row_ptr.shape[0] - 1), np.diff(row_ptr))


_PROBE = None


def philox_probe():
    """Compile tests/cuda/philox_check.cu (libsmp's device Philox next to cuRAND's) into a test library."""
    global _PROBE
    if _PROBE is None:
        out_dir = os.path.join(ROOT, "paper_1610_06656_gb300", "_build")
        os.makedirs(out_dir, exist_ok=True)
        so = os.path.join(out_dir, "philox_check.so")
        src = os.path.join(ROOT, "tests", "cuda", "philox_check.cu")
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                               "-Xcompiler", "-fPIC", "-shared", "-o", so, src])
        lib = ctypes.CDLL(so)
        lib.philox_pair.restype = ctypes.c_int
        lib.philox_pair.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 2
        _PROBE = lib
    return _PROBE
