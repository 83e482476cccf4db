"""The C-ABI library builds for sm_103a, loads, and exports every call include/smp.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1610_06656_gb300 import build as smp_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_calls():
    text = open(os.path.join(ROOT, "include", "smp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return smp_build.build()


def test_header_declares_the_path():
    calls = declared_calls()
    for name in ["smp_sketch_begin", "smp_sketch_accumulate", "smp_sketch_finalize", "smp_sample", "smp_estimate",
                 "smp_waltmin", "smp_destroy"]:
        assert name in calls


def test_library_exports_every_declared_call(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_calls():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_call(lib_path):
    from paper_1610_06656_gb300 import smp
    assert sorted(smp.SIGNATURES) == declared_calls()
    smp.load(lib_path)
    assert smp.smp_version() == 100
    assert smp.status_string(smp.SMP_ESTATE) == "SMP_ESTATE"
