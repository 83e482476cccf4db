"""GB300-native SMP-PCA: single-pass rank-r approximation of A^T B (arXiv 1610.06656).

The compute path is `libsmp.so` (hand-written CUDA for sm_103a behind a C ABI, declared in include/smp.h).
`paper_1610_06656_gb300.smp` is the thin ctypes binding with the same call names; it is imported lazily so
that the seeded input generator (`synth`) can be used without a GPU.
"""
__all__ = ["synth", "configs", "smp"]


def __getattr__(name):
    if name == "smp":
        from . import smp as _smp
        return _smp
    raise AttributeError(name)
