"""CPU binary64 oracle for SMP-PCA (arXiv 1610.06656), written from the paper.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s `cpu_baseline` /
`--impl reference` legs may import it. The product (`paper_1610_06656_gb300`) never imports it and shares no
code with it.
"""
from . import philox, smp  # noqa: F401
