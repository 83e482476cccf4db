"""GB300-native SMP-PCA: single-pass rank-r approximation of A^T B (arXiv 1610.06656).

The compute path is `libsmp.so` (hand-written CUDA for sm_103a behind a C ABI, declared in include/smp.h).
`paper_1610_06656_gb300.smp` is the thin ctypes binding with the same call names and
`paper_1610_06656_gb300.pipeline` chains the calls; neither is imported here, so the seeded input generator
(`synth`) can be used without a GPU or a built library.
"""
