"""The workloads the method is measured and checked on (sizes and generator parameters)."""
import math

# name -> dict(d, n1, n2, L, sigma, alpha, k, r, T, block_rows, dtype)
WORKLOADS = {
    # plain SMP-PCA, tiny: checked against the exact A^T B followed by a truncated SVD
    "tiny": dict(d=2000, n1=200, n2=200, L=10, sigma=0.1, alpha=0.5, k=100, r=5, T=10, block_rows=65536,
                 dtype="f64"),
    # plain SMP-PCA at scale, FP32 storage, 65,536-row blocks
    "scale": dict(d=1_000_000, n1=2000, n2=2000, L=20, sigma=0.1, alpha=0.5, k=500, r=10, T=10,
                  block_rows=65536, dtype="f32"),
    # precision form: BF16 storage
    "precision": dict(d=4_000_000, n1=4096, n2=4096, L=32, sigma=0.05, alpha=0.7, k=1024, r=20, T=15,
                      block_rows=65536, dtype="bf16"),
}


def default_m(n1, n2, r):
    """m = 4 n r ln n, n = max(n1, n2) (Section 4 default sampling budget)."""
    n = max(n1, n2)
    return 4.0 * n * r * math.log(n)
