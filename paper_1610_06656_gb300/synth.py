"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of SMP-PCA's arithmetic: it only draws the input matrices A (d x n1) and B (d x n2).
Both the CUDA path's tests/benchmark and the CPU oracle's tests consume its output, byte for byte.

Generators:
  * low rank plus noise with power-law column scales: A = Z X^T + sigma N1, B = Z Y^T + sigma N2, with Z (d x L),
    X (n1 x L), Y (n2 x L), N1, N2 i.i.d. N(0, 1); column j (0-based) of each matrix is multiplied by
    (j + 1)^-alpha. With same_ab the call returns A only (the PCA case A = B, Section 3, Remark 3).
  * the paper's synthetic matrix G D, G i.i.d. N(0, 1), D_ii = 1/i (Section 4, "Description of datasets").
  * unit columns drawn from a cone of half-angle theta around one direction (Section 4, the comparison with
    SVD(A~^T B~) and the estimator figure): each column is cos(phi) e + sin(phi) w with e a fixed random unit
    vector, w a random unit vector orthogonal to e, and phi uniform in [0, theta] (reading: the paper names the
    cone angle only).
"""
import numpy as np


def column_scale(n, alpha):
    return (np.arange(1, n + 1, dtype=np.float64) ** (-float(alpha)))


def lowrank_plus_noise(d, n1, n2, L, sigma, alpha, seed, dtype=np.float32, same_ab=False):
    """CPU (numpy) generator; returns (A, B) in `dtype` (B is None when same_ab)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = rng.standard_normal((d, L))
    X = rng.standard_normal((n1, L))
    A = Z @ X.T + sigma * rng.standard_normal((d, n1))
    A *= column_scale(n1, alpha)[None, :]
    if same_ab:
        return A.astype(dtype), None
    Y = rng.standard_normal((n2, L))
    B = Z @ Y.T + sigma * rng.standard_normal((d, n2))
    B *= column_scale(n2, alpha)[None, :]
    return A.astype(dtype), B.astype(dtype)


def gd_matrix(d, n, seed, dtype=np.float64):
    """The paper's synthetic G D (D_ii = 1/i, 1-based), Section 4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    G = rng.standard_normal((d, n))
    return (G / np.arange(1, n + 1, dtype=np.float64)[None, :]).astype(dtype)


def lowrank_plus_noise_torch(d, n1, n2, L, sigma, alpha, seed, device, dtype=None, same_ab=False,
                             block_rows=65536):
    """Device-side generator for the large workloads (torch RNG, seeded); same model as lowrank_plus_noise.

    Returns (A, B, Z, X, Y) so a checker can recompute any column of A^T B from the latent factors.
    Generated in row blocks to bound temporary memory.
    """
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    X = torch.randn(n1, L, generator=g, device=device, dtype=torch.float32)
    Y = None if same_ab else torch.randn(n2, L, generator=g, device=device, dtype=torch.float32)
    sa = torch.arange(1, n1 + 1, device=device, dtype=torch.float32).pow(-float(alpha))
    sb = None if same_ab else torch.arange(1, n2 + 1, device=device, dtype=torch.float32).pow(-float(alpha))
    A = torch.empty(d, n1, device=device, dtype=dtype)
    B = None if same_ab else torch.empty(d, n2, device=device, dtype=dtype)
    Z = torch.empty(d, L, device=device, dtype=torch.float32)
    for r0 in range(0, d, block_rows):
        r1 = min(d, r0 + block_rows)
        z = torch.randn(r1 - r0, L, generator=g, device=device, dtype=torch.float32)
        Z[r0:r1] = z
        a = (z @ X.T + sigma * torch.randn(r1 - r0, n1, generator=g, device=device)) * sa
        A[r0:r1] = a.to(dtype)
        if not same_ab:
            b = (z @ Y.T + sigma * torch.randn(r1 - r0, n2, generator=g, device=device)) * sb
            B[r0:r1] = b.to(dtype)
    return A, B, Z, X, Y


def gd(d, n, seed, dtype=np.float64):
    """Section 4's synthetic matrices: G D with G (d x n) standard Gaussian and D_ii = 1 / i (i from 1)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((d, n)) / np.arange(1, n + 1)).astype(dtype)


def gd_torch(d, n, seed, device, block_rows=8192):
    """Device-side G D (binary32, torch RNG seeded), generated in row blocks to bound temporary memory."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    dscale = 1.0 / torch.arange(1, n + 1, device=device, dtype=torch.float32)
    A = torch.empty(d, n, device=device, dtype=torch.float32)
    for r0 in range(0, d, block_rows):
        r1 = min(d, r0 + block_rows)
        A[r0:r1] = torch.randn(r1 - r0, n, generator=g, device=device, dtype=torch.float32) * dscale
    return A


def cone(d, n1, n2, theta, seed, dtype=np.float64):
    """A (d x n1) and B (d x n2) with unit columns at angle phi ~ U[0, theta] from one shared random direction."""
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(d)
    e /= np.linalg.norm(e)

    def draw(n):
        W = rng.standard_normal((d, n))
        W -= np.outer(e, e @ W)
        W /= np.linalg.norm(W, axis=0)
        phi = rng.uniform(0.0, theta, size=n)
        return (np.outer(e, np.cos(phi)) + W * np.sin(phi)).astype(dtype)

    return draw(n1), draw(n2)
