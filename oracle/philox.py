"""Philox4x32-10 and the uniform / Gaussian mappings the method draws its randomness from.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links this module; only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of `bench.py` use it.

Source of the generator: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
(SC'11), section on Philox. A Philox-4x32 round multiplies two of the four counter words by fixed odd
constants, keeps the high and low 32-bit halves of each 64-bit product, and mixes the high halves with the
other two words and the round key; the key is bumped by two Weyl constants between rounds. Ten rounds.

The paper being implemented only asks for Pi(i, j) ~ N(0, 1/k) i.i.d. (Algorithm 1, step 2, and Section 2.1,
"Step 1"); it does not say how to draw them. The reading used on both sides of the parity tests:

  key            = (seed mod 2^32, seed >> 32)
  Pi(a, t)       : counter = (t mod 2^32, t >> 32, a // 4, TAG_PI)      a = sketch row, t = data row
                   words (x0, x1) feed rows a = 4g, 4g+1 and (x2, x3) feed rows 4g+2, 4g+3
  Box-Muller     : u1 = ((x_even >> 8) + 1) * 2^-24  in (0, 1]
                   u2 = (x_odd  >> 8)      * 2^-24  in [0, 1)
                   rho = sqrt(-2 ln u1);  z_even = rho cos(2 pi u2);  z_odd = rho sin(2 pi u2)
                   Pi(a, t) = z / sqrt(k)
  sample coin    : counter = (i, j, 0, TAG_SAMPLE); u = ((x0 >> 5) * 2^26 + (x1 >> 6)) * 2^-53 in [0, 1)
  split coin     : counter = (i, j, 0, TAG_SPLIT), same 53-bit mapping
  init block     : counter = (i, 0, c // 4, TAG_INIT), same Gaussian mapping as Pi (no 1/sqrt(k))
  multinomial    : counter = (i, s, 0, TAG_MULTI) for draw s of row i, same 53-bit mapping as the coins
  SRHT sign      : counter = (t mod 2^32, t >> 32, 0, TAG_SRHT_SIGN); D_tt = -1 iff bit 0 of x0 is set
  SRHT row       : counter = (a, b mod 2^32, b >> 32, TAG_SRHT_ROW); row a of block b samples Hadamard row
                   x0 >> (32 - p) of the 2^p-row block

Both uniforms are exact in binary32 and binary64, so the two sides see identical uniforms; they differ only in
how ln / sqrt / cos / sin are rounded.
"""
import numpy as np

MASK32 = 0xFFFFFFFF
# Philox-4x32 multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
ROUNDS = 10

TAG_PI = 1
TAG_SAMPLE = 2
TAG_SPLIT = 3
TAG_INIT = 4
TAG_MULTI = 5
TAG_SRHT_SIGN = 6
TAG_SRHT_ROW = 7

TWO_M24 = 2.0 ** -24
TWO_M53 = 2.0 ** -53


def seed_key(seed):
    """Split a 64-bit seed into the two 32-bit Philox key words."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32


def philox4x32_10_scalar(ctr, key):
    """One Philox4x32-10 block on Python ints: ctr = 4 words, key = 2 words -> 4 words."""
    c0, c1, c2, c3 = (int(x) & MASK32 for x in ctr)
    k0, k1 = (int(x) & MASK32 for x in key)
    for rnd in range(ROUNDS):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0), (p1 & MASK32), ((p0 >> 32) ^ c3 ^ k1), (p0 & MASK32)
    return c0, c1, c2, c3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over numpy arrays (broadcast). Returns four uint64 arrays of 32-bit words.

    32x32 -> 64-bit products are exact in uint64, so the high and low halves are a shift and a mask.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    sh = np.uint64(32)
    msk = np.uint64(MASK32)
    for rnd in range(ROUNDS):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = m0 * c0
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> sh) ^ c1 ^ np.uint64(k0)), (p1 & msk), ((p0 >> sh) ^ c3 ^ np.uint64(k1)), (p0 & msk)
    return c0, c1, c2, c3


def box_muller(x_even, x_odd):
    """Two 32-bit words -> two standard normals (binary64), with the uniform mapping above."""
    u1 = ((np.asarray(x_even, dtype=np.uint64) >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * TWO_M24
    u2 = (np.asarray(x_odd, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * TWO_M24
    rho = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rho * np.cos(ang), rho * np.sin(ang)


def uniform53(x0, x1):
    """Two 32-bit words -> a uniform in [0, 1) with 53 random bits (exact in binary64)."""
    hi = (np.asarray(x0, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    lo = (np.asarray(x1, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo) * TWO_M53


def gaussian_rows(seed, tag, nrows_out, col_ids, word1_ids):
    """Standard normals G[a, c] for a in [0, nrows_out) and the given column ids.

    Counter (col_lo, col_hi/word1, a // 4, tag). Used for Pi (col = data row t, word1 = t >> 32) and for the
    deterministic start block of the initial subspace iteration.
    """
    k0, k1 = seed_key(seed)
    ngroups = (nrows_out + 3) // 4
    col_ids = np.asarray(col_ids, dtype=np.uint64)
    word1_ids = np.asarray(word1_ids, dtype=np.uint64)
    g = np.arange(ngroups, dtype=np.uint64)[:, None]
    x0, x1, x2, x3 = philox4x32_10(col_ids[None, :], word1_ids[None, :], g, np.uint64(tag), k0, k1)
    z0, z1 = box_muller(x0, x1)
    z2, z3 = box_muller(x2, x3)
    out = np.empty((4 * ngroups, col_ids.shape[0]), dtype=np.float64)
    out[0::4] = z0
    out[1::4] = z1
    out[2::4] = z2
    out[3::4] = z3
    return out[:nrows_out]


def pi_block(seed, k, t0, nrows):
    """Rows [t0, t0 + nrows) of Pi, as the k x nrows block Pi[:, t0:t0+nrows] (entries N(0, 1/k))."""
    t = np.arange(t0, t0 + nrows, dtype=np.uint64)
    g = gaussian_rows(seed, TAG_PI, k, t & np.uint64(MASK32), t >> np.uint64(32))
    return g / np.sqrt(float(k))


def coin_uniforms(seed, tag, rows, cols):
    """53-bit uniforms u(i, j) for the given (broadcast) row and column index arrays."""
    k0, k1 = seed_key(seed)
    x0, x1, _, _ = philox4x32_10(np.asarray(rows, dtype=np.uint64), np.asarray(cols, dtype=np.uint64),
                                 np.uint64(0), np.uint64(tag), k0, k1)
    return uniform53(x0, x1)
