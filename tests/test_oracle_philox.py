"""Pins for the oracle's random streams (Philox4x32-10, Box-Muller, the 53-bit uniform)."""
import numpy as np
import pytest
from scipy import stats

from oracle import philox

M32 = 0xFFFFFFFF


def _inv_mod32(a):
    return pow(a, -1, 1 << 32)


def _philox_inverse(out, key):
    """Undo ten Philox-4x32 rounds, derived independently from the round definition (Salmon et al. 2011):
    the low product halves give back the multiplied words (multipliers are odd, so invertible mod 2^32), and the
    high halves then unmask the other two words."""
    y0, y1, y2, y3 = out
    keys = []
    k0, k1 = key
    for rnd in range(10):
        if rnd:
            k0 = (k0 + 0x9E3779B9) & M32
            k1 = (k1 + 0xBB67AE85) & M32
        keys.append((k0, k1))
    inv0, inv1 = _inv_mod32(0xD2511F53), _inv_mod32(0xCD9E8D57)
    for k0, k1 in reversed(keys):
        c2 = (y1 * inv1) & M32
        c0 = (y3 * inv0) & M32
        c1 = y0 ^ ((0xCD9E8D57 * c2) >> 32) ^ k0
        c3 = y2 ^ ((0xD2511F53 * c0) >> 32) ^ k1
        y0, y1, y2, y3 = c0, c1, c2, c3
    return y0, y1, y2, y3


def test_scalar_matches_vectorised():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 1 << 32, size=(4, 300), dtype=np.uint64)
    for key in [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (12345, 678)]:
        v = philox.philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], *key)
        for e in range(ctr.shape[1]):
            s = philox.philox4x32_10_scalar(tuple(int(c[e]) for c in ctr), key)
            assert s == tuple(int(w[e]) for w in v)


def test_round_structure_is_invertible():
    rng = np.random.default_rng(11)
    for _ in range(200):
        ctr = tuple(int(x) for x in rng.integers(0, 1 << 32, size=4, dtype=np.uint64))
        key = tuple(int(x) for x in rng.integers(0, 1 << 32, size=2, dtype=np.uint64))
        assert _philox_inverse(philox.philox4x32_10_scalar(ctr, key), key) == ctr


def test_output_bits_balanced_and_uniform():
    n = 1 << 18
    c = np.arange(n, dtype=np.uint64)
    words = philox.philox4x32_10(c, 0, 0, philox.TAG_PI, 42, 0)
    for w in words:
        bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)).mean(axis=0)
        assert np.all(np.abs(bits - 0.5) < 6 * 0.5 / np.sqrt(n))
        top = (w >> np.uint64(24)).astype(np.int64)
        counts = np.bincount(top, minlength=256)
        chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-6


def test_avalanche_on_counter_bit():
    rng = np.random.default_rng(3)
    base = rng.integers(0, 1 << 32, size=(4, 4000), dtype=np.uint64)
    out0 = philox.philox4x32_10(*base, 9, 9)
    for bit in (0, 13, 31):
        flipped = base.copy()
        flipped[0] ^= np.uint64(1 << bit)
        out1 = philox.philox4x32_10(*flipped, 9, 9)
        for a, b in zip(out0, out1):
            x = a ^ b
            pop = np.array([bin(int(v)).count("1") for v in x])
            assert abs(pop.mean() - 16.0) < 0.3


def test_uniform_maps_are_exact_and_in_range():
    lo = np.array([0], dtype=np.uint64)
    hi = np.array([M32], dtype=np.uint64)
    # u1 in (0, 1], u2 in [0, 1)
    rho_lo, _ = philox.box_muller(hi, lo)       # u1 = 1 -> rho = 0
    assert rho_lo[0] == 0.0
    z0, z1 = philox.box_muller(lo, lo)          # u1 = 2^-24, u2 = 0 -> (rho, 0)
    assert z0[0] == pytest.approx(np.sqrt(2 * 24 * np.log(2.0)), rel=1e-15)
    assert z1[0] == 0.0
    assert philox.uniform53(lo, lo)[0] == 0.0
    assert philox.uniform53(hi, hi)[0] == 1.0 - 2.0 ** -53


def test_box_muller_is_standard_normal():
    n = 1 << 19
    c = np.arange(n, dtype=np.uint64)
    x0, x1, x2, x3 = philox.philox4x32_10(c, 0, 0, philox.TAG_PI, 2024, 1)
    z = np.concatenate(philox.box_muller(x0, x1) + philox.box_muller(x2, x3))
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 6 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * np.sqrt(2 / z.size)
    assert abs(stats.kurtosis(z, fisher=False) - 3) < 6 * np.sqrt(24 / z.size)
    # pairs are independent
    za, zb = philox.box_muller(x0, x1)
    assert abs(np.corrcoef(za, zb)[0, 1]) < 6 / np.sqrt(n)


def test_uniform53_is_uniform():
    n = 1 << 18
    u = philox.coin_uniforms(5, philox.TAG_SAMPLE, np.arange(n, dtype=np.uint64), np.uint64(17))
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert u.min() >= 0.0 and u.max() < 1.0


def test_streams_are_separated_by_tag_and_seed():
    c = np.arange(1 << 14, dtype=np.uint64)
    a = philox.coin_uniforms(1, philox.TAG_SAMPLE, c, np.uint64(0))
    b = philox.coin_uniforms(1, philox.TAG_SPLIT, c, np.uint64(0))
    d = philox.coin_uniforms(2, philox.TAG_SAMPLE, c, np.uint64(0))
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.05 and abs(np.corrcoef(a, d)[0, 1]) < 0.05
