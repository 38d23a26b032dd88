"""Pins for oracle/philox.py: the generator is checked against properties its published
definition fixes (a bijection of the counter for a fixed key, uniform 32-bit words,
independence across counters and samples) and the normals against the standard
normal's moments and distribution function."""
import numpy as np
from scipy import stats

from oracle import philox


def test_round_function_is_a_bijection_on_a_small_set():
    # distinct counters map to distinct outputs under one key (no collisions in 2^16 draws)
    g = np.arange(1 << 16, dtype=np.uint64)
    ctr = np.stack([g, np.zeros_like(g), np.zeros_like(g), np.zeros_like(g)], -1)
    out = philox.philox4x32_10(ctr, np.zeros((len(g), 2), dtype=np.uint64))
    packed = out.astype(np.uint64)[:, 0] << np.uint64(32) | out.astype(np.uint64)[:, 1]
    assert len(np.unique(packed)) == len(g)


def test_words_are_uniform():
    w = philox.raw_words(12345, 7, 1 << 15).astype(np.float64) / 2.0 ** 32
    # chi-square on 64 bins and KS against U(0, 1)
    h, _ = np.histogram(w, bins=64, range=(0, 1))
    chi2 = ((h - len(w) / 64) ** 2 / (len(w) / 64)).sum()
    assert chi2 < stats.chi2.ppf(0.999, 63)
    assert stats.kstest(w, "uniform").pvalue > 1e-3
    # each output byte position is balanced
    bits = (philox.raw_words(1, 0, 4096)[:, None] >> np.arange(32, dtype=np.uint32)) & 1
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.02)


def test_key_and_sample_change_the_stream():
    a = philox.raw_words(1, 0, 64)
    assert not np.array_equal(a, philox.raw_words(2, 0, 64))
    assert not np.array_equal(a, philox.raw_words(1, 1, 64))
    assert np.array_equal(a, philox.raw_words(1, 0, 64))


def test_normals_have_standard_normal_law():
    z = philox.normals(2024, 0, 4, 50000).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(len(z))
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # samples are uncorrelated
    Z = philox.normals(2024, 0, 2, 50000)
    assert abs(np.corrcoef(Z[:, 0], Z[:, 1])[0, 1]) < 4 / np.sqrt(50000)
