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


def test_box_muller_pairs_are_independent_normals():
    # the two normals of one Box-Muller pair (entries 2i, 2i + 1 of a sample) are
    # uncorrelated, their squared radius is chi-square with 2 degrees of freedom
    # (exponential, mean 2) and their angle is uniform: a pair built from one trigonometric
    # function twice, or a radius without the factor 2, fails here
    z = philox.normals(77, 3, 1, 100000)[:, 0]
    a, b = z[0::2], z[1::2]
    assert abs(np.corrcoef(a, b)[0, 1]) < 4 / np.sqrt(len(a))
    assert abs(np.corrcoef(a ** 2, b ** 2)[0, 1]) < 4 / np.sqrt(len(a))
    r2 = a ** 2 + b ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-3
    assert stats.kstest(np.arctan2(b, a), "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3


_TRITON_PHILOX = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"   # Triton's CPU interpreter: no GPU needed
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    r0, r1, r2, r3 = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(o0 + i, r0)
    tl.store(o1 + i, r1)
    tl.store(o2 + i, r2)
    tl.store(o3 + i, r3)

ctr = np.load(sys.argv[1])
seed = int(sys.argv[2])
cs = [torch.from_numpy(np.ascontiguousarray(ctr[:, j]).view(np.int32)) for j in range(4)]
outs = [torch.empty(ctr.shape[0], dtype=torch.int32) for _ in range(4)]
k[(1,)](*cs, *outs, seed, N=ctr.shape[0])
np.save(sys.argv[3], np.stack([o.numpy().view(np.uint32) for o in outs], -1))
"""


def test_equals_an_independent_library_philox(tmp_path):
    # Triton ships its own Philox4x32-10 (tl.philox: key = the seed's low and high words,
    # ten rounds); run through its CPU interpreter it must give the oracle's words exactly,
    # which pins the round constants, the key schedule and the round count
    import os
    import subprocess
    import sys

    import pytest
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, (64, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [0, 0, 0, 1]]
    for seed in (0, 20240607, (0xBEEF << 32) | 0x12345678):
        src, out = tmp_path / "ctr.npy", tmp_path / "out.npy"
        np.save(src, ctr)
        script = tmp_path / "tri.py"
        script.write_text(_TRITON_PHILOX)
        env = {**os.environ, "TRITON_INTERPRET": "1"}
        subprocess.run([sys.executable, str(script), str(src), str(seed), str(out)], check=True, env=env,
                       timeout=300)
        key = np.stack([np.full(len(ctr), seed & 0xFFFFFFFF, np.uint64), np.full(len(ctr), seed >> 32, np.uint64)],
                       -1)
        ref = philox.philox4x32_10(ctr.astype(np.uint64), key).astype(np.uint32)
        assert np.array_equal(ref, np.load(out)), seed
