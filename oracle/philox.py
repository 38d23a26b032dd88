"""Philox4x32-10 counter-based generator and the standard normals drawn from it
(oracle side; test infrastructure).

Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each
of the 10 rounds multiplies counter words 0 and 2 by the constants 0xD2511F53 and
0xCD9E8D57 into 64-bit products and recombines
    (c0, c1, c2, c3) <- (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
then bumps the key by the Weyl constants (0x9E3779B9, 0xBB67AE85).

Normals for the sampler (the GPU side draws the same stream): normal t of sample j
comes from Philox call g = t // 4 with counter (g mod 2^32, g >> 32, j mod 2^32,
j >> 32) and key (seed mod 2^32, seed >> 32); the words (x0, x1) and (x2, x3) give two
Box-Muller pairs with uniforms u = ((x >> 8) + 1/2) 2^-24 in (0, 1):
    r = sqrt(-2 ln u_a),  z_even = r cos(2 pi u_b),  z_odd = r sin(2 pi u_b),
evaluated in float32.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: (..., 4) uint32-valued array, key: (..., 2).  Returns (..., 4) uint32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return np.stack(c, axis=-1).astype(np.uint32)


def raw_words(seed: int, sample: int, ncalls: int) -> np.ndarray:
    """The 4*ncalls 32-bit words of calls 0..ncalls-1 for one sample."""
    g = np.arange(ncalls, dtype=np.uint64)
    ctr = np.stack([g & MASK, g >> np.uint64(32),
                    np.full_like(g, np.uint64(sample) & MASK), np.full_like(g, np.uint64(sample) >> np.uint64(32))], -1)
    key = np.broadcast_to(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64), (ncalls, 2))
    return philox4x32_10(ctr, key).reshape(-1)


def normals(seed: int, first_sample: int, nsamples: int, nper: int) -> np.ndarray:
    """(nper, nsamples) float64 array of the float32 Box-Muller normals."""
    ncalls = (nper + 3) // 4
    out = np.empty((nper, nsamples))
    for j in range(nsamples):
        x = raw_words(seed, first_sample + j, ncalls).reshape(-1, 2)   # pairs (x_a, x_b)
        u = ((x >> np.uint32(8)).astype(np.float32) + np.float32(0.5)) * np.float32(2.0 ** -24)
        r = np.sqrt(np.float32(-2.0) * np.log(u[:, 0]))
        th = np.float32(2.0 * np.pi) * u[:, 1]
        z = np.empty(2 * len(u), dtype=np.float32)
        z[0::2] = r * np.cos(th)
        z[1::2] = r * np.sin(th)
        out[:, j] = z[:nper].astype(np.float64)
    return out
