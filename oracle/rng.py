"""Counter-based random number generators of the oracle (test infrastructure only).

The paper draws Gaussian signals (Alg. 2 step 3, variance 1/d) and uniform
samples (Sec. 3.2) without fixing a generator.  Both sides of the parity
tests implement the same two published generators independently:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11): a 10-round Feistel-like bijection of a 128-bit
  counter under a 64-bit key, with multipliers 0xD2511F53 and 0xCD9E8D57 and
  Weyl key increments 0x9E3779B9 and 0xBB67AE85.
* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output t of the generator
  seeded with s is mix(s + t * 0x9E3779B97F4A7C15) with the variant-13 mixer.

Gaussian block convention (shared reading of Alg. 2 step 3): element (i, c)
of an N x d block uses counter (i mod 2^32, i div 2^32, c div 4, 0) and key
(seed mod 2^32, (seed div 2^32) xor stream).  Each of the four 32-bit outputs
x becomes the uniform u = (x >> 9) * 2^-23 + 2^-24, exactly representable in
fp32, in (0, 1).  Box-Muller on (u0, u1) gives columns 4q and 4q+1 as
r cos(2 pi u1), r sin(2 pi u1) with r = sqrt(-2 ln u0); (u2, u3) give 4q+2 and
4q+3 the same way.  The values are then scaled by sigma.

Pins: Philox against the known-answer vectors of its publication's test
suite (tests/golden/philox4x32_10_kat.txt); SplitMix64 against its
reference outputs for seed 0 (tests/golden/splitmix64_kat.txt); the
Gaussian block against its first two moments and a Kolmogorov-Smirnov test.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_SIGNALS = 0x5349474E   # Gaussian signal block of Alg. 2 step 3
STREAM_PROBES = 0x50524F42    # eigencount probe vectors of Sec. 4.3
STREAM_KMEANS = 0x4B4D4541    # k-means++ draws


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit counters (as uint64 arrays)."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0           # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return c0, c1, c2, c3


def _key(seed: int, stream: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, ((seed >> 32) ^ int(stream)) & 0xFFFFFFFF


def uniform_from_bits(x) -> np.ndarray:
    """u = (x >> 9) * 2^-23 + 2^-24 in (0, 1), exact in fp32."""
    x = np.asarray(x, dtype=np.uint64)
    return (x >> np.uint64(9)).astype(np.float64) * 2.0 ** -23 + 2.0 ** -24


def philox_bits_block(n: int, d: int, seed: int, stream: int):
    """The four Philox words for every (row, column-quad) of an n x d block."""
    q = (d + 3) // 4
    rows = np.repeat(np.arange(n, dtype=np.uint64), q)
    quads = np.tile(np.arange(q, dtype=np.uint64), n)
    k0, k1 = _key(seed, stream)
    x = philox4x32_10(rows & MASK32, rows >> np.uint64(32), quads, np.zeros_like(rows),
                      np.full(rows.shape, k0, np.uint64), np.full(rows.shape, k1, np.uint64))
    return [xi.reshape(n, q) for xi in x]


def gaussian_block(n: int, d: int, d_pad: int, seed: int, stream: int, sigma: float) -> np.ndarray:
    """N x d_pad float64 block of N(0, sigma^2) values by the convention above; padding = 0."""
    out = np.zeros((n, d_pad), dtype=np.float64)
    if n == 0 or d == 0:
        return out
    x0, x1, x2, x3 = philox_bits_block(n, d, seed, stream)
    u0, u1, u2, u3 = (uniform_from_bits(v) for v in (x0, x1, x2, x3))
    r01 = np.sqrt(-2.0 * np.log(u0))
    r23 = np.sqrt(-2.0 * np.log(u2))
    z = np.empty((n, x0.shape[1] * 4), dtype=np.float64)
    z[:, 0::4] = r01 * np.cos(2 * np.pi * u1)
    z[:, 1::4] = r01 * np.sin(2 * np.pi * u1)
    z[:, 2::4] = r23 * np.cos(2 * np.pi * u3)
    z[:, 3::4] = r23 * np.sin(2 * np.pi * u3)
    out[:, :d] = z[:, :d] * sigma
    return out


def uniform_draw(seed: int, stream: int, a: int, b: int) -> float:
    """One uniform in (0, 1) from Philox counter (a, b, 0, 0): word 0."""
    k0, k1 = _key(seed, stream)
    x = philox4x32_10(a & 0xFFFFFFFF, (a >> 32) & 0xFFFFFFFF, b & 0xFFFFFFFF, 0, k0, k1)
    return float(uniform_from_bits(x[0]))


# ---------------------------------------------------------------------------
# SplitMix64
# ---------------------------------------------------------------------------
GOLDEN64 = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_mix_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_outputs(seed: int, count: int):
    """The first ``count`` outputs of SplitMix64 seeded with ``seed`` (Python ints)."""
    return [splitmix64_mix_int(seed + (t + 1) * GOLDEN64) for t in range(count)]


def _mul64(a: np.ndarray, c: int) -> np.ndarray:
    """(a * c) mod 2^64 for uint64 arrays, by 32-bit limbs (no reliance on overflow)."""
    a = a.astype(np.uint64)
    c_lo, c_hi = np.uint64(c & 0xFFFFFFFF), np.uint64(c >> 32)
    a_lo, a_hi = a & MASK32, a >> np.uint64(32)
    lo = a_lo * c_lo
    mid = ((a_lo * c_hi) & MASK32) + ((a_hi * c_lo) & MASK32) + (lo >> np.uint64(32))
    return ((mid & MASK32) << np.uint64(32)) | (lo & MASK32)


def _add64(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a_lo, a_hi = a & MASK32, a >> np.uint64(32)
    b_lo, b_hi = b & MASK32, b >> np.uint64(32)
    lo = a_lo + b_lo
    hi = (a_hi + b_hi + (lo >> np.uint64(32))) & MASK32
    return (hi << np.uint64(32)) | (lo & MASK32)


def splitmix64_at(seed: int, t: np.ndarray) -> np.ndarray:
    """Output number t (0-based) of SplitMix64 seeded with ``seed``, vectorised over t."""
    t = np.asarray(t, dtype=np.uint64)
    z = _add64(np.full(t.shape, int(seed) & _M64, dtype=np.uint64), _mul64(t + np.uint64(1), GOLDEN64))
    z = _mul64(z ^ (z >> np.uint64(30)), 0xBF58476D1CE4E5B9)
    z = _mul64(z ^ (z >> np.uint64(27)), 0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))
