"""Counter-based Rademacher streams, oracle implementation.

The paper draws isotropic random vectors with E|z_i|^2 = 1 and E z_i z_j = 0
(eq. random_props) and names Rademacher vectors, z uniform in {-1, 1}
(Section 1).  Both the CUDA library and this oracle must draw the SAME
vectors without exchanging them, so each implements the same counter-based
generator from its published definition:

  mix64(z)   the SplitMix64 output finaliser (Steele, Lea & Flood, "Fast
             splittable pseudorandom number generators", OOPSLA 2014):
               z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
               z ^= z >> 27; z *= 0x94D049BB133111EB;
               z ^= z >> 31            (all arithmetic mod 2^64)
  key        = mix64(seed ^ mix64((level << 56) | (phase << 48) | sample))
  word(i)    = mix64(key + GAMMA * (i + 1)),   GAMMA = 0x9E3779B97F4A7C15
  sign(i)    = +1 if the top bit of word(i) is 0, else -1

`sample` < 2^48, `level` < 256, `phase` < 256.  A real Rademacher vector of
length n has entries sign(0..n-1); a complex one (used for multigrid test
vectors) has re = sign(2i), im = sign(2i+1).

Z4 noise (the complex alternative of Section 2, whose Hutchinson variance is
||offdiag(A)||_F^2 instead of 1/2 ||offdiag(A + A^T)||_F^2): entry i is
i^q with q = the top two bits of word(i) (q = word(i) >> 62), i.e. one of
1, i, -1, -i with equal probability; E|z|^2 = 1, E z = E z^2 = 0.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

PHASE_STOCH = 0     # stochastic samples zeta_s (Algorithm 2, stochastic part)
PHASE_SKETCH = 1    # sketch vectors S_l (Algorithm 2, deflation part)
PHASE_TESTVEC = 2   # multigrid set-up test vectors
PHASE_HUTCH = 3     # plain Hutchinson samples (Algorithm 1)
PHASE_HARVEST = 5   # right-hand sides of the learned preconditioner's training pairs


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, level: int, phase: int, sample: int) -> np.uint64:
    assert 0 <= level < 256 and 0 <= phase < 256 and 0 <= sample < (1 << 48)
    ctr = np.uint64((level << 56) | (phase << 48) | sample)
    return mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ mix64(ctr))


def words(seed: int, level: int, phase: int, sample: int, count: int) -> np.ndarray:
    key = stream_key(seed, level, phase, sample)
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + GAMMA * i)


def rademacher(seed: int, level: int, phase: int, sample: int, n: int) -> np.ndarray:
    """Real +-1 vector of length n (float64)."""
    w = words(seed, level, phase, sample, n)
    return np.where((w >> np.uint64(63)) == 0, 1.0, -1.0)


def rademacher_block(seed: int, level: int, phase: int, sample0: int, n: int, k: int) -> np.ndarray:
    """n x k matrix whose column j is rademacher(..., sample0 + j, n) (complex128)."""
    return np.stack([rademacher(seed, level, phase, sample0 + j, n) for j in range(k)],
                    axis=1).astype(complex)


def z4(seed: int, level: int, phase: int, sample: int, n: int) -> np.ndarray:
    """Z4 vector of length n: entry i = 1j ** (word(i) >> 62) (complex128)."""
    q = (words(seed, level, phase, sample, n) >> np.uint64(62)).astype(np.int64)
    return np.array([1.0, 1j, -1.0, -1j])[q]


NOISE_RADEMACHER = 0
NOISE_Z4 = 1


def noise(kind: int, seed: int, level: int, phase: int, sample: int, n: int) -> np.ndarray:
    """The isotropic random vector of eq. random_props: Rademacher (kind 0) or Z4 (kind 1), complex128."""
    if kind == NOISE_Z4:
        return z4(seed, level, phase, sample, n)
    return rademacher(seed, level, phase, sample, n).astype(complex)


def noise_block(kind: int, seed: int, level: int, phase: int, sample0: int, n: int, k: int) -> np.ndarray:
    """n x k matrix whose column j is noise(kind, ..., sample0 + j, n)."""
    return np.stack([noise(kind, seed, level, phase, sample0 + j, n) for j in range(k)], axis=1)


def complex_rademacher(seed: int, level: int, phase: int, sample: int, n: int) -> np.ndarray:
    """Complex vector with independent +-1 real and imaginary parts."""
    w = words(seed, level, phase, sample, 2 * n)
    s = np.where((w >> np.uint64(63)) == 0, 1.0, -1.0)
    return s[0::2] + 1j * s[1::2]
