"""Pins of the oracle's counter-based Rademacher generator: the published
SplitMix64 reference outputs, and the isotropy conditions of eq. random_props."""
import json
import os

import numpy as np

from oracle import rng

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    state = np.uint64(0)
    for want in g["outputs"]:
        with np.errstate(over="ignore"):
            state = state + rng.GAMMA
        assert int(rng.mix64(state)) == int(want, 16)


def test_rademacher_isotropy():
    n, s = 4096, 64
    Z = np.stack([rng.rademacher(7, 0, rng.PHASE_STOCH, j, n) for j in range(s)])
    assert set(np.unique(Z)) == {-1.0, 1.0}
    # E|z_i|^2 = 1 exactly; E z_i z_j = 0 within sampling error
    C = Z @ Z.T / n
    off = C[~np.eye(s, dtype=bool)]
    assert abs(Z.mean()) < 5 / np.sqrt(n * s)
    assert np.abs(off).max() < 6 / np.sqrt(n)


def test_streams_are_distinct():
    """Streams that differ in any one counter field (seed, level, phase, sample) are different, pairwise: the
    fields occupy disjoint bits of the counter, so e.g. (level 1, phase 0) and (level 0, phase 1) differ."""
    keys = [(1, 0, rng.PHASE_STOCH, 0), (2, 0, rng.PHASE_STOCH, 0), (1, 1, rng.PHASE_STOCH, 0),
            (1, 0, rng.PHASE_SKETCH, 0), (1, 0, rng.PHASE_STOCH, 1), (1, 1, rng.PHASE_SKETCH, 0),
            (1, 0, rng.PHASE_STOCH, 1 << 40)]
    vecs = [rng.rademacher(*k, 256) for k in keys]
    for i in range(len(keys)):
        for j in range(i):
            assert np.mean(vecs[i] == vecs[j]) < 0.7, (keys[i], keys[j])
    assert np.array_equal(vecs[0], rng.rademacher(1, 0, rng.PHASE_STOCH, 0, 256))
    # prefix property: component i does not depend on the vector length
    assert np.array_equal(vecs[0][:100], rng.rademacher(1, 0, rng.PHASE_STOCH, 0, 100))


def test_z4_values_isotropy_and_second_moment():
    """Z4 entries are the fourth roots of unity, equally likely; E|z|^2 = 1, E z = 0 and E z^2 = 0 (unlike
    real Rademacher vectors, for which z^2 = 1)."""
    n, s = 4096, 64
    Z = np.stack([rng.z4(11, 1, rng.PHASE_STOCH, j, n) for j in range(s)])
    vals, counts = np.unique(np.round(Z, 12), return_counts=True)
    assert set(vals.tolist()) == {1, 1j, -1, -1j}
    assert np.all(np.abs(counts / Z.size - 0.25) < 5 * np.sqrt(0.25 * 0.75 / Z.size))
    assert np.allclose(np.abs(Z), 1.0)
    assert abs(Z.mean()) < 5 / np.sqrt(Z.size)
    assert abs((Z ** 2).mean()) < 5 / np.sqrt(Z.size)
    C = np.conj(Z) @ Z.T / n
    assert np.abs(C[~np.eye(s, dtype=bool)]).max() < 6 / np.sqrt(n)
    # same counter words as the Rademacher stream: the real sign is the top bit
    r = rng.rademacher(11, 1, rng.PHASE_STOCH, 3, n)
    z = rng.z4(11, 1, rng.PHASE_STOCH, 3, n)
    assert np.array_equal(np.where(np.isin(z, [1, 1j]), 1.0, -1.0), r)
    assert np.array_equal(rng.noise(rng.NOISE_Z4, 11, 1, 0, 3, n), z)


def test_complex_rademacher_test_vectors():
    """The set-up's complex test vectors have independent +-1 real and imaginary parts (E|z|^2 = 2, E Re z Im z = 0,
    Re and Im uncorrelated across entries), drawn from consecutive words of the same counter stream."""
    n, s = 4096, 32
    Z = np.stack([rng.complex_rademacher(5, 1, rng.PHASE_TESTVEC, j, n) for j in range(s)])
    assert set(np.unique(Z.real)) == {-1.0, 1.0} and set(np.unique(Z.imag)) == {-1.0, 1.0}
    assert abs((Z.real * Z.imag).mean()) < 5 / np.sqrt(Z.size)
    assert abs(Z.real.mean()) < 5 / np.sqrt(Z.size) and abs(Z.imag.mean()) < 5 / np.sqrt(Z.size)
    w = rng.words(5, 1, rng.PHASE_TESTVEC, 0, 2 * n)
    sign = np.where((w >> np.uint64(63)) == 0, 1.0, -1.0)
    assert np.array_equal(Z[0], sign[0::2] + 1j * sign[1::2])

