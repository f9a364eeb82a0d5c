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
    a = rng.rademacher(1, 0, rng.PHASE_STOCH, 0, 256)
    for other in (rng.rademacher(2, 0, rng.PHASE_STOCH, 0, 256),
                  rng.rademacher(1, 1, rng.PHASE_STOCH, 0, 256),
                  rng.rademacher(1, 0, rng.PHASE_SKETCH, 0, 256),
                  rng.rademacher(1, 0, rng.PHASE_STOCH, 1, 256)):
        assert np.mean(a == other) < 0.7
    assert np.array_equal(a, rng.rademacher(1, 0, rng.PHASE_STOCH, 0, 256))
    # prefix property: component i does not depend on the vector length
    assert np.array_equal(a[:100], rng.rademacher(1, 0, rng.PHASE_STOCH, 0, 100))
