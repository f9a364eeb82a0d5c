"""The synthetic gauge generator against the exact 2D U(1) result:
<cos theta_P> = I_1(beta) / I_0(beta) for the Wilson plaquette action."""
import numpy as np
import pytest
from scipy.special import iv

from synthetic import gauge


@pytest.mark.parametrize("beta", [3.0, 5.0])
def test_mean_plaquette_exact(beta):
    rec = []
    gauge.quenched_u1(32, beta, 160, 11, record=rec)
    assert abs(np.mean(rec[60:]) - iv(1, beta) / iv(0, beta)) < 0.006


def test_reproducible_and_gauge_invariant_plaquette():
    a = gauge.quenched_u1(16, 3.0, 5, 4)
    b = gauge.quenched_u1(16, 3.0, 5, 4)
    assert np.array_equal(a, b)
    om = np.random.default_rng(0).uniform(-np.pi, np.pi, (16, 16))
    a2 = gauge.gauge_transform(a, om)
    assert abs(gauge.mean_plaquette(a) - gauge.mean_plaquette(a2)) < 1e-12
