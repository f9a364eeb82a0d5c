"""Pins of the bare-mass tuning (input preparation of the benchmark fields) against facts fixed outside it:
the free-field spectrum in closed form, a dense eigensolver on an interacting field, the mass shift of the
spectrum, and gauge invariance."""
import numpy as np

from oracle import schwinger as osch
from oracle import tune_mass as otm
from synthetic import gauge


def test_free_field_leftmost_eigenvalue_closed_form():
    # U = 1: eigenvalues a +- i b with a = m0 + 2 - cos p_x - cos p_t, p_x = 2 pi k / L, p_t = (2k + 1) pi / L
    # (antiperiodic in t): the smallest real part is 1 - cos(pi / L) at m0 = 0, with |Im| = sin(pi / L)
    L = 16
    lam = otm.leftmost_of_links(np.ones((L, L, 2), complex))
    assert abs(lam.real - (1.0 - np.cos(np.pi / L))) < 1e-9
    assert abs(abs(lam.imag) - np.sin(np.pi / L)) < 1e-9


def test_interacting_field_matches_dense_spectrum_and_target():
    L = 8
    U = gauge.links(gauge.quenched_u1(L, 3.0, 30, 2))
    lam = otm.leftmost_of_links(U)
    ev0 = np.linalg.eigvals(osch.dirac_dense(U, 0.0))
    assert abs(lam.real - ev0.real.min()) < 1e-9
    m0 = otm.mass_for_target(lam, 1e-3)
    ev = np.linalg.eigvals(osch.dirac_dense(U, m0))
    assert abs(ev.real.min() - 1e-3) < 1e-9


def test_leftmost_eigenvalue_is_gauge_invariant():
    L = 8
    th = gauge.quenched_u1(L, 3.0, 30, 4)
    om = np.random.default_rng(7).uniform(-np.pi, np.pi, (L, L))
    a = otm.leftmost_of_links(gauge.links(th))
    b = otm.leftmost_of_links(gauge.links(gauge.gauge_transform(th, om)))
    assert abs(a.real - b.real) < 1e-9 and abs(abs(a.imag) - abs(b.imag)) < 1e-9
