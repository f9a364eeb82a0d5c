"""Pins of the oracle's Schwinger operator against facts fixed outside it:
gamma5-hermiticity, the free-field Fourier spectrum and trace (closed form),
gauge covariance, and the fine-level size/nnz printed in Table 1."""
import json
import os

import numpy as np
import pytest

from oracle import schwinger as osch
from oracle.linalg import trace_inverse_dense, trace_inverse_sparse
from synthetic import gauge

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _field(L=8, beta=3.0, seed=0):
    return gauge.links(gauge.quenched_u1(L, beta, 20, seed))


def test_gamma5_hermiticity():
    U = _field(8)
    D = osch.dirac_dense(U, -0.05)
    g5 = osch.gamma5(8).toarray()
    assert np.abs(g5 @ D @ g5 - D.conj().T).max() < 1e-15


def _match(a, b):
    """max over a of the distance to the nearest element of b (multisets of equal size)."""
    b = list(b)
    worst = 0.0
    for z in a:
        j = int(np.argmin([abs(z - w) for w in b]))
        worst = max(worst, abs(z - b[j]))
        b.pop(j)
    return worst


@pytest.mark.parametrize("L,m0", [(4, -0.05), (6, 0.3), (8, -0.4)])
def test_free_field_spectrum_and_trace(L, m0):
    D = osch.dirac_dense(np.ones((L, L, 2), complex), m0)
    ev = np.linalg.eigvals(D)
    assert _match(ev, osch.free_field_eigenvalues(L, m0)) < 1e-12
    tr = trace_inverse_dense(D)
    assert abs(tr - osch.free_field_trace_inverse(L, m0)) < 1e-12 * abs(tr)


def test_free_field_trace_sparse_lu():
    L, m0 = 16, -0.05
    D = osch.dirac_sparse(np.ones((L, L, 2), complex), m0)
    assert abs(trace_inverse_sparse(D, block=128) - osch.free_field_trace_inverse(L, m0)) < 1e-11


def test_gauge_covariance():
    L, m0 = 8, -0.1
    rng = np.random.default_rng(3)
    th = gauge.quenched_u1(L, 3.0, 10, 1)
    om = rng.uniform(-np.pi, np.pi, (L, L))
    D = osch.dirac_dense(gauge.links(th), m0)
    D2 = osch.dirac_dense(gauge.links(gauge.gauge_transform(th, om)), m0)
    W = np.diag(np.repeat(np.exp(1j * om).ravel(), 2))     # psi -> e^{i omega} psi
    assert np.abs(W @ D @ W.conj().T - D2).max() < 1e-14
    assert abs(trace_inverse_dense(D) - trace_inverse_dense(D2)) < 1e-11


def test_dense_matches_sparse_and_hop_structure():
    U = _field(8)
    Ds = osch.dirac_sparse(U, 0.2)
    assert Ds.nnz == 9 * Ds.shape[0]
    D = Ds.toarray()
    assert np.allclose(np.diag(D), 2.2)
    # a single forward x hop from site (t=0,x=0) to (0,1): -1/2 (1 - sigma_1) U_0(0,0)
    blk = D[0:2, 2:4]
    ref = -0.5 * (np.eye(2) - osch.SIGMA[0]) * U[0, 0, 0]
    assert np.abs(blk - ref).max() < 1e-15
    # antiperiodic t boundary: hop from (t=L-1, x=0) forward to (0, 0) carries -1
    L = 8
    r = 2 * ((L - 1) * L)
    blk = D[r:r + 2, 0:2]
    ref = +0.5 * (np.eye(2) - osch.SIGMA[1]) * U[L - 1, 0, 1]
    assert np.abs(blk - ref).max() < 1e-15


def test_table1_fine_level_size_and_nnz():
    g = json.load(open(os.path.join(GOLD, "table1_fine.json")))
    L = g["L"]
    D = osch.dirac_sparse(np.ones((L, L, 2), complex), -0.13)
    assert D.shape[0] == g["n1"]
    nnz = D.nnz
    # the table prints 2.94e5 for 294912 = 9 n: three significant digits, truncated
    scale = 10.0 ** (int(np.floor(np.log10(nnz))) - g["printed_digits"] + 1)
    assert np.floor(nnz / scale) * scale == g["nnz1_printed"]
