"""2D Schwinger Wilson-Dirac operator, oracle form (numpy/scipy, FP64).

The paper uses the Schwinger discretisation of the 2-dimensional Dirac
operator (Section 4) without printing it; the formula taken here is the
standard Wilson form with two spin components and U(1) links:

  (D psi)(x) = (m0 + 2) psi(x)
      - 1/2 sum_mu [ (1 - sigma_mu) U_mu(x) psi(x + mu)
                   + (1 + sigma_mu) conj(U_mu(x - mu)) psi(x - mu) ]

with sigma_0 = sigma_1 (Pauli x) for the x direction, sigma_1 = sigma_2
(Pauli y) for the t direction, periodic in x and antiperiodic in t (a factor
-1 on every hop that crosses the t boundary).  gamma5 = sigma_3, so the
chirality of a fine degree of freedom is its spin index.  Every row has
1 + 4 * 2 = 9 non-zeros, which is the nnz(D_1) = 9 n of Table 1.

Index convention: site s = t * L + x, dof i = 2 s + spin.
Links U[t, x, mu] complex128.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=complex),      # sigma_1, x direction
    np.array([[0, -1j], [1j, 0]], dtype=complex),   # sigma_2, t direction
)
SIGMA3 = np.array([[1, 0], [0, -1]], dtype=complex)


def dirac_sparse(U: np.ndarray, m0: float) -> sp.csr_matrix:
    """Sparse D (n x n, n = 2 L^2) from links U[t, x, mu]."""
    L = U.shape[0]
    assert U.shape == (L, L, 2)
    V = L * L
    t, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    s = (t * L + x).ravel()
    rows, cols, vals = [], [], []
    eye = np.eye(2, dtype=complex)
    # diagonal
    for a in range(2):
        rows.append(2 * s + a)
        cols.append(2 * s + a)
        vals.append(np.full(V, m0 + 2.0, dtype=complex))
    for mu in range(2):
        if mu == 0:
            tf, xf = t, (x + 1) % L
            tb, xb = t, (x - 1) % L
            eta_f = np.ones_like(t, dtype=float)
            eta_b = np.ones_like(t, dtype=float)
        else:
            tf, xf = (t + 1) % L, x
            tb, xb = (t - 1) % L, x
            eta_f = np.where(t == L - 1, -1.0, 1.0)
            eta_b = np.where(t == 0, -1.0, 1.0)
        sf = (tf * L + xf).ravel()
        sb = (tb * L + xb).ravel()
        Uf = (U[t, x, mu] * eta_f).ravel()                 # U_mu(x)
        Ub = (np.conj(U[tb, xb, mu]) * eta_b).ravel()      # U_mu(x - mu)^*
        Pm = eye - SIGMA[mu]
        Pp = eye + SIGMA[mu]
        for a in range(2):
            for b in range(2):
                if Pm[a, b] != 0:
                    rows.append(2 * s + a)
                    cols.append(2 * sf + b)
                    vals.append(-0.5 * Pm[a, b] * Uf)
                if Pp[a, b] != 0:
                    rows.append(2 * s + a)
                    cols.append(2 * sb + b)
                    vals.append(-0.5 * Pp[a, b] * Ub)
    n = 2 * V
    D = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    D.sum_duplicates()
    return D


def dirac_dense(U: np.ndarray, m0: float) -> np.ndarray:
    return dirac_sparse(U, m0).toarray()


def gamma5(L: int) -> sp.dia_matrix:
    """gamma5 = sigma_3 on every site: diag(+1, -1, +1, -1, ...)."""
    d = np.tile(np.array([1.0, -1.0]), L * L)
    return sp.diags(d)


def free_field_momenta(L: int):
    """p_x = 2 pi k / L (periodic), p_t = (2k + 1) pi / L (antiperiodic)."""
    k = np.arange(L)
    px = 2 * np.pi * k / L
    pt = (2 * k + 1) * np.pi / L
    return np.meshgrid(pt, px, indexing="ij")


def free_field_eigenvalues(L: int, m0: float) -> np.ndarray:
    """Spectrum of D at U = 1: a +- i sqrt(sin^2 p_x + sin^2 p_t),
    a = m0 + 2 - cos p_x - cos p_t (Fourier transform of the formula above)."""
    PT, PX = free_field_momenta(L)
    a = m0 + 2.0 - np.cos(PX) - np.cos(PT)
    b = np.sqrt(np.sin(PX) ** 2 + np.sin(PT) ** 2)
    return np.concatenate([(a + 1j * b).ravel(), (a - 1j * b).ravel()])


def free_field_trace_inverse(L: int, m0: float) -> float:
    """tr D^{-1} at U = 1: sum over momenta of 2 a / (a^2 + b^2)."""
    PT, PX = free_field_momenta(L)
    a = m0 + 2.0 - np.cos(PX) - np.cos(PT)
    b2 = np.sin(PX) ** 2 + np.sin(PT) ** 2
    return float(np.sum(2.0 * a / (a * a + b2)))
