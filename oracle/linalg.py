"""Dense/sparse linear algebra helpers of the oracle (FP64).

  qr_positive      QR factorisation with a real positive diagonal of R: the
                   QR of Y_l in Algorithm 2 (Section 3.2).  With that
                   normalisation Q is unique for full-rank Y.
  cholesky_qr2     CholeskyQR2 (Yamamoto et al. 2015; Fukaya et al. 2014):
                   G = Y^H Y, R = chol(G), Q = Y R^{-1}, done twice.  Same Q
                   as qr_positive in exact arithmetic.
  trace_inverse_*  exact tr(D^{-1}) = sum_i (D^{-1})_ii (Section 1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def qr_positive(Y: np.ndarray):
    Q, R = np.linalg.qr(Y, mode="reduced")
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    Q = Q * ph[None, :]
    R = np.conj(ph)[:, None] * R
    return Q, R


def cholesky_qr2(Y: np.ndarray):
    def chol_qr(A):
        G = A.conj().T @ A
        R = sla.cholesky(G, lower=False)          # G = R^H R
        Q = sla.solve_triangular(R, A.T, trans="T", lower=False).T  # A R^{-1}
        return Q, R
    Q1, R1 = chol_qr(Y)
    Q2, R2 = chol_qr(Q1)
    return Q2, R2 @ R1


def trace_inverse_dense(D: np.ndarray) -> complex:
    return complex(np.trace(np.linalg.inv(D)))


def trace_inverse_sparse(D: sp.spmatrix, block: int = 512) -> complex:
    """sum_i e_i^T D^{-1} e_i by a sparse LU and blocks of unit vectors."""
    n = D.shape[0]
    lu = spla.splu(sp.csc_matrix(D), permc_spec="MMD_AT_PLUS_A")
    tr = 0.0 + 0.0j
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        E = np.zeros((n, i1 - i0), dtype=complex)
        E[np.arange(i0, i1), np.arange(i1 - i0)] = 1.0
        X = lu.solve(E)
        tr += np.sum(X[np.arange(i0, i1), np.arange(i1 - i0)])
    return complex(tr)


class DirectSolver:
    """x = D^{-1} b by sparse LU (scipy SuperLU), columns of b solved together.  The level operators are
    nearest-neighbour stencils, structurally symmetric, so the fill-reducing column order is minimum degree
    on A^T + A (a quarter of the fill of the column-only order on the 16-dof coarse levels)."""

    def __init__(self, D: sp.spmatrix):
        self.n = D.shape[0]
        if self.n <= 2048:
            self._dense = np.linalg.inv(D.toarray())
            self._lu = None
        else:
            self._dense = None
            self._lu = spla.splu(sp.csc_matrix(D), permc_spec="MMD_AT_PLUS_A")

    def solve(self, b: np.ndarray) -> np.ndarray:
        if self._dense is not None:
            return self._dense @ b
        return self._lu.solve(np.asarray(b, dtype=complex))
