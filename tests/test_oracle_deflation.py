"""Pins of the exactly deflated Hutchinson oracle (Section 2): the singular values from gamma5 D are those of
D, the trace split is exact, the direct part by the eigenpair formula equals the k-solve trace, the subspace
iteration (the GPU's method) converges to the exact subspace, and the deflated estimator is unbiased with the
closed-form Rademacher variance, below the undeflated one."""
import math

import numpy as np
import pytest

from oracle import deflation as odf
from oracle import rng
from oracle import schwinger as osch
from synthetic import gauge


def rad_var(M):
    S = M + M.T
    np.fill_diagonal(S, 0)
    return 0.5 * np.sum(np.abs(S) ** 2)


@pytest.fixture(scope="module")
def op():
    U = gauge.links(gauge.field(16, 3.0, 0))
    D = osch.dirac_dense(U, -0.05)
    return D, np.linalg.inv(D)


def test_singular_values_and_trace_split(op):
    D, Dinv = op
    k = 24
    V, mu, tau = odf.singular_deflation_dense(D, k)
    sv = np.sort(np.linalg.svd(D, compute_uv=False))[:k]
    assert np.allclose(np.sort(np.abs(mu)), sv, rtol=1e-10, atol=0)
    assert np.abs(V.conj().T @ V - np.eye(k)).max() < 1e-12
    Pi = V @ V.conj().T
    total = np.trace((np.eye(D.shape[0]) - Pi) @ Dinv) + tau
    assert abs(total - np.trace(Dinv)) < 1e-11 * abs(np.trace(Dinv))
    # direct part: eigenpair formula = tr(V^H D^{-1} V) with k solves
    assert abs(odf.deflation_trace(lambda b: Dinv @ b, V) - tau) < 1e-10 * abs(tau)


def test_subspace_iteration_converges_to_the_exact_subspace(op):
    """The block power method on D^{-1} gamma5 converges to the singular subspace at the rate
    sigma_k / sigma_{k+1}; k = 6 has the widest gap of this operator (0.834), so 160 sweeps reach 1e-9."""
    D, Dinv = op
    k = 6
    V, mu, tau = odf.singular_deflation_dense(D, k)
    W = odf.subspace_iteration(lambda b: Dinv @ b, D.shape[0], k, 160, seed=3)
    assert np.abs(W.conj().T @ W - np.eye(k)).max() < 1e-12
    err = np.abs(W @ W.conj().T - V @ V.conj().T).max()
    assert err < 1e-9, err
    # the k-solve direct part of the converged basis is the eigenpair formula
    assert abs(odf.deflation_trace(lambda b: Dinv @ b, W) - tau) < 1e-8 * abs(tau)
    # fewer sweeps: still an orthonormal basis, farther from the subspace
    W5 = odf.subspace_iteration(lambda b: Dinv @ b, D.shape[0], k, 5, seed=3)
    assert np.abs(W5 @ W5.conj().T - V @ V.conj().T).max() > err


def test_deflated_hutchinson_unbiased_with_smaller_variance(op):
    D, Dinv = op
    n, k = D.shape[0], 32
    V, _, tau = odf.singular_deflation_dense(D, k)
    M = (np.eye(n) - V @ V.conj().T) @ Dinv
    N = 4000
    Z = np.stack([rng.rademacher(11, 0, rng.PHASE_HUTCH, j, n) for j in range(N)], axis=1)
    taus = np.einsum("is,ij,js->s", Z, M, Z)
    v = rad_var(M)
    assert abs(taus.mean() + tau - np.trace(Dinv)) < 4.5 * math.sqrt(v / N)
    assert abs(taus.var(ddof=1) / v - 1) < 0.1
    assert v < 0.5 * rad_var(Dinv)
    # Algorithm 1 on the deflated operator (at least 20 samples, so the variance it stops on is meaningful)
    r = odf.deflated_hutchinson(lambda b: Dinv @ b, V, tau, n, 0.01, seed=7, min_samples=20)
    assert abs(r["tau"] - np.trace(Dinv)) < 5 * math.sqrt(r["V"] / r["s"])
    # the samples are the projected ones: zeta^H D^{-1} zeta - (V^H zeta)^H (V^H D^{-1} zeta) = zeta^T M zeta
    z0 = rng.rademacher(7, 0, rng.PHASE_HUTCH, 0, n)
    assert abs(r["samples"][0] - z0 @ M @ z0) < 1e-10 * abs(z0 @ M @ z0)
