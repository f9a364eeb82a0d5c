"""Exactly deflated Hutchinson estimator (Section 2, "Exact Deflation"), oracle form (FP64).

The paper splits tr(D^{-1}) = tr((I - Pi) D^{-1}) + tr(Pi D^{-1}) with a projector Pi on a k-dimensional
subspace of small modes of D, estimates the first term with Algorithm 1 and computes the second directly.
Reading used here (the comparator's deflating subspace): the k right singular vectors of D belonging to its
smallest singular values, with the orthogonal projector Pi = V_k V_k^H (the paper's singular-triplet variant).
For the gamma5-hermitian Wilson operator, Q = gamma5 D is Hermitian and its eigenpairs (mu_i, v_i) give the
singular triplets of D: sigma_i = |mu_i|, right vector v_i, left vector u_i = sign(mu_i) gamma5 v_i, since
D v_i = gamma5 Q v_i = mu_i gamma5 v_i.  The direct part is then
    tr(Pi D^{-1}) = sum_i (1 / sigma_i) u_i^H v_i = sum_i (v_i^H gamma5 v_i) / mu_i,
and the stochastic samples are zeta^H (I - Pi) D^{-1} zeta = zeta^H D^{-1} zeta - (V^H zeta)^H (V^H D^{-1} zeta).

  singular_deflation_dense   the k smallest |mu| eigenpairs of gamma5 D by a dense Hermitian eigensolver
  subspace_iteration         V <- orth(D^{-1} gamma5 V) repeated (block power method on Q^{-1}): converges to
                             the same subspace; the method the CUDA path uses
  deflated_hutchinson        Algorithm 1 on (I - Pi) D^{-1}, plus the direct part
"""
from __future__ import annotations

import numpy as np

from . import rng
from .linalg import qr_positive

PHASE_DEFL = 4  # random stream of the starting block of the subspace iteration


def gamma5_signs(n: int) -> np.ndarray:
    """gamma5 = sigma_3 on every fine site: +1, -1, +1, ... (n = 2 L^2)."""
    return np.tile(np.array([1.0, -1.0]), n // 2)


def singular_deflation_dense(D: np.ndarray, k: int):
    """(V [n x k], mu [k], tau_defl): eigenpairs of the Hermitian gamma5 D with the k smallest |mu|."""
    g5 = gamma5_signs(D.shape[0])
    Q = g5[:, None] * D
    Q = 0.5 * (Q + Q.conj().T)      # Hermitian up to rounding
    mu, W = np.linalg.eigh(Q)
    idx = np.argsort(np.abs(mu))[:k]
    V, mu = W[:, idx], mu[idx]
    tau = complex(np.sum(np.einsum("ik,i,ik->k", np.conj(V), g5, V) / mu))
    return V, mu, tau


def subspace_iteration(solve, n: int, k: int, sweeps: int, seed: int):
    """Block power method on Q^{-1} = D^{-1} gamma5 from k Rademacher vectors (stream PHASE_DEFL, level 0,
    samples 0..k-1): V <- qr(D^{-1} gamma5 V), `sweeps` times (QR with real positive diagonal)."""
    g5 = gamma5_signs(n)
    V = rng.rademacher_block(seed, 0, PHASE_DEFL, 0, n, k)
    for _ in range(sweeps):
        V, _ = qr_positive(solve(g5[:, None] * V))
    return V


def deflation_trace(solve, V) -> complex:
    """tr(V^H D^{-1} V) = tr(Pi D^{-1}) for the orthogonal projector Pi = V V^H (k solves)."""
    return complex(np.sum(np.conj(V) * solve(V)))


def deflated_hutchinson(solve, V, tau_defl, n: int, eps: float, seed: int, smax: int = 100000,
                        min_samples: int = 2, noise: int = rng.NOISE_RADEMACHER):
    """Algorithm 1 on (I - V V^H) D^{-1} with the stop V/s <= (eps |tau_total|)^2 on the total
    tau_total = mean + tau_defl.  Sample s uses stream (seed, level 0, PHASE_HUTCH, s).  Returns
    dict(tau, tau_defl, V, s, samples)."""
    taus = []
    Vv = 0.0
    mean = 0.0
    for s in range(1, smax + 1):
        z = rng.noise(noise, seed, 0, rng.PHASE_HUTCH, s - 1, n)
        y = solve(z)
        c, g = V.conj().T @ z, V.conj().T @ y
        taus.append(complex(np.vdot(z, y) - np.vdot(c, g)))
        mean = sum(taus) / s
        if s >= 2:
            Vv = sum(abs(t - mean) ** 2 for t in taus) / (s - 1)
            if s >= min_samples and Vv / s <= (abs(mean + tau_defl) * eps) ** 2:
                break
    return dict(tau=mean + tau_defl, tau_defl=tau_defl, V=Vv, s=len(taus), samples=np.array(taus))
