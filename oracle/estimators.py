"""Stochastic trace estimators of the paper, oracle form (FP64, direct solves).

  hutchinson        Algorithm 1 (plain Hutchinson with the relative-accuracy
                    stop V/s <= (tau eps)^2).
  LevelDifference   the level differences of the MG-MLMC decomposition:
                    accumulated form  A_l = Phat_l D_l^{-1} Rhat_l
                                             - Phat_{l+1} D_{l+1}^{-1} Rhat_{l+1}
                    (eq. mlmc_decomp_matrix / mlmc_decomp_trace), fine-size
                    vectors; reduced form A_l = D_l^{-1} - P_l D_{l+1}^{-1} P_l^H
                    (eq. mlmc_dec_trace_reduced), level-size vectors.
  mgmlmc_pp         Algorithm 2 (MG-MLMC++, optimal or uniform accuracies).
                    With d_l = 0 on every level it is plain MG-MLMC.

Readings of the paper used here (each is also what the CUDA path does):
  * tau in the stop test of Algorithm 2 is the running estimate
    tau + tau_L = sum_{l<L} (tau_l + tau_l^lr) + tau_L, and its modulus is
    used (samples are complex; the exact trace is real).
  * the sums over j in eq. accuracy_opt and in the rho_l update run over the
    L-1 stochastic level differences; the uniform policy sets
    rho_l^2 = (eps |tau|)^2 / (L-1).
  * tau_L = tr(D_L^{-1}) exactly (Phat_L has orthonormal columns).
  * a level is tested for the stop only once it holds >= min_samples
    (default 2) samples, since V needs s >= 2; rho_l is only formed when all
    levels have a variance.
  * the sample cost C_{s,l} is a per-level constant supplied by the caller
    (the nnz-proportional flop model of Section 4 with fixed solve counts).
  * the QR of Y_l is the one with a real positive diagonal of R.
  * sample s (0-based) of level l uses the Rademacher stream
    (seed, level l, phase STOCH, sample s); sketch column j uses
    (seed, l, SKETCH, j).  noise = rng.NOISE_Z4 draws Z4 vectors from the
    same streams instead (Section 2 names both distributions).
  * gamma5-weighted traces tr(gamma5 D^{-1}) (Section 1: traces "after
    multiplication with certain gamma-matrices"): every level difference is
    replaced by gamma5 A_l and the coarsest term by tr(gamma5 Phat_L D_L^{-1}
    Rhat_L).  gamma5 = sigma_3 on the fine level; on coarse levels it is the
    chirality sign of the dof.  The aggregation keeps chiralities apart, so
    gamma5 Phat_l = Phat_l gamma5_l and the level-size forms stay valid.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import rng
from .linalg import DirectSolver, qr_positive


def hutchinson(solve, n: int, eps: float, seed: int, smax: int = 1000, min_samples: int = 2,
               noise: int = rng.NOISE_RADEMACHER, weight=None):
    """Algorithm 1.  solve(b) returns D^{-1} b; weight (optional, n-vector) estimates tr(diag(weight) D^{-1})
    (e.g. the gamma5 signs).  Returns (tau, V, s, samples)."""
    taus = []
    tau = 0.0
    V = float("nan")
    for s in range(1, smax + 1):
        z = rng.noise(noise, seed, 0, rng.PHASE_HUTCH, s - 1, n)
        x = solve(z)
        if weight is not None:
            x = weight * x
        taus.append(np.vdot(z, x))                 # zeta^H (W) D^{-1} zeta
        tau = sum(taus) / s
        if s >= 2:
            V = sum(abs(ti - tau) ** 2 for ti in taus) / (s - 1)
            if s >= min_samples and V / s <= (abs(tau) * eps) ** 2:
                break
    return tau, V, len(taus), np.array(taus)


class LevelDifference:
    """x -> A_l x for a multigrid hierarchy, with direct solves on every level."""

    def __init__(self, H, form: str = "accumulated", gamma5: bool = False):
        assert form in ("accumulated", "reduced")
        self.H, self.form, self.gamma5 = H, form, gamma5
        self.solvers = [DirectSolver(Dl) for Dl in H.D]
        self.Phat = [H.Phat(l) for l in range(H.levels)]

    def vec_size(self, l: int) -> int:
        return self.H.n[0] if self.form == "accumulated" else self.H.n[l]

    def weight(self, l: int):
        """gamma5 of the space the level-l vectors live in (None without gamma5 weighting)."""
        if not self.gamma5:
            return None
        return self.H.gamma5(0 if self.form == "accumulated" else l)

    def apply(self, l: int, Z: np.ndarray) -> np.ndarray:
        """A_l Z, or gamma5 A_l Z for gamma5-weighted traces."""
        H = self.H
        if self.form == "accumulated":
            Pl, Pn = self.Phat[l], self.Phat[l + 1]
            a = Pl @ self.solvers[l].solve(Pl.conj().T @ Z)
            b = Pn @ self.solvers[l + 1].solve(Pn.conj().T @ Z)
            Y = a - b
        else:
            P = H.P[l]
            Y = self.solvers[l].solve(Z) - P @ self.solvers[l + 1].solve(P.conj().T @ Z)
        W = self.weight(l)
        return Y if W is None else W @ Y

    def coarsest_trace(self) -> complex:
        """tau_L = tr(Phat_L D_L^{-1} Rhat_L) (or with gamma5 in front), by the cyclic property
        tr(Rhat_L W Phat_L D_L^{-1}) with Rhat = Phat^H; in the reduced form Phat_L is P_{L-1} applied to
        level L-1 (eq. mlmc_dec_trace_reduced)."""
        H = self.H
        X = self.solvers[-1].solve(np.eye(H.n[-1]))
        if self.form == "accumulated":
            Ph = self.Phat[-1]
            W = H.gamma5(0) if self.gamma5 else sp.identity(H.n[0])
        else:
            Ph = H.P[-1]
            W = H.gamma5(H.levels - 2) if self.gamma5 else sp.identity(H.n[-2])
        M = (Ph.conj().T @ W @ Ph).toarray()
        return complex(np.trace(M @ X))

    def exact_traces(self):
        """[tr(A_l) for l < L-1] and tau_L by dense inverses (small levels only)."""
        H = self.H
        if not self.gamma5:
            tri = [complex(np.trace(np.linalg.inv(Dl.toarray()))) for Dl in H.D]
            return [tri[l] - tri[l + 1] for l in range(H.levels - 1)], tri[-1]
        out = []
        for l in range(H.levels - 1):
            n = self.vec_size(l)
            out.append(complex(np.trace(self.apply(l, np.eye(n, dtype=complex)))))
        return out, self.coarsest_trace()


def update_active(active, V, N, cost, eps, tau_total, policy="optimal", min_samples=2):
    """The target-accuracy update and stop test of Algorithm 2 for one step s.

    rho_l = (sqrt(C_l V_l) / sum_j sqrt(C_j V_j))^(1/2) * eps |tau| (optimal,
    eq. optimal_variance) or rho_l^2 = (eps |tau|)^2 / (L-1) (uniform);
    level l becomes inactive when V_l / N_l <= rho_l^2.  Nothing changes
    until every level has a variance (N_j >= 2).
    """
    nd = len(active)
    out = list(active)
    if any(n < 2 for n in N):
        return out
    denom = sum(math.sqrt(cost[j] * V[j]) for j in range(nd))
    for l in range(nd):
        if not active[l] or N[l] < min_samples:
            continue
        if policy == "uniform":
            rho2 = (eps * abs(tau_total)) ** 2 / nd
        else:
            w = math.sqrt(cost[l] * V[l]) / denom if denom > 0 else 1.0 / nd
            rho2 = w * (eps * abs(tau_total)) ** 2
        if V[l] / N[l] <= rho2:
            out[l] = False
    return out


def mgmlmc_pp(ld: LevelDifference, eps: float, d, k: int, seed: int, policy: str = "optimal",
              cost=None, min_samples: int = 2, max_samples: int = 100000, noise: int = rng.NOISE_RADEMACHER,
              Q_given=None):
    """Algorithm 2.  d: deflation vectors per level difference (list or int).  The weighting (gamma5) is that
    of ld.  Q_given (optional list of n x d_l bases) replaces the sketch's Q in the projection of the
    stochastic samples (to replay another implementation's samples on the same Q)."""
    H = ld.H
    nL = H.levels
    nd = nL - 1
    d = [d] * nd if np.isscalar(d) else list(d)
    cost = [1.0] * nd if cost is None else list(cost)
    # deflation part: k sweeps of the block power method, then the low-rank trace
    Q = [None] * nd
    tau_lr = [0.0j] * nd
    for l in range(nd):
        if d[l] == 0:
            continue
        n = ld.vec_size(l)
        S = rng.noise_block(noise, seed, l, rng.PHASE_SKETCH, 0, n, d[l])
        for _ in range(k):
            Y = ld.apply(l, S)
            Ql, _ = qr_positive(Y)
            S = Ql
        Q[l] = S
        tau_lr[l] = complex(np.sum(np.conj(S) * ld.apply(l, S)))
    if Q_given is not None:
        Q = list(Q_given)
    # coarsest level directly
    tau_L = ld.coarsest_trace()
    # stochastic part
    active = [True] * nd
    samples = [[] for _ in range(nd)]
    mean = [0.0j] * nd
    V = [float("nan")] * nd
    tau = 0.0j
    s = 0
    while any(active) and s < max_samples:
        s += 1
        for l in range(nd):
            if not active[l]:
                continue
            zeta = rng.noise(noise, seed, l, rng.PHASE_STOCH, len(samples[l]), ld.vec_size(l))
            y = ld.apply(l, zeta)
            z = zeta if Q[l] is None else zeta - Q[l] @ (Q[l].conj().T @ zeta)
            samples[l].append(complex(np.vdot(z, y)))
            N = len(samples[l])
            mean[l] = sum(samples[l]) / N
            V[l] = (sum(abs(t - mean[l]) ** 2 for t in samples[l]) / (N - 1)) if N >= 2 else float("nan")
        tau = sum(mean[l] + tau_lr[l] for l in range(nd))
        active = update_active(active, V, [len(x) for x in samples], cost, eps,
                               tau + tau_L, policy, min_samples)
    N = [len(x) for x in samples]
    sigma = math.sqrt(sum(V[l] / N[l] for l in range(nd) if N[l] >= 2))
    return dict(tau=tau + tau_L, tau_L=tau_L, tau_lr=tau_lr, mean=mean, V=V, N=N,
                samples=[np.array(x) for x in samples], sigma=sigma, Q=Q, steps=s)
