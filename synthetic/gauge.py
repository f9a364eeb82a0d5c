"""Seeded synthetic inputs: quenched compact U(1) gauge fields on an L x L torus.

This module is the only code shared by the CUDA path and the oracle. It holds
no arithmetic of the trace-estimation method: it only draws the gauge field
that the Schwinger operator is built from.

Action: Wilson plaquette action S = -beta * sum_P cos(theta_P) with
theta_P(x) = theta_0(x) + theta_1(x+e0) - theta_0(x+e1) - theta_1(x), the
gauge field periodic in both directions.  (The fermion boundary condition,
antiperiodic in time, belongs to the operator, not to the gauge field.)

Update: single-hit Metropolis, checkerboarded so that links updated together
share no plaquette: x-links on even rows, x-links on odd rows, t-links on even
columns, t-links on odd columns.  One sweep is these four sub-sweeps.  The
random stream is numpy's PCG64 seeded with `seed`; every sub-sweep draws a
fixed number of variates so the field is a pure function of
(L, beta, sweeps, seed, step).

Array layout: theta[t, x, mu] (float64, radians in [-pi, pi)), mu = 0 is the
x direction, mu = 1 the t direction; t is the slow index, x the fast one.
"""
from __future__ import annotations

import numpy as np


def plaquette_angles(theta: np.ndarray) -> np.ndarray:
    """theta_P[t, x] = theta_0(t,x) + theta_1(t,x+1) - theta_0(t+1,x) - theta_1(t,x)."""
    th0 = theta[..., 0]
    th1 = theta[..., 1]
    return th0 + np.roll(th1, -1, axis=1) - np.roll(th0, -1, axis=0) - th1


def mean_plaquette(theta: np.ndarray) -> float:
    return float(np.mean(np.cos(plaquette_angles(theta))))


def _wrap(a: np.ndarray) -> np.ndarray:
    return np.mod(a + np.pi, 2.0 * np.pi) - np.pi


def quenched_u1(L: int, beta: float, sweeps: int, seed: int, step: float = 1.0,
                hot: bool = True, record=None) -> np.ndarray:
    """Return theta[t, x, mu] after `sweeps` Metropolis sweeps.

    `record`, if a list, receives the mean plaquette after every sweep.
    """
    if L < 2 or L % 2:
        raise ValueError("L must be even and >= 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    if hot:
        theta = rng.uniform(-np.pi, np.pi, size=(L, L, 2))
    else:
        theta = np.zeros((L, L, 2))
    rows = np.arange(L)[:, None] % 2  # parity of t
    cols = np.arange(L)[None, :] % 2  # parity of x
    for _ in range(sweeps):
        for mu in (0, 1):
            for parity in (0, 1):
                prop = rng.uniform(-step, step, size=(L, L))
                acc = rng.uniform(0.0, 1.0, size=(L, L))
                P = plaquette_angles(theta)
                if mu == 0:
                    # theta_0(t,x) enters P[t,x] with +1 and P[t-1,x] with -1.
                    Pm = np.roll(P, 1, axis=0)
                    dS = -beta * (np.cos(P + prop) - np.cos(P)
                                  + np.cos(Pm - prop) - np.cos(Pm))
                    mask = (rows == parity) & np.ones((1, L), bool)
                else:
                    # theta_1(t,x) enters P[t,x] with -1 and P[t,x-1] with +1.
                    Pm = np.roll(P, 1, axis=1)
                    dS = -beta * (np.cos(P - prop) - np.cos(P)
                                  + np.cos(Pm + prop) - np.cos(Pm))
                    mask = (cols == parity) & np.ones((L, 1), bool)
                take = mask & (acc < np.exp(-np.minimum(dS, 50.0)))
                theta[..., mu] = np.where(take, _wrap(theta[..., mu] + prop), theta[..., mu])
        if record is not None:
            record.append(mean_plaquette(theta))
    return theta


def links(theta: np.ndarray) -> np.ndarray:
    """Complex links U[t, x, mu] = exp(i theta) (complex128, C-contiguous)."""
    return np.ascontiguousarray(np.exp(1j * theta))


def gauge_transform(theta: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """theta'_mu(x) = omega(x) + theta_mu(x) - omega(x+mu), omega[t, x] in radians."""
    out = np.empty_like(theta)
    out[..., 0] = omega + theta[..., 0] - np.roll(omega, -1, axis=1)
    out[..., 1] = omega + theta[..., 1] - np.roll(omega, -1, axis=0)
    return _wrap(out)


_CACHE: dict = {}


def field(L: int, beta: float, seed: int, sweeps: int | None = None) -> np.ndarray:
    """Memoised theta for the standard recipe (hot start, step 1.0).

    Default sweep count: 500 for L <= 64, 100 above (2D U(1) decorrelates
    within tens of sweeps at beta <= 5; the larger lattices only need enough
    sweeps to leave the hot start behind).
    """
    if sweeps is None:
        sweeps = 500 if L <= 64 else 100
    key = (L, float(beta), int(seed), int(sweeps))
    if key not in _CACHE:
        _CACHE[key] = quenched_u1(L, beta, sweeps, seed)
    return _CACHE[key].copy()
