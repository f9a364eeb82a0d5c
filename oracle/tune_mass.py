"""Bare-mass tuning for the benchmark workloads (input preparation, oracle side).

The workloads put the smallest |eigenvalue| of D near a target (1e-3): the
spectrum of D(m0) is that of D(0) shifted by m0, so with lambda_c the
eigenvalue of D(0) of smallest real part on the real axis (found by
shift-invert Arnoldi from scipy around a shift left of the spectrum), the mass is
m0 = target - Re(lambda_c).  Writes tests/golden/masses.json.

    python -m oracle.tune_mass 128:3.0 512:5.0
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as spla

from synthetic import gauge

from . import schwinger

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden", "masses.json")


def leftmost_of_links(U: np.ndarray, shift: float = -0.3, k: int = 16) -> complex:
    """The eigenvalue of smallest real part of D(m0 = 0) on the links U: the k eigenvalues nearest to `shift`
    (shift-invert Arnoldi), of which the leftmost."""
    D = schwinger.dirac_sparse(U, 0.0)
    ev = spla.eigs(D, k=k, sigma=shift, return_eigenvectors=False, tol=1e-10)
    return complex(ev[np.argmin(ev.real)])


def leftmost_real(L: int, beta: float, seed: int = 0, shift: float = -0.3, k: int = 16) -> complex:
    return leftmost_of_links(gauge.links(gauge.field(L, beta, seed)), shift, k)


def mass_for_target(lam_c: complex, target: float = 1e-3) -> float:
    """m0 that moves the leftmost eigenvalue lam_c of D(0) to real part `target` (D(m0) = D(0) + m0 I)."""
    return target - lam_c.real


def main(specs, target: float = 1e-3):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for spec in specs:
        L, beta = spec.split(":")
        L, beta = int(L), float(beta)
        t = time.time()
        lam = leftmost_real(L, beta)
        m0 = mass_for_target(lam, target)
        data["L%d_beta%g_seed0" % (L, beta)] = dict(
            L=L, beta=beta, seed=0, sweeps=500 if L <= 64 else 100, lambda_c=[lam.real, lam.imag],
            target=target, m0=round(m0, 6),
            note="m0 = target - Re(lambda_c), lambda_c the leftmost eigenvalue of D(m0=0); "
                 "written by oracle/tune_mass.py")
        print(spec, lam, m0, "%.1fs" % (time.time() - t), flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
