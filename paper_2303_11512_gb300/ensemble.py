"""Ensembles of gauge fields and cycle tuning on top of the C ABI.

    runs = run_ensemble(fields, eps=1e-3)        # fields: list of Field(U_host, L, m0, name)
    best = tune_cycle(ctx, U, L, m0)             # fastest V(nu1, nu2) for this operator

`run_ensemble` admits fields by an estimate of their device memory against the free memory of the GPU
(largest first, so a field that cannot fit is reported instead of failing mid-run), then runs MG-MLMC++
(set-up + Algorithm 2) field after field on one stream and reports each field's time to the target accuracy
and the ensemble throughput.  Every solve of a field is batched over its right-hand sides and, within each
round of Algorithm 2, over its level differences (see trace_estimate).

`tune_cycle` times a short probe (set-up and one batched fine-level solve) for each candidate cycle and returns
the fastest; it is what chose the V(2,2) cycle of the L = 512 benchmark workload.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import api


@dataclasses.dataclass
class Field:
    U: np.ndarray          # complex128 [L, L, 2] host links
    L: int
    m0: float
    name: str = ""


def levels_for(L: int, agg: int = 4) -> list:
    """Lattice sides of the default hierarchy (coarsen while the side exceeds 8 and stays a multiple of 4 agg)."""
    sides = [L]
    while sides[-1] > 8 and sides[-1] % (4 * agg) == 0:
        sides.append(sides[-1] // agg)
    return sides


def memory_estimate(L: int, ntv: int = 8, nrhs_max: int = 256, d: int = 32, m: int = 16, agg: int = 4) -> int:
    """Upper estimate of the device bytes one field's estimate holds: per level the FGMRES bases (FP32,
    2m + 1 vectors), the FP64 right-hand side / solution / residual and sample vectors of a full batch,
    the Hutch++ basis and sketch work, the prolongator, stencils and SAP inverses; plus the coarsest inverse."""
    sides = levels_for(L, agg)
    total = 0
    for i, s in enumerate(sides):
        dof = 2 if i == 0 else 2 * ntv
        n = s * s * dof
        if i < len(sides) - 1:
            total += n * nrhs_max * ((2 * m + 1) * 8 + 8 * 16)    # Krylov bases + FP64 work vectors
            total += n * d * 16 * 4                                # Q, Y and copies
            total += n * ntv * 16 * 2                              # prolongator (FP64 + FP32)
            total += s * s * (5 * dof * dof * 24 + 4 * dof * dof * 24)  # stencil + SAP inverses (FP64 + FP32)
        else:
            total += n * n * 24                                    # dense inverse FP64 + FP32
    return int(total * 1.25)                                      # allocator slack


def admit(fields, free_bytes: int, **est_kw):
    """Split fields into (admitted, rejected) by memory_estimate against free_bytes (each field runs alone,
    so a field is admitted when its own estimate fits)."""
    ok, no = [], []
    for f in sorted(fields, key=lambda f: -f.L):
        (ok if memory_estimate(f.L, **est_kw) <= free_bytes else no).append(f)
    return ok, no


def run_ensemble(fields, eps: float = 1e-3, mg_params: dict | None = None, est_params: dict | None = None,
                 free_bytes: int | None = None) -> dict:
    mg_params = dict(mg_params or {})
    est_params = dict(est_params or {})
    if free_bytes is None:
        free_bytes = torch.cuda.mem_get_info()[0]
    kw = {k: est_params[k] for k in ("nrhs_max", "d") if k in est_params}
    if "ntv" in mg_params:
        kw["ntv"] = mg_params["ntv"]
    admitted, rejected = admit(fields, free_bytes, **kw)
    ctx = api.Context()
    runs = []
    t_all = time.perf_counter()
    try:
        for f in admitted:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            U = torch.from_numpy(np.ascontiguousarray(f.U, dtype=np.complex128)).cuda()
            h = api.mg_setup(ctx, U, f.L, f.m0, **mg_params)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            r = api.trace_estimate(ctx, h, eps=eps, **est_params)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            h.close()
            del U
            runs.append(dict(name=f.name, L=f.L, m0=f.m0, tau=r["tau"], sigma=r["sigma"], N=r["N"],
                             solves=r["solves"], setup_s=t_setup, time_s=t))
    finally:
        ctx.close()
    wall = time.perf_counter() - t_all
    return dict(runs=runs, rejected=[(f.name, f.L, memory_estimate(f.L, **kw)) for f in rejected],
                wall_s=wall, fields_per_s=len(runs) / wall if wall > 0 else 0.0,
                solves_per_s=sum(r["solves"] for r in runs) / wall if wall > 0 else 0.0)


def tune_cycle(ctx: api.Context, U: torch.Tensor, L: int, m0: float, candidates=((1, 1), (1, 2), (2, 2), (3, 3)),
               nrhs: int = 16, seed: int = 7, **mg_params) -> dict:
    """Time set-up + one mixed-precision fine-level solve of nrhs Rademacher vectors per candidate cycle;
    returns {"best": (nu1, nu2), "times": {(nu1, nu2): seconds}, "iters": {...}}."""
    times, iters = {}, {}
    for pre, post in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = api.mg_setup(ctx, U, L, m0, pre_smooth=pre, post_smooth=post, **mg_params)
        b = api.mgmlmc_rademacher(ctx, seed, 0, 0, 0, h.n[0], nrhs)
        x = torch.empty_like(b)
        st = api.fgmres_batched(ctx, h, 0, b, x, prec=api.MIXED)
        torch.cuda.synchronize()
        times[(pre, post)] = time.perf_counter() - t0
        iters[(pre, post)] = st["iters"]
        h.close()
    best = min(times, key=times.get)
    return dict(best=best, times=times, iters=iters)
