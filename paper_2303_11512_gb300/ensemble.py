"""Ensembles of gauge fields and cycle tuning on top of the C ABI.

    runs = run_ensemble(fields, eps=1e-3)        # fields: list of Field(U_host, L, m0, name)
    best = tune_cycle(ctx, U, L, m0)             # fastest V(nu1, nu2) for this operator
    python -m paper_2303_11512_gb300.ensemble    # the 16-field ensemble (L 128..1024, three masses)

`run_ensemble` admits fields by an estimate of their device memory against the free memory of the GPU
(largest first, so a field that cannot fit is reported instead of failing mid-run), then runs MG-MLMC++
(set-up + Algorithm 2) for every admitted field and reports each field's time to the target accuracy and the
ensemble throughput.  With concurrency > 1 up to that many fields run at the same time, each on its own host
thread, context and CUDA stream, as long as their memory estimates fit together (the library's calls release
the interpreter lock while the GPU works).  Every solve of a field is batched over its right-hand sides and,
within each round of Algorithm 2, over its level differences (see trace_estimate).

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


def group_fields(admitted, free_bytes: int, concurrency: int, **est_kw):
    """Consecutive groups of at most `concurrency` admitted fields whose memory estimates fit free_bytes
    together (the order of `admitted`, largest first, is kept)."""
    groups, cur, used = [], [], 0
    for f in admitted:
        need = memory_estimate(f.L, **est_kw)
        if cur and (len(cur) >= concurrency or used + need > free_bytes):
            groups.append(cur)
            cur, used = [], 0
        cur.append(f)
        used += need
    if cur:
        groups.append(cur)
    return groups


def _run_field(f: Field, eps: float, mg_params: dict, est_params: dict) -> dict:
    """One field on its own stream and context: set-up + Algorithm 2, timed on the host around the stream."""
    stream = torch.cuda.Stream()
    ctx = api.Context(stream)
    try:
        with torch.cuda.stream(stream):
            stream.synchronize()
            t0 = time.perf_counter()
            U = torch.from_numpy(np.ascontiguousarray(f.U, dtype=np.complex128)).cuda()
            h = api.mg_setup(ctx, U, f.L, f.m0, **mg_params)
            stream.synchronize()
            t_setup = time.perf_counter() - t0
            r = api.trace_estimate(ctx, h, eps=eps, **est_params)
            stream.synchronize()
            t = time.perf_counter() - t0
            h.close()
            del U
    finally:
        ctx.close()
    return dict(name=f.name, L=f.L, m0=f.m0, tau=r["tau"], sigma=r["sigma"], N=r["N"], solves=r["solves"],
                setup_s=t_setup, time_s=t, start_s=t0)


def run_ensemble(fields, eps: float = 1e-3, mg_params: dict | None = None, est_params: dict | None = None,
                 free_bytes: int | None = None, concurrency: int = 1) -> dict:
    import concurrent.futures as cf
    mg_params = dict(mg_params or {})
    est_params = dict(est_params or {})
    if free_bytes is None:
        free_bytes = torch.cuda.mem_get_info()[0]
    kw = {k: est_params[k] for k in ("nrhs_max", "d") if k in est_params}
    if "ntv" in mg_params:
        kw["ntv"] = mg_params["ntv"]
    admitted, rejected = admit(fields, free_bytes, **kw)
    groups = group_fields(admitted, free_bytes, concurrency, **kw)
    runs = []
    torch.cuda.synchronize()
    t_all = time.perf_counter()
    for g in groups:
        if len(g) == 1:
            runs.append(_run_field(g[0], eps, mg_params, est_params))
            continue
        with cf.ThreadPoolExecutor(max_workers=len(g)) as ex:
            runs.extend(ex.map(lambda f: _run_field(f, eps, mg_params, est_params), g))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_all
    for r in runs:
        r["start_s"] -= t_all
    return dict(runs=runs, rejected=[(f.name, f.L, memory_estimate(f.L, **kw)) for f in rejected],
                groups=[[f.name for f in g] for g in groups], wall_s=wall,
                fields_per_s=len(runs) / wall if wall > 0 else 0.0,
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


def _field(args):
    from synthetic import gauge
    L, beta, seed = args
    return gauge.links(gauge.field(L, beta, seed))


def ensemble_fields(Ls=(128, 256, 512, 1024), masses=(-0.02, -0.05, -0.08), n=16, beta=3.0, workers=None):
    """The 16-field ensemble: L cycling over Ls, m0 over masses, seeds 0..n-1, quenched U(1) fields at beta
    (generated in a spawn process pool, before any GPU work of the caller's process is required)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    specs = [(Ls[i % len(Ls)], beta, i) for i in range(n)]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        links = list(ex.map(_field, specs))
    return [Field(U, L, masses[i % len(masses)], "f%02d_L%d_m%+.2f" % (i, L, masses[i % len(masses)]))
            for i, ((L, _, _), U) in enumerate(zip(specs, links))]


def run_c4(n: int = 16, eps: float = 1e-3, concurrency: int = 2, workload: dict | None = None) -> dict:
    """The 16-field ensemble (L 128..1024, m0 in {-0.02, -0.05, -0.08}, beta 3) with the benchmark workload's
    hierarchy and estimator parameters, autotuned launch variants and batches of up to 64 rhs."""
    W = dict(workload or {})
    fields = ensemble_fields(n=n)
    mg_params = dict(ntv=W.get("ntv", 8), bootstrap=W.get("bootstrap", 2), bootstrap_its=W.get("bootstrap_its", 6),
                     pre_smooth=W.get("pre_smooth", 2), post_smooth=W.get("post_smooth", 2),
                     tensor_cores=W.get("tensor_cores", 2), autotune=1)
    est_params = dict(d=W.get("d", 32), k=W.get("k", 2), nrhs_max=64, nrhs_first=W.get("nrhs_first", 8), cost_mode=1)
    out = run_ensemble(fields, eps=eps, mg_params=mg_params, est_params=est_params, concurrency=concurrency)
    out["runs"] = [dict(r, tau=[r["tau"].real, r["tau"].imag]) for r in sorted(out["runs"], key=lambda r: r["name"])]
    out["concurrency"] = concurrency
    return out


def main():
    import argparse
    import json
    import os
    import sys
    ap = argparse.ArgumentParser()
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--concurrency", type=int, default=2)
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import __graft_entry__ as g
    g.build()
    import bench
    out = run_c4(n=a.n, eps=a.eps, concurrency=a.concurrency, workload=bench.WORKLOAD)
    for r in out["runs"]:
        print(json.dumps(r), flush=True)
    print(json.dumps({k: v for k, v in out.items() if k != "runs"}), flush=True)
    if a.out:
        json.dump(out, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
