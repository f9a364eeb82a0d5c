"""Parameter scans of MG-MLMC++ (the paper's Section 4 study, Fig. 2): the sketch size d_l and the number k of
block power sweeps of the Hutch++ deflation, and the uniform against the optimal target accuracies of the
level differences, on one synthetic gauge field.  d = 0 is plain MG-MLMC.

    python -m paper_2303_11512_gb300.scan                 # L = 512 workload of the benchmark
    python -m paper_2303_11512_gb300.scan --L 128 --eps 2e-3
    python -m paper_2303_11512_gb300.scan --setup         # test vectors per chirality x sample form

The set-up scan (the paper's Table 1 hierarchies have 2 and then 4 test vectors per chirality; the benchmark 8)
builds the hierarchy with ntv in {2, 4, 8} and runs plain MG-MLMC and MG-MLMC++ in the accumulated and the
reduced form of the level differences, reporting the set-up time, the per-level sample variances V_l, N_l and the
time to the target accuracy.  With ntv != 8 the coarse levels have 4 or 8 dof and run on the CUDA cores.

For every configuration the estimate is run to the target accuracy on the same hierarchy and reported with
its wall time (CUDA events on the context stream), its samples N_l, and the paper's cost model (arithmetic
operations of the operator applications): the library's counted flops of all solves (inner iterations + 1 per
solve times 8 flops per complex non-zero of the level operator) plus the projections (2 x 8 n_l d_l per
stochastic sample, c = Q^H zeta and g = Q^H y) and the CholeskyQR2 passes of the sketch (2 passes of
8 n_l d_l^2 for the Gram matrix and 4 n_l d_l^2 for Y R^{-1}, k times per level).  Prints one JSON line per
configuration and a summary table.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def sketch_flops(n, d, k):
    return sum(k * 2 * (8.0 * nl * dl * dl + 4.0 * nl * dl * dl) for nl, dl in zip(n, d))


def projection_flops(n, d, N):
    return sum(2 * 8.0 * nl * dl * Nl for nl, dl, Nl in zip(n, d, N))


def run(L=512, beta=5.0, eps=1e-3, ds=(0, 8, 16, 32, 48, 64), ks=(1, 2, 3), uniform_for=((0, 1), (32, 2)),
        seed=0, out=None):
    import torch

    import bench
    from . import api
    from synthetic import gauge
    W = bench.WORKLOAD
    m0 = bench.mass_for(L, beta, seed)
    U = torch.from_numpy(gauge.links(gauge.field(L, beta, seed))).cuda()
    ctx = api.Context()
    h = api.mg_setup(ctx, U, L, m0, ntv=W["ntv"], bootstrap=W["bootstrap"], bootstrap_its=W["bootstrap_its"],
                     pre_smooth=W["pre_smooth"], post_smooth=W["post_smooth"], tensor_cores=W["tensor_cores"])
    nd = h.levels - 1
    confs = [(0, 1, api.OPTIMAL)] + [(d, k, api.OPTIMAL) for d in ds if d > 0 for k in ks]
    confs += [(d, k, api.UNIFORM) for d, k in uniform_for]
    stream = ctx.stream
    rows = []
    # one untimed estimate first (workspaces, graphs)
    api.trace_estimate(ctx, h, eps=eps, d=32, k=2, nrhs_max=W["nrhs_max"], nrhs_first=W["nrhs_first"], cost_mode=1)
    for d, k, pol in confs:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = api.trace_estimate(ctx, h, eps=eps, d=d, k=k, nrhs_max=W["nrhs_max"], nrhs_first=W["nrhs_first"],
                               cost_mode=1, policy=pol, seed=seed)
        b.record(stream)
        torch.cuda.synchronize()
        dl = [d] * nd
        nl = h.n[:nd]
        flops = r["flops"] + projection_flops(nl, dl, r["N"]) + sketch_flops(nl, dl, k if d else 0)
        row = dict(L=L, d=d, k=k if d else 0, policy="uniform" if pol == api.UNIFORM else "optimal",
                   seconds=a.elapsed_time(b) / 1e3, N=r["N"], solves=r["solves"], mflops=flops / 1e6,
                   tau=r["tau"].real, rel_sigma=r["sigma"] / abs(r["tau"]))
        rows.append(row)
        print(json.dumps(row), flush=True)
    h.close()
    ctx.close()
    if out:
        json.dump(rows, open(out, "w"), indent=1)
    print("%6s %3s %2s %8s %9s %12s %22s" % ("L", "d", "k", "policy", "time [s]", "MFlop", "N_l"))
    for r in rows:
        print("%6d %3d %2d %8s %9.3f %12.0f %22s" % (r["L"], r["d"], r["k"], r["policy"], r["seconds"], r["mflops"],
                                                   r["N"]))
    return rows


def run_setup(L=512, beta=5.0, eps=1e-3, ntvs=(2, 4, 8), forms=("accumulated", "reduced"), dks=((0, 1), (32, 2)),
              seed=0, out=None):
    import torch

    import bench
    from . import api
    from synthetic import gauge
    W = bench.WORKLOAD
    m0 = bench.mass_for(L, beta, seed)
    U = torch.from_numpy(gauge.links(gauge.field(L, beta, seed))).cuda()
    ctx = api.Context()
    stream = ctx.stream
    rows = []
    for ntv in ntvs:
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h = api.mg_setup(ctx, U, L, m0, ntv=ntv, bootstrap=W["bootstrap"], bootstrap_its=W["bootstrap_its"],
                         pre_smooth=W["pre_smooth"], post_smooth=W["post_smooth"], tensor_cores=W["tensor_cores"])
        b.record(stream)
        torch.cuda.synchronize()
        t_setup = a.elapsed_time(b) / 1e3
        api.trace_estimate(ctx, h, eps=eps, d=0, k=1, nrhs_max=W["nrhs_max"], nrhs_first=W["nrhs_first"],
                           cost_mode=1)  # untimed: workspaces
        for form in forms:
            for d, k in dks:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = api.trace_estimate(ctx, h, eps=eps, d=d, k=k, nrhs_max=W["nrhs_max"],
                                       nrhs_first=W["nrhs_first"], cost_mode=1, seed=seed,
                                       form=api.ACCUMULATED if form == "accumulated" else api.REDUCED)
                b.record(stream)
                torch.cuda.synchronize()
                row = dict(L=L, ntv=ntv, coarse_dof=2 * ntv, form=form, d=d, k=k, setup_s=t_setup,
                           seconds=a.elapsed_time(b) / 1e3, N=r["N"], V=r["V"], solves=r["solves"],
                           inner_iters=r["inner_iters"], tau=r["tau"].real, rel_sigma=r["sigma"] / abs(r["tau"]))
                rows.append(row)
                print(json.dumps(row), flush=True)
        h.close()
    ctx.close()
    if out:
        json.dump(rows, open(out, "w"), indent=1)
    print("%4s %12s %3s %2s %8s %9s %22s %s" % ("ntv", "form", "d", "k", "setup", "time [s]", "N_l", "V_l"))
    for r in rows:
        print("%4d %12s %3d %2d %8.3f %9.3f %22s %s" % (r["ntv"], r["form"], r["d"], r["k"], r["setup_s"],
                                                         r["seconds"], r["N"], ["%.3g" % v for v in r["V"]]))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--setup", action="store_true", help="scan test vectors per chirality and the sample form")
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--beta", type=float, default=5.0)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--out", default=None, help="write the rows as JSON")
    a = ap.parse_args()
    import __graft_entry__ as g
    g.build()
    if a.setup:
        run_setup(L=a.L, beta=a.beta, eps=a.eps, out=a.out)
    else:
        run(L=a.L, beta=a.beta, eps=a.eps, out=a.out)


if __name__ == "__main__":
    main()
