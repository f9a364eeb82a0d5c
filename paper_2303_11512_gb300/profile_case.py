"""Small, self-contained cases for kernel profiling (ncu captures).

    python -m paper_2303_11512_gb300.profile_case --case solve --level 1 --nrhs 64
    python -m paper_2303_11512_gb300.profile_case --case stencil --nrhs 256

`solve` builds the benchmark hierarchy (L = 512, beta = 5) and runs one
mixed-precision FGMRES solve on the chosen level (so every kernel of the V-cycle
and the Krylov loop runs a few hundred times on level-sized data larger than L2);
`stencil` applies the FP32 fine operator to nrhs vectors ten times.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="solve", choices=["solve", "stencil"])
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--level", type=int, default=1)
    ap.add_argument("--nrhs", type=int, default=64)
    a = ap.parse_args()
    import torch

    import bench
    from paper_2303_11512_gb300 import api, build
    from synthetic import gauge

    build.build()
    W = bench.WORKLOAD
    beta = W["beta"]
    m0 = bench.mass_for(a.L, beta, W["seed"])
    U = torch.from_numpy(gauge.links(gauge.field(a.L, beta, W["seed"]))).cuda()
    ctx = api.Context()
    if a.case == "stencil":
        n = 2 * a.L * a.L
        x = torch.randn((a.nrhs, n), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(10):
            api.schwinger_apply(ctx, U, a.L, m0, x, y, api.FP32)
    else:
        h = api.mg_setup(ctx, U, a.L, m0, ntv=W["ntv"], bootstrap=W["bootstrap"], bootstrap_its=W["bootstrap_its"],
                         pre_smooth=W["pre_smooth"], post_smooth=W["post_smooth"])
        b = api.mgmlmc_rademacher(ctx, 1, 0, 0, 0, h.n[a.level], a.nrhs)
        x = torch.empty_like(b)
        st = api.fgmres_batched(ctx, h, a.level, b, x, prec=api.MIXED, tol=1e-10)
        print("iters", st["iters"], "relres", st["max_relres"])
        h.close()
    torch.cuda.synchronize()
    ctx.close()


if __name__ == "__main__":
    main()
