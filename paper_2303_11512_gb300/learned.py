"""Training and evaluation of the learned gauge-covariant correction (C ABI nn_*).

    python -m paper_2303_11512_gb300.learned --L-train 128 --L-eval 256 --pairs 4096 --steps 1500

Pairs (r, e) come from the library's own V-cycle and solves on the training field: r = zeta - D V(zeta),
e = D^{-1} zeta - V(zeta), both divided by ||r|| (the net is applied to unit-norm residuals).  The net is
trained with the library's forward/backward/Adam kernels, then its weights are loaded into a net built on
the evaluation field (the layers are local and gauge covariant, so one set of weights serves any lattice) and
FGMRES to the FP64 true residual 1e-10 is timed with the V-cycle alone (precond 1) and with V-cycle + net
(precond 2).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def harvest(api, ctx, h, n_pairs: int, batch: int, seed: int):
    """n_pairs (r, e) pairs at the fine level of hierarchy h, FP32 complex [n_pairs, n]."""
    import torch
    n = h.n[0]
    R = torch.empty((n_pairs, n), dtype=torch.complex64, device="cuda")
    E = torch.empty_like(R)
    for s0 in range(0, n_pairs, batch):
        nb = min(batch, n_pairs - s0)
        z = api.mgmlmc_rademacher(ctx, seed, 0, 0, s0, n, nb).to(torch.complex64)
        v = torch.empty_like(z)
        h.vcycle(0, z, v, api.FP32)
        dv = torch.empty_like(z)
        h.apply(0, v, dv, api.FP32)
        r1 = z - dv
        x = torch.empty_like(z)
        api.fgmres_batched(ctx, h, 0, z, x, prec=api.FP32, tol=1e-6)
        s = torch.linalg.vector_norm(r1, dim=1, keepdim=True)
        R[s0:s0 + nb] = r1 / s
        E[s0:s0 + nb] = (x - v) / s
    return R, E


def timed_solves(api, ctx, h, precond: int, nrhs: int, seed: int, reps: int = 2):
    import torch
    b = api.mgmlmc_rademacher(ctx, seed, 0, 0, 0, h.n[0], nrhs)
    x = torch.empty_like(b)
    st = api.fgmres_batched(ctx, h, 0, b, x, prec=api.MIXED, tol=1e-10, precond=precond)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        st = api.fgmres_batched(ctx, h, 0, b, x, prec=api.MIXED, tol=1e-10, precond=precond)
    torch.cuda.synchronize()
    return dict(iters=int(st["iters"]), converged=bool(st["converged"]), relres=float(st["max_relres"]),
                s_per_solve=(time.perf_counter() - t0) / reps), x


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L-train", type=int, default=128)
    ap.add_argument("--L-eval", type=int, default=256)
    ap.add_argument("--beta", type=float, default=3.0)
    ap.add_argument("--m0", type=float, default=-0.08)
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--channels", type=int, default=16)
    ap.add_argument("--nrhs", type=int, default=16)
    a = ap.parse_args()
    import torch

    from paper_2303_11512_gb300 import api, build
    from synthetic import gauge
    build.build()
    ctx = api.Context()
    out = dict(L_train=a.L_train, L_eval=a.L_eval, beta=a.beta, m0=a.m0, layers=a.layers, channels=a.channels)
    # training field and pairs
    Ut = torch.from_numpy(gauge.links(gauge.field(a.L_train, a.beta, 1))).cuda()
    ht = api.mg_setup(ctx, Ut, a.L_train, a.m0)
    t0 = time.perf_counter()
    R, E = harvest(api, ctx, ht, a.pairs, 64, seed=3)
    torch.cuda.synchronize()
    out["harvest_s"] = time.perf_counter() - t0
    Rv, Ev = harvest(api, ctx, ht, 64, 64, seed=4)   # held out
    net = api.Net(ctx, Ut, a.L_train, a.layers, a.channels, seed=2)
    l0, _ = net.loss_grad(Rv, Ev)
    t0 = time.perf_counter()
    g = torch.Generator(device="cpu").manual_seed(0)
    for it in range(a.steps):
        idx = torch.randint(0, a.pairs, (a.batch,), generator=g).cuda()
        net.train_step(R[idx].contiguous(), E[idx].contiguous(), a.lr)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    l1, _ = net.loss_grad(Rv, Ev)
    out["heldout_loss"] = [l0, l1]
    params = net.get_params()
    del R, E
    res = {}
    for L in sorted({a.L_train, a.L_eval}):
        U = Ut if L == a.L_train else torch.from_numpy(gauge.links(gauge.field(L, a.beta, 5))).cuda()
        h = ht if L == a.L_train else api.mg_setup(ctx, U, L, a.m0)
        n2 = api.Net(ctx, U, L, a.layers, a.channels, seed=2)
        n2.set_params(params)
        n2.attach(h)
        s1, x1 = timed_solves(api, ctx, h, 1, a.nrhs, seed=9)
        s2, x2 = timed_solves(api, ctx, h, 2, a.nrhs, seed=9)
        s1["agree"] = float((torch.abs(x1 - x2).max() / torch.abs(x1).max()).item())
        res[str(L)] = dict(vcycle=s1, vcycle_net=s2)
        n2.close()
        if h is not ht:
            h.close()
    out["solves"] = res
    ht.close()
    net.close()
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
