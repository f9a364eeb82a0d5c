"""The L = 128 MG-MLMC configuration in both precision forms against the CPU FP64 oracle.

L = 128 (n = 32768), beta = 3, m0 tuned so that the smallest |eigenvalue| of D is about 1e-3, three levels
(128 -> 32 -> 8, n = 32768 / 16384 / 1024), 4x4 aggregates, 8 test vectors per chirality, Galerkin coarse
operators, MG-MLMC (no deflation, d = 0), batches of up to 64 Rademacher right-hand sides per launch, FGMRES with
the V-cycle to the true relative residual 1e-10.  Two forms of the solves: all FP64, and FP32 inner FGMRES +
V-cycle (tensor-core coarse kernels) with FP64 true-residual refinement.  The oracle imports the GPU's
prolongators, builds its own Galerkin operators and solves with sparse LU, so every computed sample is compared.

Stated errors against the oracle: per-sample tau 1e-8 relative (solver residual 1e-10 and a condition number of
about 10^2 on these level differences), trace estimate 1e-8 relative on identical samples, coarsest trace 1e-10.
"""
import json
import os

import numpy as np
import pytest

from oracle import multigrid as omg
from oracle import rng as orng
from oracle import schwinger as osch
from oracle.estimators import LevelDifference
from synthetic import gauge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
L, BETA = 128, 3.0


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def c1():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    m0 = json.load(open(os.path.join(ROOT, "tests", "golden", "masses.json")))["L128_beta3_seed0"]["m0"]
    U = gauge.links(gauge.field(L, BETA, 0))
    ctx = api.Context()
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), L, m0, ntv=8)
    assert h.levels == 3 and h.side == [128, 32, 8]
    Ps = [omg.prolongator_from_blocks(h.get_prolongator(l, 4, 8), h.side[l], h.dof[l], 4, 8)
          for l in range(h.levels - 1)]
    H = omg.Hierarchy.from_prolongators(osch.dirac_sparse(U, m0), L, Ps, agg=4)
    yield dict(api=api, ctx=ctx, h=h, H=H, ld=LevelDifference(H))
    h.close()
    ctx.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_mlmc_l128_both_forms(c1, form):
    api, ctx, h, H, ld = c1["api"], c1["ctx"], c1["h"], c1["H"], c1["ld"]
    prec = api.FP64 if form == "fp64" else api.MIXED
    r = api.trace_estimate(ctx, h, eps=2e-3, d=0, k=1, nrhs_max=64, nrhs_first=16, cost_mode=1, seed=3,
                           keep_samples=2048, prec=prec, tol=1e-10)
    assert r["sigma"] <= 1.25 * 2e-3 * abs(r["tau"])
    tau_ref = ld.coarsest_trace()
    assert abs(r["tau_L"] - tau_ref) < 1e-10 * abs(tau_ref)
    n0 = H.n[0]
    for l in range(h.levels - 1):
        nc = r["computed"][l]
        Z = orng.rademacher_block(3, l, orng.PHASE_STOCH, 0, n0, nc)
        t_ref = np.einsum("ij,ij->j", np.conj(Z), ld.apply(l, Z))
        err = relerr(r["samples"][l][:nc], t_ref)
        assert err < 1e-8, (form, l, err)
        tau_ref += t_ref[: r["N"][l]].mean()
    assert abs(r["tau"] - tau_ref) < 1e-8 * abs(tau_ref)
    print("\n[C1 %s] tau %s sigma %.3g N %s solves %d" % (form, r["tau"], r["sigma"], r["N"], r["solves"]))
