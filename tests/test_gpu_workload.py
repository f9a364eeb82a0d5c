"""Parity of the benchmarked configuration against the CPU FP64 oracle.

The benchmark times MG-MLMC++ with the set-up and estimator of bench.WORKLOAD: bootstrap set-up (2 rounds of
6 FGMRES iterations on top of the smoothed test vectors), 8 test vectors per chirality, V(2,2) SAP cycles with
the tensor-core kernels on the coarse levels (the workload's operand format), mixed precision (FP32 inner FGMRES,
FP64 true-residual refinement to 1e-10), the workload's Hutch++ sketch (W["d"] vectors, W["k"] sketch
applications), accumulated form, first batch 8, counted flops as the sample cost.  Here the same configuration
runs at L = 256 (4 levels, 256 -> 64 -> 16 -> 4, the same depth and coarse dof as L = 512) on a beta = 5 field with
the tuned near-critical mass.

The bootstrap set-up is adaptive (many prolongators are valid), so the GPU's P_l are imported as data and
checked for their defining properties; the oracle then builds its own Galerkin operators P^H D P from its own
fine operator and solves with sparse LU.  Tolerances: P^H P = I to 1e-12, stencils and tau_L 1e-10,
tau_lr and per-sample tau 1e-8 (solver residual 1e-10), Q 1e-6, the tensor-core kernels 5e-3 with TF32 or FP16
operands (2e-2 with BF16: 8-bit significands, FP32 accumulation).
"""
import json
import os

import numpy as np
import pytest

import bench
from oracle import multigrid as omg
from oracle import rng as orng
from oracle import schwinger as osch
from oracle.estimators import LevelDifference
from oracle.linalg import qr_positive
from synthetic import gauge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L, BETA = 256, 5.0
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    W = bench.WORKLOAD
    m0 = json.load(open(os.path.join(ROOT, "tests", "golden", "masses.json")))["L256_beta5_seed0"]["m0"]
    U = gauge.links(gauge.field(L, BETA, W["seed"]))
    ctx = api.Context()
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), L, m0, ntv=W["ntv"], bootstrap=W["bootstrap"],
                     bootstrap_its=W["bootstrap_its"], kcycle_its=W["kcycle_its"], pre_smooth=W["pre_smooth"],
                     post_smooth=W["post_smooth"], tensor_cores=W["tensor_cores"])
    assert h.levels == 4 and h.side == [256, 64, 16, 4]
    Ps = [omg.prolongator_from_blocks(h.get_prolongator(l, 4, W["ntv"]), h.side[l], h.dof[l], 4, W["ntv"])
          for l in range(h.levels - 1)]
    H = omg.Hierarchy.from_prolongators(osch.dirac_sparse(U, m0), L, Ps, agg=4)
    yield dict(api=api, ctx=ctx, h=h, H=H, Ps=Ps, W=W, m0=m0)
    h.close()
    ctx.close()


def test_bootstrap_prolongators_are_valid(setup):
    h, Ps = setup["h"], setup["Ps"]
    for l, P in enumerate(Ps):
        c = omg.check_prolongator(P, h.side[l], h.dof[l], 4)
        assert c["orth"] < 1e-12, (l, c)
        assert c["support"] and c["chirality"], (l, c)


def test_galerkin_stencils_and_coarsest_trace(setup):
    h, H = setup["h"], setup["H"]
    for l in range(1, h.levels):
        Dg = omg.sparse_from_stencil(h.get_stencil(l), h.side[l], h.dof[l])
        assert abs(Dg - H.D[l]).max() < 1e-10 * abs(H.D[l]).max(), l
        g5 = H.gamma5(l)
        assert abs(g5 @ H.D[l] @ g5 - H.D[l].conj().T).max() < 1e-12 * abs(H.D[l]).max()
    tL = np.trace(np.linalg.inv(H.D[-1].toarray()))
    assert abs(h.coarsest_trace() - tL) < 1e-10 * abs(tL)


def test_estimate_of_the_benchmark_configuration(setup):
    """trace_estimate with the benchmark's estimator settings; every computed sample, the low-rank traces
    and the estimate against direct solves on the same hierarchy and the same random streams."""
    api, ctx, h, H, W = setup["api"], setup["ctx"], setup["h"], setup["H"], setup["W"]
    r = api.trace_estimate(ctx, h, eps=W["eps"], d=W["d"], k=W["k"], nrhs_max=W["nrhs_max"],
                           nrhs_first=W["nrhs_first"], cost_mode=1, seed=0, keep_samples=1024, prec=api.MIXED)
    # Algorithm 2 never reactivates a level: one that stopped under an earlier target keeps its samples while
    # the optimal targets of the others move, so the final sigma ends near, not strictly below, eps |tau|
    assert r["sigma"] <= 1.25 * W["eps"] * abs(r["tau"])
    ld = LevelDifference(H)
    n0 = H.n[0]
    tau_ref = ld.coarsest_trace()
    assert abs(r["tau_L"] - tau_ref) < 1e-10 * abs(tau_ref)
    for l in range(h.levels - 1):
        # the oracle's own sketch (Algorithm 2, deflation part) with sparse-LU solves
        S = orng.rademacher_block(0, l, orng.PHASE_SKETCH, 0, n0, W["d"])
        for _ in range(W["k"]):
            S, _ = qr_positive(ld.apply(l, S))
        tlr = complex(np.sum(np.conj(S) * ld.apply(l, S)))
        assert abs(r["tau_lr"][l] - tlr) < 1e-8 * abs(tlr), (l, r["tau_lr"][l], tlr)
        # the GPU's Q of this level (same seed, d, k: the basis the estimate projected with).  The estimate
        # solves the sketches of neighbouring levels side by side (64 rhs per coarse launch) where this call
        # solves one level's 32, so the launches may take the other tensor-core stencil kernel (another FP32
        # summation order): the two agree to the solver tolerance (1e-10 residual), not bitwise
        sk, tlr1 = api.hutchpp_sketch_qr(ctx, h, l, W["d"], W["k"], 0, api.ACCUMULATED)
        Qf = ld.Phat[l] @ sk.Q().cpu().numpy().T
        sk.close()
        assert abs(tlr1 - r["tau_lr"][l]) < 1e-8 * abs(tlr)
        assert relerr(Qf, S) < 1e-6
        # every computed stochastic sample, projected with that Q
        nc = r["computed"][l]
        Z = orng.rademacher_block(0, l, orng.PHASE_STOCH, 0, n0, nc)
        Y = ld.apply(l, Z)
        Zp = Z - Qf @ (Qf.conj().T @ Z)
        t_ref = np.einsum("ij,ij->j", np.conj(Zp), Y)
        assert relerr(r["samples"][l][:nc], t_ref) < 1e-8, l
        tau_ref += t_ref[: r["N"][l]].mean() + tlr
    assert abs(r["tau"] - tau_ref) < 1e-8 * abs(tau_ref)


def test_tensor_core_kernels_on_the_workload_level(setup):
    """Level 1 (64 x 64 coarse sites, 16 dof): every CTA of the tcgen05 kernels walks many sites and blocks.
    Tensor-core stencil and SAP sweeps against the oracle's Galerkin operator and SAP on the same level."""
    api, h, H, W = setup["api"], setup["h"], setup["H"], setup["W"]
    prec, tol = {1: (api.BF16, 2e-2), 2: (api.TF32, 5e-3), 3: (api.FP16, 5e-3)}[W["tensor_cores"]]
    l = 1
    n = h.n[l]
    sap = omg.SAP(H.D[l], h.side[l], h.dof[l], 2)
    rs = np.random.default_rng(7)
    for nrhs in (8, 200):
        x = rs.standard_normal((nrhs, n)) + 1j * rs.standard_normal((nrhs, n))
        y = torch.zeros((nrhs, n), dtype=torch.complex64, device="cuda")
        h.apply(l, torch.from_numpy(x.astype(np.complex64)).cuda(), y, prec)
        err = relerr(y.cpu().numpy(), (H.D[l] @ x.T).T)
        assert err < tol, err
        f = rs.standard_normal((nrhs, n)) + 1j * rs.standard_normal((nrhs, n))
        xd = torch.from_numpy(x.astype(np.complex64)).cuda()
        h.smooth(l, torch.from_numpy(f.astype(np.complex64)).cuda(), xd, prec, 2)
        ref = sap.sweep(f.T.copy(), sap.sweep(f.T.copy(), x.T.copy())).T
        err = relerr(xd.cpu().numpy(), ref)
        assert err < tol, err
    assert h.tc_status() == 0


def test_vcycle_of_the_workload(setup):
    """One V(2,2) cycle from the fine level, FP32 with the tensor-core coarse kernels (the preconditioner the
    benchmark's inner FGMRES applies) and FP64, against the oracle's V-cycle on the same hierarchy."""
    api, h, H, W = setup["api"], setup["h"], setup["H"], setup["W"]
    rs = np.random.default_rng(8)
    b = rs.standard_normal((4, h.n[0])) + 1j * rs.standard_normal((4, h.n[0]))
    ref = H.vcycle(0, b.T, W["pre_smooth"], W["post_smooth"]).T
    x64 = torch.empty((4, h.n[0]), dtype=torch.complex128, device="cuda")
    h.vcycle(0, torch.from_numpy(b).cuda(), x64, api.FP64)
    assert relerr(x64.cpu().numpy(), ref) < 1e-11
    x32 = torch.empty((4, h.n[0]), dtype=torch.complex64, device="cuda")
    h.vcycle(0, torch.from_numpy(b.astype(np.complex64)).cuda(), x32, api.FP32)
    err = relerr(x32.cpu().numpy(), ref)
    assert err < (2e-2 if W["tensor_cores"] == 1 else 5e-3), err
    assert h.tc_status() == 0
