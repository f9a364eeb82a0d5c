"""GPU parity of the estimator options and entry points beyond the default path, against the CPU oracle:
Z4 noise streams (bit-exact), the accumulated-form level difference on fine-size vectors
(eq. mlmc_decomp_matrix), gamma5-weighted traces with Z4 vectors through Algorithm 2, plain Hutchinson
(Algorithm 1) with unpreconditioned GMRES(30) on the L = 16 workload, and the V-cycle (FP64, FP32, and FP32
with the TF32 or BF16 tensor-core coarse levels) against the oracle's V-cycle.  Tolerances as in
test_gpu_parity: samples and estimates 1e-8 at solver residual 1e-12, V-cycles 1e-12 (FP64) / 2e-5 (FP32) /
5e-3 (TF32) / 2e-2 (BF16)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla  # noqa: F401

from oracle import estimators as oest
from oracle import multigrid as omg
from oracle import rng as orng
from oracle import schwinger as osch
from synthetic import gauge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    return api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def h64(api, ctx):
    U = gauge.links(gauge.field(64, 3.0, 2, sweeps=60))
    m0 = -0.05
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), 64, m0, ntv=8, setup_sweeps=4, seed=3)
    H = omg.Hierarchy(osch.dirac_sparse(U, m0), 64, ntv=8, setup_sweeps=4, seed=3)
    yield h, H, U, m0
    h.close()


def test_noise_streams_bit_exact(api, ctx):
    z = api.mgmlmc_noise(ctx, api.NOISE_Z4, 77, 1, orng.PHASE_STOCH, 5, 999, 4).cpu().numpy()
    for r in range(4):
        assert np.array_equal(z[r], orng.z4(77, 1, orng.PHASE_STOCH, 5 + r, 999))
    a = api.mgmlmc_noise(ctx, api.NOISE_RADEMACHER, 77, 1, orng.PHASE_STOCH, 5, 999, 2).cpu().numpy()
    b = api.mgmlmc_rademacher(ctx, 77, 1, orng.PHASE_STOCH, 5, 999, 2).cpu().numpy()
    assert np.array_equal(a, b)


def test_level_sample_accumulated_form_on_fine_vectors(api, ctx, h64):
    h, H, _, _ = h64
    ld = oest.LevelDifference(H, "accumulated")
    for l in range(H.levels - 1):
        Z = orng.rademacher_block(9, l, orng.PHASE_STOCH, 0, H.n[0], 3)
        zd = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
        y = torch.empty_like(zd)
        st = api.mlmc_level_sample(ctx, h, l, zd, y, form=api.ACCUMULATED, tol=1e-12, prec=api.MIXED)
        assert st["converged"]
        assert relerr(y.cpu().numpy(), ld.apply(l, Z).T) < 1e-8


@pytest.mark.parametrize("form", ["accumulated", "reduced"])
def test_gamma5_trace_with_z4_noise(api, ctx, form):
    """tr(gamma5 D^{-1}) by Algorithm 2 with Z4 vectors: identical N, samples, low-rank parts and tau_L."""
    U = gauge.links(gauge.field(32, 3.0, 2, sweeps=60))
    m0 = -0.05
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), 32, m0, ntv=8, setup_sweeps=4, seed=3)
    H = omg.Hierarchy(osch.dirac_sparse(U, m0), 32, ntv=8, setup_sweeps=4, seed=3)
    try:
        nd = H.levels - 1
        cost = [1.0 + l for l in range(nd)]
        fm = api.ACCUMULATED if form == "accumulated" else api.REDUCED
        r = api.trace_estimate(ctx, h, eps=0.3, d=6, k=2, seed=13, cost=cost, nrhs_first=16, nrhs_max=64,
                               form=fm, keep_samples=2048, tol=1e-12, noise=api.NOISE_Z4,
                               weight=api.TRACE_GAMMA5, max_samples=300)
        ld = oest.LevelDifference(H, form, gamma5=True)
        ro = oest.mgmlmc_pp(ld, 0.3, 6, 2, seed=13, cost=cost, noise=orng.NOISE_Z4, max_samples=300)
        assert r["N"] == ro["N"]
        for l in range(nd):
            assert relerr(r["samples"][l][: ro["N"][l]], ro["samples"][l]) < 1e-8
            assert abs(r["tau_lr"][l] - ro["tau_lr"][l]) < 1e-8 * max(abs(ro["tau_lr"][l]), 1.0)
        assert abs(r["tau_L"] - ro["tau_L"]) < 1e-10 * abs(ro["tau_L"])
        assert abs(r["tau"] - ro["tau"]) < 1e-8 * max(abs(ro["tau"]), 1.0)
        exact = np.trace(osch.gamma5(32).toarray() @ np.linalg.inv(H.D[0].toarray()))
        assert abs(r["tau"] - exact) < 4.5 * r["sigma"]
    finally:
        h.close()


def test_plain_hutchinson_gmres30(api, ctx):
    """Algorithm 1 on the L = 16 workload (beta 3, m0 -0.05, 500 Metropolis sweeps) with unpreconditioned
    GMRES(30): samples equal the oracle's (exact solves) at solver residual 1e-12; at 1e-10 the estimate is
    within 4.5 sigma of the dense-LU trace.  Also with Z4 vectors and gamma5 weighting."""
    L, m0 = 16, -0.05
    U = gauge.links(gauge.field(L, 3.0, 0))
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), L, m0, ntv=4, setup_sweeps=2)
    try:
        Dd = osch.dirac_dense(U, m0)
        A = np.linalg.inv(Dd)
        exact = np.trace(A)
        r = api.hutchinson_estimate(ctx, h, eps=0.02, seed=4, keep_samples=4096, precond=0, m=30, tol=1e-12,
                                    maxit=20000, prec=api.FP64)
        tau, V, s, taus = oest.hutchinson(lambda b: A @ b, A.shape[0], 0.02, seed=4)
        assert r["N"] == s
        assert relerr(r["samples"][:s], taus) < 1e-8
        assert abs(r["tau"] - tau) < 1e-8 * abs(tau)
        r10 = api.hutchinson_estimate(ctx, h, eps=0.02, seed=4, precond=0, m=30, tol=1e-10, maxit=20000,
                                      prec=api.FP64)
        assert abs(r10["tau"] - exact) < 4.5 * r10["sigma"]
        g5 = np.tile([1.0, -1.0], L * L)
        r5 = api.hutchinson_estimate(ctx, h, eps=0.5, seed=6, keep_samples=4096, precond=0, m=30, tol=1e-12,
                                     maxit=20000, prec=api.FP64, noise=api.NOISE_Z4, weight=api.TRACE_GAMMA5,
                                     max_samples=400)
        t5, V5, s5, taus5 = oest.hutchinson(lambda b: A @ b, A.shape[0], 0.5, seed=6, noise=orng.NOISE_Z4,
                                            weight=g5, smax=400)
        assert r5["N"] == s5 and relerr(r5["samples"][:s5], taus5) < 1e-8
    finally:
        h.close()


@pytest.mark.parametrize("mode", ["fp64", "fp32", "tf32", "bf16", "fp16"])
def test_vcycle_parity(api, ctx, h64, mode):
    """mg_vcycle against the oracle's V(1,1) cycle on the same (deterministic) hierarchy; with tensor cores
    the coarse level's SAP sweeps and the residual after pre-smoothing run as tcgen05 GEMMs (TF32 or BF16)."""
    h, H, U, m0 = h64
    hh = h
    if mode != "fp64":   # the same hierarchy without / with TF32 / with BF16 tensor-core coarse kernels
        hh = api.mg_setup(ctx, torch.from_numpy(U).cuda(), 64, m0, ntv=8, setup_sweeps=4, seed=3,
                          tensor_cores={"fp32": 0, "tf32": 2, "bf16": 1, "fp16": 3}[mode])
    try:
        rs = np.random.default_rng(3)
        b = rs.standard_normal((5, H.n[0])) + 1j * rs.standard_normal((5, H.n[0]))
        ref = H.vcycle(0, b.T, 1, 1).T
        if mode == "fp64":
            x = torch.empty((5, H.n[0]), dtype=torch.complex128, device="cuda")
            hh.vcycle(0, torch.from_numpy(b).cuda(), x, api.FP64)
            tol = 1e-12
        else:
            x = torch.empty((5, H.n[0]), dtype=torch.complex64, device="cuda")
            hh.vcycle(0, torch.from_numpy(b.astype(np.complex64)).cuda(), x, api.FP32)
            tol = {"fp32": 2e-5, "tf32": 5e-3, "bf16": 2e-2, "fp16": 5e-3}[mode]
        err = relerr(x.cpu().numpy(), ref)
        assert err < tol, err
        assert hh.tc_status() == 0
    finally:
        if hh is not h:
            hh.close()


def test_deflation_basis_and_deflated_hutchinson(api, ctx):
    """Exactly deflated Hutchinson (Section 2; the paper's comparator) on the L = 16 workload field: the GPU's
    block power iteration on D^{-1} gamma5 equals the oracle's from the same start vectors (basis 1e-6, direct
    part tr(V^H D^{-1} V) 1e-8); with 160 sweeps it spans the exact singular subspace of the oracle's dense
    Hermitian eigensolver (k = 6, the widest gap); the deflated samples equal the oracle's on the GPU's basis
    (1e-8, same N)."""
    L, m0 = 16, -0.05
    U = gauge.links(gauge.field(L, 3.0, 0))
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), L, m0, ntv=4, setup_sweeps=2)
    try:
        from oracle import deflation as odf
        D = osch.dirac_dense(U, m0)
        A = np.linalg.inv(D)
        n, k = D.shape[0], 6
        sk, tdf, res = api.deflation_basis(ctx, h, k, 40, seed=3, tol=1e-12, prec=api.FP64)
        Vg = sk.Q().cpu().numpy().T
        Vo = odf.subspace_iteration(lambda b: A @ b, n, k, 40, seed=3)
        assert relerr(Vg, Vo) < 1e-6
        assert abs(tdf - odf.deflation_trace(lambda b: A @ b, Vg)) < 1e-8 * abs(tdf)
        sk.close()
        sk2, tdf2, res2 = api.deflation_basis(ctx, h, k, 160, seed=3, tol=1e-12, prec=api.FP64)
        V2 = sk2.Q().cpu().numpy().T
        Vex, mu, tex = odf.singular_deflation_dense(D, k)
        assert np.abs(V2 @ V2.conj().T - Vex @ Vex.conj().T).max() < 1e-7
        assert abs(tdf2 - tex) < 1e-7 * abs(tex)
        assert res2 < res and res2 < 1e-6, (res, res2)
        r = api.hutchinson_estimate(ctx, h, eps=0.01, seed=7, keep_samples=4096, tol=1e-12, prec=api.FP64,
                                    deflate=sk2, min_samples=20)
        ro = odf.deflated_hutchinson(lambda b: A @ b, V2, tdf2, n, 0.01, seed=7, min_samples=20)
        assert r["N"] == ro["s"]
        assert relerr(r["samples"][: ro["s"]], ro["samples"]) < 1e-8
        assert abs(r["tau"] - ro["tau"]) < 1e-8 * abs(ro["tau"])
        assert abs(r["tau"] - np.trace(A)) < 5 * r["sigma"]
        sk2.close()
    finally:
        h.close()
