"""GPU parity: every CUDA step, called through the C ABI, against the CPU FP64
oracle on the same seeded inputs.  Tolerances (element-wise, relative to the
largest reference entry): stencil 1e-13 (FP64) / 1e-6 (FP32); multigrid
set-up (prolongators, Galerkin stencils, coarsest trace) 1e-10; solves and
level-difference samples 1e-8 at solver residual 1e-12; trace estimates 1e-8
for identical samples; Rademacher streams bit-exact."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import estimators as oest
from oracle import multigrid as omg
from oracle import rng as orng
from oracle import schwinger as osch
from synthetic import gauge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
    for h, _ in _HIER.values():
        h.close()
    _HIER.clear()
    c.close()


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


_FIELDS = {}


def field(L, beta=3.0, seed=0):
    key = (L, beta, seed)
    if key not in _FIELDS:
        _FIELDS[key] = gauge.links(gauge.field(L, beta, seed, sweeps=60))
    return _FIELDS[key]


def rand_vecs(n, k, seed):
    rs = np.random.default_rng(seed)
    return rs.standard_normal((k, n)) + 1j * rs.standard_normal((k, n))


# ---------------------------------------------------------------- RNG
def test_rademacher_bit_exact(api, ctx):
    z = api.mgmlmc_rademacher(ctx, 123, 2, orng.PHASE_SKETCH, 7, 1001, 5).cpu().numpy()
    for r in range(5):
        ref = orng.rademacher(123, 2, orng.PHASE_SKETCH, 7 + r, 1001)
        assert np.array_equal(z[r].real, ref) and np.all(z[r].imag == 0)


# ---------------------------------------------------------------- fine stencil
@pytest.mark.parametrize("L,nrhs", [(4, 1), (16, 3), (18, 5), (34, 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stencil_parity(api, ctx, L, nrhs, prec):
    U = field(L, 3.0, 1) if L % 2 == 0 and L >= 8 else gauge.links(gauge.quenched_u1(L, 3.0, 10, 1))
    m0 = -0.07
    x = rand_vecs(2 * L * L, nrhs, L)
    D = osch.dirac_sparse(U, m0)
    ref = (D @ x.T).T
    if prec == "fp64":
        xd = cuda(x)
        yd = torch.empty_like(xd)
        api.schwinger_apply(ctx, cuda(U), L, m0, xd, yd, api.FP64)
        assert relerr(yd.cpu().numpy(), ref) < 1e-13
    else:
        xd = cuda(x.astype(np.complex64))
        yd = torch.empty_like(xd)
        api.schwinger_apply(ctx, cuda(U), L, m0, xd, yd, api.FP32)
        ref32 = (D @ x.astype(np.complex64).astype(complex).T).T
        assert relerr(yd.cpu().numpy(), ref32) < 1e-6


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stencil_full_size_sampled(api, ctx, prec):
    """L = 512, the benchmark's 256-rhs FP32 launch (FP64: 64 rhs), sampled outputs."""
    L, m0 = 512, -0.1
    nrhs = 256 if prec == "fp32" else 64
    U = gauge.links(gauge.quenched_u1(L, 5.0, 3, 2))
    n = 2 * L * L
    g = torch.Generator(device="cuda").manual_seed(0)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    xd = torch.randn((nrhs, n), dtype=dt, device="cuda", generator=g)
    yd = torch.empty_like(xd)
    api.schwinger_apply(ctx, cuda(U), L, m0, xd, yd, api.FP32 if prec == "fp32" else api.FP64)
    torch.cuda.synchronize()
    rs = np.random.default_rng(1)
    rows = rs.integers(0, n, 3000)
    rhs = rs.integers(0, nrhs, 3000)
    D = osch.dirac_sparse(U, m0).tocsr()
    xs = xd.cpu().numpy().astype(complex)
    ys = yd.cpu().numpy()
    ref = np.array([D[r] @ xs[k] for r, k in zip(rows, rhs)]).ravel()
    got = ys[rhs, rows]
    assert relerr(got, ref) < (1e-6 if prec == "fp32" else 1e-13)
    # every rhs of the launch was written
    assert torch.isfinite(torch.view_as_real(yd)).all()


# ---------------------------------------------------------------- hierarchy
_HIER = {}


def hierarchies(api, ctx, L, m0=-0.05, ntv=8, seed=3, tensor_cores=2):
    """GPU hierarchy and the oracle's; tensor_cores: 2 = TF32 coarse images (the library default), 1 = BF16, 3 = FP16."""
    key = (L, m0, ntv, seed, tensor_cores)
    if key not in _HIER:
        U = field(L, 3.0, 2)
        h = api.mg_setup(ctx, cuda(U), L, m0, ntv=ntv, setup_sweeps=4, seed=seed, tensor_cores=tensor_cores)
        H = omg.Hierarchy(osch.dirac_sparse(U, m0), L, ntv=ntv, setup_sweeps=4, seed=seed)
        _HIER[key] = (h, H)
    return _HIER[key]


@pytest.mark.parametrize("L", [32, 64])
def test_hierarchy_parity(api, ctx, L):
    h, H = hierarchies(api, ctx, L)
    assert h.levels == H.levels and h.n == H.n
    for l in range(H.levels - 1):
        Pg = h.get_prolongator(l, 4, 8)                     # [agg][c][j][m]
        blocks = omg.aggregate_blocks(H.side[l], H.dof[l], 4)
        Po = H.P[l].tocsr()
        Lc, dc = H.side[l + 1], H.dof[l + 1]
        ref = np.empty_like(Pg)
        for T in range(Lc):
            for X in range(Lc):
                for c in range(2):
                    cols = (T * Lc + X) * dc + c * 8 + np.arange(8)
                    ref[T * Lc + X, c] = Po[blocks[X, T, c]][:, cols].toarray()
        assert relerr(Pg, ref) < 1e-10
    for l in range(1, H.levels):
        Sg = h.get_stencil(l)
        So = omg.stencil_blocks(H.D[l], H.side[l], H.dof[l]).reshape(Sg.shape)
        assert relerr(Sg, So) < 1e-10
    tL = np.trace(np.linalg.inv(H.D[-1].toarray()))
    assert abs(h.coarsest_trace() - tL) < 1e-10 * abs(tL)


def test_level_operators_and_transfers(api, ctx):
    h, H = hierarchies(api, ctx, 64)
    for l in range(H.levels):
        x = rand_vecs(H.n[l], 3, 10 + l)
        ref = (H.D[l] @ x.T).T
        y = torch.empty((3, H.n[l]), dtype=torch.complex128, device="cuda")
        h.apply(l, cuda(x), y, api.FP64)
        assert relerr(y.cpu().numpy(), ref) < 1e-12
        y32 = torch.empty((3, H.n[l]), dtype=torch.complex64, device="cuda")
        h.apply(l, cuda(x.astype(np.complex64)), y32, api.FP32)
        assert relerr(y32.cpu().numpy(), ref) < 2e-5
        if l + 1 < H.levels:
            P = H.P[l]
            xc = torch.empty((3, H.n[l + 1]), dtype=torch.complex128, device="cuda")
            h.restrict(l, cuda(x), xc, api.FP64)
            assert relerr(xc.cpu().numpy(), (P.conj().T @ x.T).T) < 1e-12
            v = rand_vecs(H.n[l + 1], 3, 20 + l)
            xf = torch.empty((3, H.n[l]), dtype=torch.complex128, device="cuda")
            h.prolong(l, cuda(v), xf, api.FP64)
            assert relerr(xf.cpu().numpy(), (P @ v.T).T) < 1e-12


TC_MODE = {"tf32": 2, "bf16": 1, "fp16": 3}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "fp16"])
def test_smoother_parity(api, ctx, prec):
    """SAP sweeps (the smoother of the V-cycle) against the oracle's SAP on the same level operator; TF32, BF16
    and FP16 tensor-core sweeps on the coarse levels (BF16: 8-bit significands; TF32 and FP16: 11-bit; FP32
    accumulation)."""
    h, H = hierarchies(api, ctx, 64, tensor_cores=TC_MODE.get(prec, 2))
    tol = {"fp64": 1e-12, "fp32": 2e-5, "tf32": 5e-3, "bf16": 2e-2, "fp16": 5e-3}[prec]
    for l in range(H.levels - 1):
        if prec in TC_MODE and l == 0:
            continue  # tensor-core smoother runs on coarse levels
        f = rand_vecs(H.n[l], 3, 40 + l)
        x0 = rand_vecs(H.n[l], 3, 50 + l)
        sap = omg.SAP(H.D[l], H.side[l], H.dof[l], 4 if l == 0 else 2)
        ref = sap.sweep(f.T.copy(), sap.sweep(f.T.copy(), x0.T.copy())).T
        dt = np.complex128 if prec == "fp64" else np.complex64
        xd = cuda(x0.astype(dt))
        h.smooth(l, cuda(f.astype(dt)), xd, {"fp64": api.FP64, "fp32": api.FP32, "tf32": api.TF32,
                                             "bf16": api.BF16, "fp16": api.FP16}[prec], 2)
        err = relerr(xd.cpu().numpy(), ref)
        assert err < tol, (l, err)
    assert h.tc_status() == 0


@pytest.mark.parametrize("fmt", ["tf32", "bf16", "fp16"])
def test_tensor_core_stencil(api, ctx, fmt):
    """tcgen05 coarse stencil (TF32, BF16 or FP16 operands, FP32 accumulation) against the oracle's Galerkin
    operator; ragged rhs counts."""
    h, H = hierarchies(api, ctx, 64, tensor_cores=TC_MODE[fmt])
    for l in range(1, H.levels):
        for nrhs in (1, 37, 130):
            x = rand_vecs(H.n[l], nrhs, 60 + nrhs)
            ref = (H.D[l] @ x.T).T
            y = torch.zeros((nrhs, H.n[l]), dtype=torch.complex64, device="cuda")
            h.apply(l, cuda(x.astype(np.complex64)), y, {"tf32": api.TF32, "bf16": api.BF16, "fp16": api.FP16}[fmt])
            err = relerr(y.cpu().numpy(), ref)
            assert err < (2e-2 if fmt == "bf16" else 5e-3), (l, nrhs, err)
    assert h.tc_status() == 0


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_block_and_site_stencil_kernels(api, ctx, fmt):
    """With 16-bit images the coarse stencil has two tcgen05 kernels: one site per item, and 2x2 sites per item
    sharing the block's slabs (N = 32 / 96 / 128 MMA windows).  Each is forced through the launch-variant table for
    every batch bucket (ragged rhs counts included) and checked against the oracle's Galerkin operator and SAP
    sweeps (the SAP residual runs the colour-block form of the block kernel); the two kernels agree to FP32
    accumulation order."""
    h, H = hierarchies(api, ctx, 64, tensor_cores=TC_MODE[fmt])
    f, prec = {"bf16": (1, api.BF16), "fp16": (2, api.FP16)}[fmt]
    tol = 2e-2 if fmt == "bf16" else 5e-3
    out = {}
    try:
        for variant in (0, 16):
            api.tune_clear()
            api.tune_set([dict(kind=1, side=H.side[l], bucket=b, format=f, variant=variant)
                          for l in range(1, H.levels) for b in (8, 16, 32, 64, 128, 256)])
            for l in range(1, H.levels):
                for nrhs in (1, 8, 37, 130, 256):
                    x = rand_vecs(H.n[l], nrhs, 70 + nrhs)
                    y = torch.zeros((nrhs, H.n[l]), dtype=torch.complex64, device="cuda")
                    h.apply(l, cuda(x.astype(np.complex64)), y, prec)
                    out[variant, l, nrhs] = y.cpu().numpy()
                    err = relerr(out[variant, l, nrhs], (H.D[l] @ x.T).T)
                    assert err < tol, (variant, l, nrhs, err)
            sap = omg.SAP(H.D[1], H.side[1], H.dof[1], 2)
            for nrhs in (3, 40, 130):  # one 32-row tile, one 64-row tile, three 64-row tiles (ragged)
                fv, x0 = rand_vecs(H.n[1], nrhs, 80 + nrhs), rand_vecs(H.n[1], nrhs, 90 + nrhs)
                ref = sap.sweep(fv.T.copy(), sap.sweep(fv.T.copy(), x0.T.copy())).T
                xd = cuda(x0.astype(np.complex64))
                h.smooth(1, cuda(fv.astype(np.complex64)), xd, prec, 2)
                err = relerr(xd.cpu().numpy(), ref)
                assert err < tol, (variant, nrhs, err)
            assert h.tc_status() == 0
    finally:
        api.tune_clear()
    for (variant, l, nrhs), y in out.items():
        if variant == 16:
            assert relerr(y, out[0, l, nrhs]) < 1e-5, (l, nrhs)


# ---------------------------------------------------------------- solver
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("level", [0, 1])
def test_fgmres_parity(api, ctx, prec, level):
    h, H = hierarchies(api, ctx, 64)
    n = H.n[level]
    b = rand_vecs(n, 6, 30 + level)
    st = api.fgmres_batched(ctx, h, level, cuda(b), x := torch.empty((6, n), dtype=torch.complex128, device="cuda"),
                            tol=1e-12, m=16, prec=api.MIXED if prec == "mixed" else api.FP64)
    assert st["converged"] and st["max_relres"] <= 1e-12
    ref = spla.splu(H.D[level].tocsc()).solve(b.T).T
    assert relerr(x.cpu().numpy(), ref) < 1e-8


def test_fgmres_fp32_and_unpreconditioned(api, ctx):
    h, H = hierarchies(api, ctx, 32)
    n = H.n[0]
    b = rand_vecs(n, 3, 5)
    ref = spla.splu(H.D[0].tocsc()).solve(b.T).T
    x32 = torch.empty((3, n), dtype=torch.complex64, device="cuda")
    st = api.fgmres_batched(ctx, h, 0, cuda(b.astype(np.complex64)), x32, tol=1e-5, prec=api.FP32)
    assert st["converged"]
    assert relerr(x32.cpu().numpy(), ref) < 1e-3
    x = torch.empty((3, n), dtype=torch.complex128, device="cuda")
    st = api.fgmres_batched(ctx, h, 0, cuda(b), x, tol=1e-10, prec=api.FP64, precond=0, m=30, maxit=20000)
    assert st["converged"] and relerr(x.cpu().numpy(), ref) < 1e-6


def test_not_converged_is_reported(api, ctx):
    from paper_2303_11512_gb300 import _lib
    h, H = hierarchies(api, ctx, 32)
    b = cuda(rand_vecs(H.n[0], 2, 1))
    x = torch.empty_like(b)
    with pytest.raises(_lib.MgmlmcError) as e:
        api.fgmres_batched(ctx, h, 0, b, x, tol=1e-14, maxit=2, prec=api.FP64)
    assert e.value.code == _lib.ERR_NOT_CONVERGED
    st = api.fgmres_batched(ctx, h, 0, b, x, tol=1e-14, maxit=2, prec=api.FP64, raise_on_nonconvergence=False)
    assert not st["converged"] and st["iters"] <= 2


def test_invalid_arguments(api, ctx):
    from paper_2303_11512_gb300 import _lib
    U = cuda(field(32))
    with pytest.raises(_lib.MgmlmcError) as e:
        api.mg_setup(ctx, U[:20, :20].contiguous(), 20, 0.0)
    assert e.value.code == _lib.ERR_INVALID_ARG
    x = torch.zeros((2, 2 * 32 * 32), dtype=torch.complex128, device="cuda")
    with pytest.raises(_lib.MgmlmcError):
        api.schwinger_apply(ctx, U, 32, 0.0, x, x, api.FP64)
    # nrhs = 0 is a no-op
    e0 = torch.zeros((0, 2 * 32 * 32), dtype=torch.complex128, device="cuda")
    api.schwinger_apply(ctx, U, 32, 0.0, e0, torch.zeros_like(e0), api.FP64)


# ---------------------------------------------------------------- level differences
@pytest.mark.parametrize("form", ["accumulated", "reduced"])
def test_level_sample_parity(api, ctx, form):
    h, H = hierarchies(api, ctx, 64)
    ld = oest.LevelDifference(H, form)
    seed, nrhs = 17, 5
    for l in range(H.levels - 1):
        nv = ld.vec_size(l)
        Z = np.stack([orng.rademacher(seed, l, orng.PHASE_STOCH, s, nv) for s in range(nrhs)], axis=1)
        tau_ref = np.einsum("ij,ij->j", Z, ld.apply(l, Z.astype(complex)))
        zf = api.mgmlmc_rademacher(ctx, seed, l, orng.PHASE_STOCH, 0, nv, nrhs)
        zl = api.mg_restrict_to_level(ctx, h, l, zf) if form == "accumulated" else zf
        y = torch.empty_like(zl)
        st = api.mlmc_level_sample(ctx, h, l, zl, y, tol=1e-12, prec=api.MIXED)
        assert st["converged"]
        tau = api.hutchpp_project(ctx, None, zl, y)
        assert relerr(tau, tau_ref) < 1e-8


@pytest.mark.parametrize("L,d", [(32, 8), (64, 8), (32, 48)])
def test_sketch_parity(api, ctx, L, d):
    h, H = hierarchies(api, ctx, L)
    ld = oest.LevelDifference(H)
    for l in range(H.levels - 1):
        sk, tlr = api.hutchpp_sketch_qr(ctx, h, l, d, 2, 9, api.ACCUMULATED, tol=1e-12, prec=api.MIXED)
        n = ld.vec_size(l)
        S = orng.rademacher_block(9, l, orng.PHASE_SKETCH, 0, n, d)
        for _ in range(2):
            S, _ = oest.qr_positive(ld.apply(l, S))
        tlr_ref = complex(np.sum(np.conj(S) * ld.apply(l, S)))
        assert abs(tlr - tlr_ref) < 1e-8 * abs(tlr_ref)
        Qg = sk.Q().cpu().numpy().T                      # n_l x d
        Qf = ld.Phat[l] @ Qg
        assert relerr(Qf, S) < 1e-6
        assert np.abs(Qg.conj().T @ Qg - np.eye(d)).max() < 1e-12
        # projected samples with this sketch against the oracle's z^H A zeta using the GPU's Q
        zf = api.mgmlmc_rademacher(ctx, 4, l, orng.PHASE_STOCH, 0, n, 3)
        zl = api.mg_restrict_to_level(ctx, h, l, zf)
        y = torch.empty_like(zl)
        api.mlmc_level_sample(ctx, h, l, zl, y, tol=1e-12)
        tau = api.hutchpp_project(ctx, sk, zl, y)
        Z = zf.cpu().numpy().T
        Y = ld.apply(l, Z)
        Zp = Z - S @ (S.conj().T @ Z)
        tau_ref = np.einsum("ij,ij->j", np.conj(Zp), Y)
        assert relerr(tau, tau_ref) < 1e-7
        sk.close()


# ---------------------------------------------------------------- Algorithm 2 end to end
@pytest.mark.parametrize("L,d,form", [(32, 8, "accumulated"), (64, 4, "accumulated"), (32, 0, "reduced")])
def test_trace_estimate_parity(api, ctx, L, d, form):
    h, H = hierarchies(api, ctx, L)
    nd = H.levels - 1
    cost = [1.0 + l for l in range(nd)]
    eps = 0.02
    r = api.trace_estimate(ctx, h, eps=eps, d=d, k=2, seed=11, cost=cost, nrhs_first=16, nrhs_max=64,
                           form=api.ACCUMULATED if form == "accumulated" else api.REDUCED, keep_samples=4096,
                           tol=1e-12)
    ro = oest.mgmlmc_pp(oest.LevelDifference(H, form), eps, d, 2, seed=11, cost=cost)
    assert r["N"] == ro["N"]
    for l in range(nd):
        assert relerr(r["samples"][l][: ro["N"][l]], ro["samples"][l]) < 1e-8
    assert abs(r["tau"] - ro["tau"]) < 1e-8 * abs(ro["tau"])
    assert abs(r["sigma"] - ro["sigma"]) < 1e-6 * ro["sigma"]
    assert r["sigma"] <= eps * abs(r["tau"]) * (1 + 1e-9)


# ---------------------------------------------------------------- fewer test vectors (Table 1)
@pytest.mark.parametrize("ntv", [2, 4])
def test_fewer_test_vectors(api, ctx, ntv):
    """Table 1's 2 and 4 test vectors per chirality (4 and 8 coarse dof per site; runtime-shape transfer, coarse
    stencil and SAP kernels, no tensor cores): prolongators, Galerkin stencils and the coarsest trace against the
    oracle's own hierarchy, level operators, a V-cycle, and level-difference samples in both forms."""
    h, H = hierarchies(api, ctx, 64, ntv=ntv)
    assert h.levels == H.levels and h.dof[1] == 2 * ntv
    for l in range(H.levels - 1):
        Pg = h.get_prolongator(l, 4, ntv)
        blocks = omg.aggregate_blocks(H.side[l], H.dof[l], 4)
        Po = H.P[l].tocsr()
        Lc, dc = H.side[l + 1], H.dof[l + 1]
        ref = np.empty_like(Pg)
        for T in range(Lc):
            for X in range(Lc):
                for c in range(2):
                    cols = (T * Lc + X) * dc + c * ntv + np.arange(ntv)
                    ref[T * Lc + X, c] = Po[blocks[X, T, c]][:, cols].toarray()
        assert relerr(Pg, ref) < 1e-10
    for l in range(1, H.levels):
        Sg = h.get_stencil(l)
        So = omg.stencil_blocks(H.D[l], H.side[l], H.dof[l]).reshape(Sg.shape)
        assert relerr(Sg, So) < 1e-10
        x = rand_vecs(H.n[l], 3, 40 + l)
        y = torch.empty((3, H.n[l]), dtype=torch.complex128, device="cuda")
        h.apply(l, cuda(x), y, api.FP64)
        assert relerr(y.cpu().numpy(), (H.D[l] @ x.T).T) < 1e-12
    tL = np.trace(np.linalg.inv(H.D[-1].toarray()))
    assert abs(h.coarsest_trace() - tL) < 1e-10 * abs(tL)
    b = rand_vecs(H.n[0], 3, 8)
    ref = H.vcycle(0, b.T, 1, 1).T
    x64 = torch.empty((3, H.n[0]), dtype=torch.complex128, device="cuda")
    h.vcycle(0, cuda(b), x64, api.FP64)
    assert relerr(x64.cpu().numpy(), ref) < 1e-11
    x32 = torch.empty((3, H.n[0]), dtype=torch.complex64, device="cuda")
    h.vcycle(0, cuda(b.astype(np.complex64)), x32, api.FP32)
    assert relerr(x32.cpu().numpy(), ref) < 1e-4
    for form in ("accumulated", "reduced"):
        ld = oest.LevelDifference(H, form)
        for l in range(H.levels - 1):
            nv = ld.vec_size(l)
            Z = np.stack([orng.rademacher(5, l, orng.PHASE_STOCH, s, nv) for s in range(4)], axis=1)
            tau_ref = np.einsum("ij,ij->j", Z, ld.apply(l, Z.astype(complex)))
            zf = api.mgmlmc_rademacher(ctx, 5, l, orng.PHASE_STOCH, 0, nv, 4)
            zl = api.mg_restrict_to_level(ctx, h, l, zf) if form == "accumulated" else zf
            yy = torch.empty_like(zl)
            st = api.mlmc_level_sample(ctx, h, l, zl, yy, tol=1e-12, prec=api.MIXED)
            assert st["converged"]
            assert relerr(api.hutchpp_project(ctx, None, zl, yy), tau_ref) < 1e-8, (form, l)
