"""The allocation-free projection entry point against the regular one.

hutchpp_project_noalloc exists for callers that cannot allocate device memory
when they need projected samples (a framework that owns all device memory
through its own allocator, or a serving loop that forbids cudaMalloc after
start-up).  It must give the same samples as hutchpp_project, call after call,
although every call reuses the same fixed device scratch array.  This file is
collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ref(Q, z, y):
    """tau_r = zeta_r^H y_r - (Q^H zeta_r)^H (Q^H y_r) in numpy FP64 (Q rows are the basis vectors)."""
    Qm = Q.T
    c = Qm.conj().T @ z.T
    g = Qm.conj().T @ y.T
    return np.einsum("rn,rn->r", np.conj(z), y) - np.einsum("ir,ir->r", np.conj(c), g)


def test_noalloc_projection_matches_hutchpp_project():
    import __graft_entry__ as gentry
    gentry.build()
    from paper_2303_11512_gb300 import _lib, api
    from synthetic import gauge

    ctx = api.Context()
    U = torch.from_numpy(gauge.links(gauge.field(32, 3.0, 7, sweeps=30))).cuda()
    h = api.mg_setup(ctx, U, 32, -0.05, ntv=4, setup_sweeps=2, seed=2)
    sk, _ = api.hutchpp_sketch_qr(ctx, h, 0, 8, 2, 5, tol=1e-10)
    Q = sk.Q()
    n = h.n[0]
    gen = torch.Generator(device="cuda").manual_seed(3)
    # two calls in a row with different shapes: the second must not see the first's scratch
    for nrhs in (37, 13):
        z = torch.randn((nrhs, n), dtype=torch.complex128, device="cuda", generator=gen)
        y = torch.randn((nrhs, n), dtype=torch.complex128, device="cuda", generator=gen)
        ref = api.hutchpp_project(ctx, sk, z, y)
        tau = torch.full((nrhs,), float("nan"), dtype=torch.complex128, device="cuda")
        api.hutchpp_project_noalloc(Q, z, y, tau)
        torch.cuda.synchronize()
        got = tau.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # no deflation (d = 0) reduces to zeta^H y
    tau0 = torch.empty((13,), dtype=torch.complex128, device="cuda")
    api.hutchpp_project_noalloc(None, z, y, tau0)
    ref0 = api.hutchpp_project(ctx, None, z, y)
    assert np.abs(tau0.cpu().numpy() - ref0).max() <= 1e-12 * np.abs(ref0).max()
    # sizes beyond the fixed scratch are rejected before anything is launched
    big = torch.zeros((257, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(_lib.MgmlmcError) as e:
        api.hutchpp_project_noalloc(None, big, big, torch.zeros((257,), dtype=torch.complex128, device="cuda"))
    assert e.value.code == _lib.ERR_INVALID_ARG
    sk.close()
    h.close()
    ctx.close()


def test_noalloc_at_the_limits_tiny_rows_and_side_stream():
    """nrhs = 256 and d = 32 fill the scratch array completely; n = 8 leaves most row chunks empty (they must
    contribute zeros); a call on a side stream, synchronised before the comparison.  Reference: numpy FP64."""
    import __graft_entry__ as gentry
    gentry.build()
    from paper_2303_11512_gb300 import api

    rs = np.random.default_rng(11)
    for nrhs, d, n in ((256, 32, 3000), (7, 4, 8), (3, 0, 8)):
        Qn = np.linalg.qr(rs.standard_normal((n, max(d, 1))) + 1j * rs.standard_normal((n, max(d, 1))))[0].T[:d]
        z = rs.standard_normal((nrhs, n)) + 1j * rs.standard_normal((nrhs, n))
        y = rs.standard_normal((nrhs, n)) + 1j * rs.standard_normal((nrhs, n))
        ref = _ref(Qn, z, y) if d else np.einsum("rn,rn->r", np.conj(z), y)
        Qd = torch.from_numpy(np.ascontiguousarray(Qn)).cuda() if d else None
        tau = torch.full((nrhs,), float("nan"), dtype=torch.complex128, device="cuda")
        api.hutchpp_project_noalloc(Qd, torch.from_numpy(z).cuda(), torch.from_numpy(y).cuda(), tau)
        torch.cuda.synchronize()
        assert np.abs(tau.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    side = torch.cuda.Stream()
    z = torch.from_numpy(rs.standard_normal((9, 500)) + 0j).cuda()
    y = torch.from_numpy(rs.standard_normal((9, 500)) + 0j).cuda()
    tau = torch.full((9,), float("nan"), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        api.hutchpp_project_noalloc(None, z, y, tau, stream=side)
    side.synchronize()
    ref = np.einsum("rn,rn->r", np.conj(z.cpu().numpy()), y.cpu().numpy())
    assert np.abs(tau.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
