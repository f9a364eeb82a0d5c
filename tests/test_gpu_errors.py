"""Error paths on the GPU, made on the host side (no fault, no trap, no hang): a NaN gauge link and a NaN
right-hand side report MGMLMC_ERR_NAN; a rank-deficient basis reports MGMLMC_ERR_NOT_POSDEF from CholeskyQR2;
the coarsest-level Gauss-Jordan kernel's grid barrier, told to wait for one arrival more than the grid has,
runs out of its bounded wait and reports MGMLMC_ERR_TIMEOUT, after which the same context inverts normally.
Also the parity of those two entry points: the dense inverse (n = 1024, the coarsest size of the L = 512
workload, and ragged n) against numpy, CholeskyQR2 against the oracle's Householder QR."""
import numpy as np
import pytest

from oracle.linalg import qr_positive
from synthetic import gauge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import _lib, api
    ctx = api.Context()
    yield api, _lib, ctx
    ctx.close()


def test_nan_gauge_link_and_nan_rhs(env):
    api, _lib, ctx = env
    U = gauge.links(gauge.field(32, 3.0, 1, sweeps=20))
    bad = U.copy()
    bad[3, 5, 1] = np.nan
    with pytest.raises(_lib.MgmlmcError) as e:
        api.mg_setup(ctx, torch.from_numpy(bad).cuda(), 32, -0.05)
    assert e.value.code == _lib.ERR_NAN
    h = api.mg_setup(ctx, torch.from_numpy(U).cuda(), 32, -0.05, ntv=4, setup_sweeps=2)
    try:
        b = torch.randn((3, h.n[0]), dtype=torch.complex128, device="cuda")
        b[1, 17] = float("nan")
        x = torch.empty_like(b)
        for prec in (api.FP64, api.MIXED):
            with pytest.raises(_lib.MgmlmcError) as e:
                api.fgmres_batched(ctx, h, 0, b, x, prec=prec)
            assert e.value.code == _lib.ERR_NAN
        b[1, 17] = 0.5   # the context and hierarchy stay usable
        st = api.fgmres_batched(ctx, h, 0, b, x, prec=api.MIXED)
        assert st["converged"]
    finally:
        h.close()


@pytest.mark.parametrize("d", [24, 50, 64])
def test_cholqr2_parity_and_rank_deficiency(env, d):
    api, _lib, ctx = env
    rs = np.random.default_rng(2)
    n = 5000
    Y = rs.standard_normal((n, d)) + 1j * rs.standard_normal((n, d))
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda()
    api.hutchpp_cholqr2(ctx, Yd)
    Q = Yd.cpu().numpy().T
    Qr, _ = qr_positive(Y)
    assert np.abs(Q - Qr).max() < 1e-12
    assert np.abs(Q.conj().T @ Q - np.eye(d)).max() < 1e-13
    Y[:, 7] = Y[:, 3]   # rank d - 1
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda()
    with pytest.raises(_lib.MgmlmcError) as e:
        api.hutchpp_cholqr2(ctx, Yd)
    assert e.value.code == _lib.ERR_NOT_POSDEF


@pytest.mark.parametrize("n", [1, 37, 1024])
def test_dense_inverse_parity(env, n):
    api, _lib, ctx = env
    rs = np.random.default_rng(n)
    A = rs.standard_normal((n, n)) + 1j * rs.standard_normal((n, n)) + 4 * np.sqrt(n) * np.eye(n)
    ref = np.linalg.inv(A)
    Ad = torch.from_numpy(A).cuda()
    api.mg_dense_inverse(ctx, Ad, api.FP64)
    assert np.abs(Ad.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    A32 = torch.from_numpy(A.astype(np.complex64)).cuda()
    api.mg_dense_inverse(ctx, A32, api.FP32)
    assert np.abs(A32.cpu().numpy() - ref).max() < 1e-4 * np.abs(ref).max()


def test_dense_inverse_singular_and_barrier_timeout(env):
    api, _lib, ctx = env
    rs = np.random.default_rng(5)
    n = 300
    A = rs.standard_normal((n, n)) + 1j * rs.standard_normal((n, n))
    S = A.copy()
    S[:, 11] = 0.0   # a zero column: no pivot for column 11
    with pytest.raises(_lib.MgmlmcError) as e:
        api.mg_dense_inverse(ctx, torch.from_numpy(S).cuda(), api.FP64)
    assert e.value.code == _lib.ERR_NAN
    # every barrier wait runs out after 1000 polls: the kernel stops and reports, the device stays usable
    with pytest.raises(_lib.MgmlmcError) as e:
        api.mg_dense_inverse(ctx, torch.from_numpy(A).cuda(), api.FP64, barrier_polls=-1000)
    assert e.value.code == _lib.ERR_TIMEOUT
    Ad = torch.from_numpy(A).cuda()
    api.mg_dense_inverse(ctx, Ad, api.FP64)
    ref = np.linalg.inv(A)
    assert np.abs(Ad.cpu().numpy() - ref).max() < 1e-11 * np.abs(ref).max()
