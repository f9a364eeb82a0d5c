"""GPU checks of the learned gauge-covariant preconditioner: forward output and
loss gradients against the FP64 oracle network (same bf16-rounded weights),
gauge covariance of the CUDA forward, and training on (residual, error) pairs
harvested from the library's own V-cycle and solves, used as a correction after
the V-cycle inside FGMRES."""
import numpy as np
import pytest

from oracle import nn as onn
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
    c.close()


def _setup(api, ctx, L=16, C=4, layers=4, seed=0, tc=False):
    th = gauge.quenched_u1(L, 3.0, 20, seed)
    U = gauge.links(th)
    W, b = onn.init_params(C, layers, seed + 1)
    rs = np.random.default_rng(seed + 2)
    b = [0.2 * rs.standard_normal(bb.shape) for bb in b]
    net = api.Net(ctx, torch.from_numpy(U).cuda(), L, layers, C, seed=3, tensor_cores=tc)
    net.set_params(api.pack_params(W, b))
    W32, b32 = api.unpack_params(net.get_params(), layers, C)   # the exact float32 values in use
    ref = onn.Net(U, W32, [bb.astype(float) for bb in b32], round_bf16=True, tc=tc)
    return th, U, net, ref


def _fields(L, nrhs, seed):
    rs = np.random.default_rng(seed)
    a = (rs.standard_normal((nrhs, L * L, 2)) + 1j * rs.standard_normal((nrhs, L * L, 2))).astype(np.complex64)
    return a


def test_forward_matches_oracle(api, ctx):
    """FP32 CUDA-core layers against the oracle with the same BF16 weights."""
    for C in (4, 8, 16):
        th, U, net, ref = _setup(api, ctx, L=16, C=C, layers=4, seed=C)
        assert net.format == 0
        r = _fields(16, 3, 7)
        y = net.forward(torch.from_numpy(r.reshape(3, -1)).cuda()).cpu().numpy().reshape(3, -1, 2)
        yr = ref.forward(r.astype(complex))
        assert np.abs(y - yr).max() < 2e-5 * np.abs(yr).max(), C
        net.close()


def _relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max()), float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,C,nrhs", [(16, 4, 3), (16, 8, 3), (16, 16, 3), (128, 16, 4), (128, 4, 2), (256, 8, 1)])
def test_tensor_core_forward_matches_oracle(api, ctx, L, C, nrhs):
    """tcgen05 layers (BF16 operands, FP32 accumulation) against the oracle in the same number format (layer
    inputs rounded to bfloat16).  The two round the same values to BF16 except where the FP32 and FP64 values
    fall on different sides of a rounding midpoint (a 2^-8 change of one input, about one element in 2^16),
    so the bound is 2e-3 of the largest output (4e-4 norm-wise) instead of FP32 rounding.  L = 16: gathered
    tiles (a tile spans several lattice rows).  L = 128 and 256: the hidden and last layers stage row segments
    by TMA (halo sites wrapped at both row ends at L = 128, interior at L = 256); 4 rhs at L = 128 give 512
    tiles, several per CTA, with the TMEM accumulator ring and the stage ring wrapping many times."""
    th, U, net, ref = _setup(api, ctx, L=L, C=C, layers=4, seed=C + L, tc=True)
    assert net.format == 1
    r = _fields(L, nrhs, 7 + L)
    y = net.forward(torch.from_numpy(r.reshape(nrhs, -1)).cuda()).cpu().numpy().reshape(nrhs, -1, 2)
    yr = ref.forward(r.astype(complex))
    emax, enorm = _relerr(y, yr)
    assert emax < 2e-3 and enorm < 4e-4, (emax, enorm)
    # and it is the tensor-core format, not the FP32 one: the exact-input oracle is further away
    y32 = onn.Net(U, ref.W, ref.b, round_bf16=False).forward(r.astype(complex))
    assert _relerr(y, y32)[1] > 4 * enorm
    net.close()


@pytest.mark.parametrize("L,nrhs", [(64, 8), (128, 2)])
def test_tensor_core_gradients_match_oracle(api, ctx, L, nrhs):
    """Loss and gradients of the tensor-core layers (input gradient by the gathered mixing with the
    conjugate-transposed weights, weight gradient as a tcgen05 GEMM over the sites) against the oracle's
    hand-derived backward in the same number format.  L = 64 with 8 rhs: 512 chunks of 64 sites for the
    weight gradient, several per CTA (the stage ring wraps and TMEM accumulates across chunks); L = 128: the
    row-segment staging in the forward and the input gradient."""
    C, layers = 16, 4
    th, U, net, ref = _setup(api, ctx, L=L, C=C, layers=layers, seed=41, tc=True)
    r = _fields(L, nrhs, 11)
    e = _fields(L, nrhs, 12)
    loss, g = net.loss_grad(torch.from_numpy(r.reshape(nrhs, -1)).cuda(), torch.from_numpy(e.reshape(nrhs, -1)).cuda())
    lref, gW, gb = ref.backward(r.astype(complex), e.astype(complex))
    assert abs(loss - lref) < 1e-4 * abs(lref)
    gref = api.pack_params(gW, gb).astype(np.float64)
    Wg, bg = api.unpack_params(g, layers, C)
    for l in range(layers):
        emax, enorm = _relerr(Wg[l], gW[l])
        assert emax < 5e-3 and enorm < 1e-3, (l, emax, enorm)
    for l in range(layers - 1):
        emax, enorm = _relerr(bg[l], gb[l])
        assert enorm < 1e-3, (l, emax, enorm)
    assert np.linalg.norm(g - gref) < 1e-3 * np.linalg.norm(gref)
    net.close()


def test_harvested_pairs(api, ctx):
    """nn_harvest_pairs: R = (zeta - D V zeta)/s, E = (D^{-1} zeta - V zeta)/s with s = |zeta - D V zeta|, for
    the Rademacher stream (seed, 0, PHASE_HARVEST, s).  Checked against the oracle operator: |R| = 1,
    D E = R to the solver tolerance, and R equal to the residual of the library's own FP32 V-cycle."""
    from oracle import rng as orng
    from oracle import schwinger as osch
    L, m0 = 32, -0.05
    U = gauge.links(gauge.field(L, 3.0, 2, sweeps=40))
    Ut = torch.from_numpy(U).cuda()
    h = api.mg_setup(ctx, Ut, L, m0)
    count, seed, s0 = 5, 3, 2
    R, E = api.nn_harvest_pairs(ctx, h, count, seed=seed, sample0=s0, tol=1e-6)
    R, E = R.cpu().numpy().astype(complex), E.cpu().numpy().astype(complex)
    D = osch.dirac_sparse(U, m0)
    assert np.allclose(np.linalg.norm(R, axis=1), 1.0, atol=1e-6)
    Z = np.ascontiguousarray(orng.rademacher_block(seed, 0, orng.PHASE_HARVEST, s0, h.n[0], count).T)
    v = torch.empty((count, h.n[0]), dtype=torch.complex64, device="cuda")
    h.vcycle(0, torch.from_numpy(Z.astype(np.complex64)).cuda(), v, api.FP32)
    r1 = Z - (D @ v.cpu().numpy().astype(complex).T).T
    s = np.linalg.norm(r1, axis=1)
    assert np.abs(r1 / s[:, None] - R).max() < 1e-5
    # D E - R = (D x - zeta) / s: the FP32 solve's residual, at most tol |zeta| / s (plus FP32 rounding)
    res = np.linalg.norm((D @ E.T).T - R, axis=1)
    bound = 1e-6 * np.linalg.norm(Z, axis=1) / s
    assert np.all(res < 1.5 * bound + 1e-6), (res, bound)
    assert np.linalg.norm(E, axis=1).min() > 1e-3
    h.close()


def test_gradients_match_oracle(api, ctx):
    L, C, layers = 16, 8, 4
    th, U, net, ref = _setup(api, ctx, L=L, C=C, layers=layers, seed=4)
    r = _fields(L, 4, 11)
    e = _fields(L, 4, 12)
    loss, g = net.loss_grad(torch.from_numpy(r.reshape(4, -1)).cuda(), torch.from_numpy(e.reshape(4, -1)).cuda())
    lref, gW, gb = ref.backward(r.astype(complex), e.astype(complex))
    assert abs(loss - lref) < 1e-5 * abs(lref)
    gref = api.pack_params(gW, gb).astype(np.float64)
    # the packed reference holds real and imaginary parts of dL/dconj... as dL/dRe + i dL/dIm
    assert np.abs(g - gref).max() < 2e-4 * np.abs(gref).max()
    net.close()


def test_gauge_covariance_on_gpu(api, ctx):
    L, C = 16, 4
    th, U, net, _ = _setup(api, ctx, L=L, C=C, seed=5)   # FP32 layers: covariant to rounding
    om = np.random.default_rng(1).uniform(-np.pi, np.pi, (L, L))
    Om = np.exp(1j * om).ravel()
    U2 = gauge.links(gauge.gauge_transform(th, om))
    net2 = api.Net(ctx, torch.from_numpy(U2).cuda(), L, 4, C, seed=3, tensor_cores=False)
    net2.set_params(net.get_params())
    r = _fields(L, 2, 3)
    y = net.forward(torch.from_numpy(r.reshape(2, -1)).cuda()).cpu().numpy().reshape(2, -1, 2)
    r2 = (Om[None, :, None] * r).astype(np.complex64)
    y2 = net2.forward(torch.from_numpy(r2.reshape(2, -1)).cuda()).cpu().numpy().reshape(2, -1, 2)
    assert np.abs(y2 - Om[None, :, None] * y).max() < 1e-5 * np.abs(y).max()
    net.close()
    net2.close()


def test_training_and_use_in_fgmres(api, ctx):
    """Pairs (r1, e1): r1 = zeta - D V(zeta), e1 = D^{-1} zeta - V(zeta) from the hierarchy's own V-cycle and
    solves; a few hundred Adam steps lower the loss, and the trained net used after the V-cycle (precond = 2)
    still converges to the FP64 tolerance.  Iteration counts with and without it are recorded."""
    L = 64
    U = torch.from_numpy(gauge.links(gauge.field(L, 3.0, 4, sweeps=60))).cuda()
    h = api.mg_setup(ctx, U, L, -0.08, ntv=8)
    net = api.Net(ctx, U, L, layers=4, channels=8, seed=2)
    n = h.n[0]

    def pairs(nr, seed):
        z = api.mgmlmc_rademacher(ctx, seed, 0, 0, 0, n, nr).to(torch.complex64)
        v = torch.empty_like(z)
        h.vcycle(0, z, v, api.FP32)
        r1 = torch.empty_like(z)
        h.apply(0, v, r1, api.FP32)
        r1 = z - r1
        x = torch.empty_like(z)
        api.fgmres_batched(ctx, h, 0, z, x, prec=api.FP32, tol=1e-6)
        s = torch.linalg.vector_norm(r1, dim=1, keepdim=True)   # the net sees unit-norm residuals
        return (r1 / s).contiguous(), ((x - v) / s).contiguous()

    r_tr, e_tr = pairs(32, 1)
    l0 = net.train_step(r_tr, e_tr, 2e-3)
    for it in range(300):
        l = net.train_step(r_tr, e_tr, 2e-3)
    r_te, e_te = pairs(16, 2)
    lt, _ = net.loss_grad(r_te, e_te)
    assert l < 0.9 * l0 and lt < 0.95 * l0
    net.attach(h)
    b = api.mgmlmc_rademacher(ctx, 9, 0, 0, 0, n, 16)
    x1, x2 = torch.empty_like(b), torch.empty_like(b)
    s1 = api.fgmres_batched(ctx, h, 0, b, x1, prec=api.MIXED, tol=1e-10, precond=1)
    s2 = api.fgmres_batched(ctx, h, 0, b, x2, prec=api.MIXED, tol=1e-10, precond=2, raise_on_nonconvergence=False)
    print("\n[learned correction] loss %.4f -> %.4f (held-out %.4f); FGMRES V-cycle %s ; V-cycle + net %s"
          % (l0, l, lt, {k: s1[k] for k in ("iters", "outer", "max_relres")},
             {k: s2[k] for k in ("iters", "outer", "max_relres")}))
    assert s1["converged"] and s2["converged"]
    assert s2["iters"] < s1["iters"]          # what the trained network gains over the V-cycle alone
    assert torch.abs(x1 - x2).max().item() < 1e-7 * torch.abs(x1).max().item()
    print("\n[learned correction] loss %.4f -> %.4f (held-out %.4f); FGMRES iterations V-cycle %d, "
          "V-cycle + net %d" % (l0, l, lt, s1["iters"], s2["iters"]))
    h.close()
    net.close()
