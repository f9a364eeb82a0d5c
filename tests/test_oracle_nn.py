"""Pins of the oracle's gauge-covariant preconditioner network: its explicit
backward pass against central finite differences of its forward pass, gauge
covariance (M(Omega r; U^Omega) = Omega M(r; U)), the transporter identity
T_d(x) -> Omega(x) T_d(x) conj(Omega(x + d)), and bfloat16 rounding on known
values."""
import numpy as np
import pytest

from oracle import nn as onn
from synthetic import gauge


def small_net(L=8, C=3, layers=3, seed=0, round_bf16=False):
    th = gauge.quenched_u1(L, 3.0, 10, seed)
    W, b = onn.init_params(C, layers, seed + 1)
    b = [bb + 0.3 * np.random.default_rng(seed + 2).standard_normal(bb.shape) for bb in b]
    return th, W, b, onn.Net(gauge.links(th), W, b, round_bf16=round_bf16)


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.00390625, 1.005859375, np.pi, 0.1, -2.5])
    want = np.array([1.0, 1.0, 1.0078125, 3.140625, 0.10009765625, -2.5])
    assert np.array_equal(onn.bf16_round(vals), want)


def test_backward_matches_finite_differences():
    th, W, b, net = small_net()
    rs = np.random.default_rng(5)
    V = net.L ** 2
    r = rs.standard_normal((2, V, 2)) + 1j * rs.standard_normal((2, V, 2))
    e = rs.standard_normal((2, V, 2)) + 1j * rs.standard_normal((2, V, 2))
    L0, gW, gb = net.backward(r, e)
    h = 1e-6
    for l, (d, k, c) in [(0, (4, 1, 0)), (1, (0, 2, 2)), (2, (8, 1, 1)), (1, (5, 0, 1))]:
        for part in (1.0, 1j):
            net.W[l][d, k, c] += h * part
            Lp, _ = net.loss(r, e)
            net.W[l][d, k, c] -= 2 * h * part
            Lm, _ = net.loss(r, e)
            net.W[l][d, k, c] += h * part
            fd = (Lp - Lm) / (2 * h)
            an = gW[l][d, k, c].real if part == 1.0 else gW[l][d, k, c].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (l, d, k, c, part, fd, an)
    for l, k in [(0, 1), (1, 2)]:
        net.b[l][k] += h
        Lp, _ = net.loss(r, e)
        net.b[l][k] -= 2 * h
        Lm, _ = net.loss(r, e)
        net.b[l][k] += h
        assert abs((Lp - Lm) / (2 * h) - gb[l][k]) < 1e-6 * max(1.0, abs(gb[l][k]))


def test_gauge_covariance():
    th, W, b, net = small_net(round_bf16=True)
    L = net.L
    om = np.random.default_rng(9).uniform(-np.pi, np.pi, (L, L))
    Om = np.exp(1j * om).ravel()
    th2 = gauge.gauge_transform(th, om)
    net2 = onn.Net(gauge.links(th2), W, b, round_bf16=True)
    nb = onn.neighbour_index(L)
    assert np.abs(net2.T - Om[:, None] * net.T * np.conj(Om[nb])).max() < 1e-13
    rs = np.random.default_rng(3)
    r = rs.standard_normal((2, L * L, 2)) + 1j * rs.standard_normal((2, L * L, 2))
    y = net.forward(r)
    y2 = net2.forward(Om[None, :, None] * r)
    assert np.abs(y2 - Om[None, :, None] * y).max() < 1e-12 * np.abs(y).max()


def test_transport_of_constant_field_is_trivial():
    L = 6
    net = onn.Net(np.ones((L, L, 2), complex), *onn.init_params(2, 2, 0), round_bf16=False)
    T = net.T.reshape(L, L, 9)
    # unit links: only the t-boundary crossings carry -1
    for d, (dx, dt) in enumerate(onn.OFFSETS):
        want = np.ones((L, L))
        if dt == 1:
            want[L - 1, :] = -1
        if dt == -1:
            want[0, :] = -1
        assert np.allclose(T[:, :, d], want)


def test_reversed_path_identity():
    """conj(T_d(y - d)) = T_(-d)(y) for every site and offset, to FP64 rounding: the transporter of a reversed
    path (the two L-shaped paths of a diagonal reversed together), which turns the adjoint scatter of the input
    gradient into a gathered mixing."""
    th, W, b, net = small_net(L=8)
    L = net.L
    T, nb = net.T, net.nb
    for d, (dx, dt) in enumerate(onn.OFFSETS):
        md = onn.OFFSETS.index((-dx, -dt))
        assert md == 8 - d
        src = nb[:, md]                        # y - d for every y
        assert np.abs(np.conj(T[src, d]) - T[:, md]).max() < 1e-15, d
    # the averaging of the two paths matters: one L-shaped path alone does not satisfy it on a random field
    U = gauge.links(th)
    one = U[..., 0] * np.roll(U[..., 1], -1, axis=1)        # T_(+1,+1) via x then t only
    back = np.conj(np.roll(np.roll(one, 1, axis=0), 1, axis=1))
    assert not np.allclose(back.ravel(), T[:, 0])


def test_input_gradient_as_gathered_mixing():
    """sum over d of conj(T_d(x)) (conj(W_d)^T gz(x)) scattered to x + d equals the gather
    sum_e T_e(y) conj(W_(8-e))^T gz(y + e) (the form of the library's tensor-core backward)."""
    th, W, b, net = small_net(L=8, C=3)
    rs = np.random.default_rng(3)
    V = net.L ** 2
    Wl = net.W[1]                                                   # [9, c_out, c_in]
    gz = rs.standard_normal((2, V, 3)) + 1j * rs.standard_normal((2, V, 3))
    gu = np.einsum("dkc,rxk->rxdc", np.conj(Wl), gz)
    ga = np.zeros((2, V, 3), complex)
    for d in range(9):
        np.add.at(ga, (slice(None), net.nb[:, d], slice(None)), np.conj(net.T)[None, :, d, None] * gu[:, :, d, :])
    gg = np.zeros_like(ga)
    for e in range(9):
        Be = np.conj(Wl[8 - e]).T                                   # [c_in, c_out]
        gg += net.T[None, :, e, None] * np.einsum("ck,rxk->rxc", Be, gz[:, net.nb[:, e], :])
    assert np.abs(ga - gg).max() < 1e-12 * np.abs(ga).max()


def test_tensor_core_format_within_bf16_bounds():
    """The tensor-core number format against the exact network: rounding each layer input to bfloat16 (8
    significant bits, relative error <= 2^-9 per part) moves the output by a few 2^-9 (norm-wise); rounding
    gz and u in the backward moves the gradients by a similar amount.  Both stay far from the exact values'
    scale, and the loss agrees to a few 2^-9."""
    th, W, b, exact = small_net(L=8, C=4, layers=4, round_bf16=True)
    tc = onn.Net(gauge.links(th), W, b, round_bf16=True, tc=True)
    rs = np.random.default_rng(6)
    V = exact.L ** 2
    r = rs.standard_normal((2, V, 2)) + 1j * rs.standard_normal((2, V, 2))
    e = rs.standard_normal((2, V, 2)) + 1j * rs.standard_normal((2, V, 2))
    y0, y1 = exact.forward(r), tc.forward(r)
    rel = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    assert 1e-5 < rel < 8 * 2.0 ** -9, rel          # it does round, and within the bound
    L0, gW0, gb0 = exact.backward(r, e)
    L1, gW1, gb1 = tc.backward(r, e)
    assert abs(L1 - L0) < 8 * 2.0 ** -9 * abs(L0)
    for l in range(4):
        relg = np.linalg.norm(gW1[l] - gW0[l]) / np.linalg.norm(gW0[l])
        assert 1e-6 < relg < 16 * 2.0 ** -9, (l, relg)
    for l in range(3):
        assert np.linalg.norm(gb1[l] - gb0[l]) < 16 * 2.0 ** -9 * np.linalg.norm(gb0[l])
