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
