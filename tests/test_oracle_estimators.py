"""Pins of the oracle's estimators: unbiasedness and the closed-form Rademacher
variance 1/2 ||offdiag(A + A^T)||_F^2 (Section 2) for Hutchinson, for the
MG-MLMC level differences (both forms) and for the Hutch++-deflated samples;
the Hutch++ trace split; CholeskyQR2 against Householder QR; the stop rule of
Algorithm 2 on hand-computed numbers; Algorithm 2 end to end against the
exact trace, statistically and in the full-sketch special case (d = n), where
it is exact."""
import math

import numpy as np
import pytest

from oracle import multigrid as mg
from oracle import rng
from oracle import schwinger as osch
from oracle.estimators import LevelDifference, hutchinson, mgmlmc_pp, update_active
from oracle.linalg import cholesky_qr2, qr_positive, trace_inverse_dense
from synthetic import gauge


def rad_var(M):
    """Variance of zeta^T M zeta for real Rademacher zeta (Section 2)."""
    S = M + M.T
    np.fill_diagonal(S, 0)
    return 0.5 * np.sum(np.abs(S) ** 2)


def sample_stats(M, nsamp, level=0, phase=rng.PHASE_STOCH, seed=3):
    n = M.shape[0]
    Z = np.stack([rng.rademacher(seed, level, phase, j, n) for j in range(nsamp)], axis=1)
    taus = np.einsum("is,ij,js->s", Z, M, Z)
    return taus.mean(), taus.var(ddof=1)


@pytest.fixture(scope="module")
def small():
    U = gauge.links(gauge.field(16, 3.0, 0))
    D = osch.dirac_sparse(U, -0.05)
    return D, mg.Hierarchy(D, 16, ntv=4, setup_sweeps=3, seed=2)


def test_hutchinson_mean_and_variance(small):
    D, _ = small
    A = np.linalg.inv(D.toarray())
    N = 6000
    mean, var = sample_stats(A, N)
    v = rad_var(A)
    assert abs(mean - np.trace(A)) < 4.5 * math.sqrt(v / N)
    assert abs(var / v - 1) < 0.08


def test_hutchinson_algorithm1_stop(small):
    D, _ = small
    A = np.linalg.inv(D.toarray())
    eps = 0.02
    tau, V, s, taus = hutchinson(lambda b: A @ b, A.shape[0], eps, seed=1)
    assert V / s <= (abs(tau) * eps) ** 2
    prev = taus[:-1]
    if len(prev) >= 2:   # it did not stop one sample earlier
        assert prev.var(ddof=1) / len(prev) > (abs(prev.mean()) * eps) ** 2
    assert abs(tau - np.trace(A)) < 5 * math.sqrt(V / s)


@pytest.mark.parametrize("form", ["accumulated", "reduced"])
def test_level_difference_unbiased(small, form):
    _, H = small
    ld = LevelDifference(H, form)
    M = ld.apply(0, np.eye(ld.vec_size(0)))
    tr_exact = np.trace(np.linalg.inv(H.D[0].toarray())) - np.trace(np.linalg.inv(H.D[1].toarray()))
    assert abs(np.trace(M) - tr_exact) < 1e-10 * abs(tr_exact)
    N = 5000
    mean, var = sample_stats(M, N, seed=9)
    v = rad_var(M)
    assert abs(mean - tr_exact) < 4.5 * math.sqrt(v / N)
    assert abs(var / v - 1) < 0.1


def test_hutchpp_split_and_deflated_variance(small):
    _, H = small
    ld = LevelDifference(H)
    n = ld.vec_size(0)
    A = ld.apply(0, np.eye(n))
    S = rng.rademacher_block(4, 0, rng.PHASE_SKETCH, 0, n, 16)
    Q, _ = qr_positive(ld.apply(0, ld.apply(0, S)))
    # exact split tr(A) = tr(Q^H A Q) + tr((I - QQ^H) A) for this (and any) orthonormal Q
    Pi = np.eye(n) - Q @ Q.conj().T
    assert abs(np.trace(Q.conj().T @ A @ Q) + np.trace(Pi @ A) - np.trace(A)) < 1e-11 * abs(np.trace(A))
    # projected samples z^H A zeta, z = (I - QQ^H) zeta, are zeta^T (Pi A) zeta
    M = Pi @ A
    N = 5000
    mean, var = sample_stats(M, N, seed=12)
    v = rad_var(M)
    assert abs(mean - np.trace(M)) < 4.5 * math.sqrt(v / N)
    assert abs(var / v - 1) < 0.1
    assert v < rad_var(A)      # the deflation reduced the variance


def test_cholesky_qr2_matches_householder():
    rs = np.random.default_rng(0)
    Y = rs.standard_normal((300, 12)) + 1j * rs.standard_normal((300, 12))
    Y[:, 3] = Y[:, 2] + 1e-5 * Y[:, 3]          # mildly ill-conditioned
    Q1, R1 = cholesky_qr2(Y)
    Q2, R2 = qr_positive(Y)
    assert np.abs(Q1.conj().T @ Q1 - np.eye(12)).max() < 1e-13
    assert np.abs(Q1 @ R1 - Y).max() < 1e-12 * np.abs(Y).max()
    assert np.abs(Q1 - Q2).max() < 1e-9
    assert np.all(np.diag(R2).real > 0) and np.abs(np.diag(R2).imag).max() < 1e-14


def test_stop_rule_hand_computed():
    # optimal: denom = sqrt(1*9) + sqrt(1*1) = 4 ; w = (3/4, 1/4); (eps tau)^2 = 1
    act = update_active([True, True], [9.0, 1.0], [10, 10], [1.0, 1.0], 0.1, 10.0, "optimal")
    assert act == [True, False]           # 0.9 > 0.75 ; 0.1 <= 0.25
    act = update_active([True, True], [7.0, 1.0], [10, 10], [1.0, 1.0], 0.1, 10.0, "optimal")
    assert act == [False, False]          # w0 = sqrt7/(sqrt7+1) = 0.7257 >= 0.7
    # costs enter as sqrt(C V): with C = (1, 1), w0 = sqrt(3.5)/(sqrt(3.5)+4) = 0.3187 < 0.35,
    # with C = (16, 1), w0 = sqrt(56)/(sqrt(56)+4) = 0.6517 >= 0.35
    act = update_active([True, True], [3.5, 16.0], [10, 10], [1.0, 1.0], 0.1, 10.0, "optimal")
    assert act == [True, True]            # level 1: w1 = 0.681 < 1.6
    act = update_active([True, True], [3.5, 16.0], [10, 10], [16.0, 1.0], 0.1, 10.0, "optimal")
    assert act == [False, True]
    # uniform: rho^2 = 1 / 2
    act = update_active([True, True], [9.0, 1.0], [10, 10], [1.0, 1.0], 0.1, 10.0, "uniform")
    assert act == [True, False]
    # the uniform split is over the L - 1 = 2 stochastic level differences, not over L = 3 levels:
    # V_0 / N_0 = 0.45 <= 1/2 stops level 0 (it would stay active against 1/3)
    act = update_active([True, True], [4.5, 1.0], [10, 10], [1.0, 1.0], 0.1, 10.0, "uniform")
    assert act == [False, False]
    # no decision before every level has a variance
    assert update_active([True, True], [0.0, 1.0], [1, 10], [1, 1], 0.1, 10.0) == [True, True]


@pytest.mark.parametrize("form", ["accumulated", "reduced"])
@pytest.mark.parametrize("noise", [rng.NOISE_RADEMACHER, rng.NOISE_Z4])
def test_full_sketch_gives_the_exact_trace(small, form, noise):
    """Special case of Algorithm 2 fixed by the mathematics: with a sketch as wide as the space (d = n), Q is
    unitary, every projected sample z^H A zeta has z = (I - QQ^H) zeta = 0, the low-rank part tr(Q^H A Q) is
    tr(A), and the estimate is the exact trace tr(D^{-1}) (dense inverse) with zero variance."""
    D, H = small
    ld = LevelDifference(H, form)
    n = ld.vec_size(0)
    r = mgmlmc_pp(ld, 1e-3, n, 1, seed=6, noise=noise)
    exact = trace_inverse_dense(D.toarray())
    assert abs(r["tau"] - exact) < 1e-10 * abs(exact)
    assert r["N"] == [2] and max(abs(t) for t in r["samples"][0]) < 1e-10 * abs(exact)
    assert abs(r["tau_lr"][0] - (exact - r["tau_L"])) < 1e-10 * abs(exact)


@pytest.mark.parametrize("d", [0, 8])
def test_algorithm2_end_to_end(small, d):
    D, H = small
    ld = LevelDifference(H)
    exact = trace_inverse_dense(D.toarray())
    eps = 0.01
    r = mgmlmc_pp(ld, eps, d, 2, seed=21)
    assert r["sigma"] <= eps * abs(r["tau"]) * 1.0000001
    assert abs(r["tau"] - exact) < 4.5 * r["sigma"]
    assert abs(r["tau"].imag) < 4.5 * r["sigma"]
    assert r["N"][0] >= 2


def z4_var(M):
    """Variance of zeta^H M zeta for Z4 zeta: ||offdiag(M)||_F^2 (Section 2)."""
    S = np.array(M, copy=True)
    np.fill_diagonal(S, 0)
    return np.sum(np.abs(S) ** 2)


def test_z4_hutchinson_mean_and_variance(small):
    D, _ = small
    A = np.linalg.inv(D.toarray())
    N = 6000
    Z = np.stack([rng.z4(3, 0, rng.PHASE_HUTCH, j, A.shape[0]) for j in range(N)], axis=1)
    taus = np.einsum("is,ij,js->s", np.conj(Z), A, Z)
    v = z4_var(A)
    assert abs(taus.mean() - np.trace(A)) < 4.5 * math.sqrt(v / N)
    assert abs(taus.var(ddof=1) / v - 1) < 0.08
    # the two formulas differ where A is far from symmetric: for an antisymmetric off-diagonal part the
    # real Rademacher samples are exact (variance 0) while Z4 samples keep ||offdiag(M)||_F^2
    rs = np.random.default_rng(1)
    K = rs.standard_normal((40, 40)) + 1j * rs.standard_normal((40, 40))
    M = K - K.T + np.diag(rs.standard_normal(40))
    Zr = np.stack([rng.rademacher(5, 0, rng.PHASE_HUTCH, j, 40) for j in range(2000)], axis=1)
    Zq = np.stack([rng.z4(5, 0, rng.PHASE_HUTCH, j, 40) for j in range(2000)], axis=1)
    tr_r = np.einsum("is,ij,js->s", Zr, M, Zr)
    tr_q = np.einsum("is,ij,js->s", np.conj(Zq), M, Zq)
    assert rad_var(M) < 1e-20 and np.abs(tr_r - np.trace(M)).max() < 1e-12
    assert abs(tr_q.var(ddof=1) / z4_var(M) - 1) < 0.1
    # Algorithm 1 with Z4 vectors
    tau, V, s, _ = hutchinson(lambda b: A @ b, A.shape[0], 0.02, seed=3, noise=rng.NOISE_Z4)
    assert V / s <= (abs(tau) * 0.02) ** 2 and abs(tau - np.trace(A)) < 5 * math.sqrt(V / s)


def test_gamma5_trace_properties():
    """tr(gamma5 D^{-1}) is real (gamma5 D is Hermitian by gamma5-hermiticity) and vanishes in the free
    field, where D^{-1}(p) = (a - i(sigma1 sin p_x + sigma2 sin p_t)) / (a^2 + b^2) is traceless against
    sigma3."""
    L = 8
    U = gauge.links(gauge.field(L, 3.0, 4, sweeps=30))
    D = osch.dirac_dense(U, -0.05)
    g5 = osch.gamma5(L).toarray()
    t = np.trace(g5 @ np.linalg.inv(D))
    assert abs(t.imag) < 1e-11 * max(1.0, abs(t)) and abs(t) > 1e-6
    D0 = osch.dirac_dense(np.ones((L, L, 2), dtype=complex), 0.3)
    assert abs(np.trace(g5 @ np.linalg.inv(D0))) < 1e-12


def test_gamma5_weighted_hutchinson(small):
    """Algorithm 1 for tr(gamma5 D^{-1}) (Section 1: traces after multiplication with a gamma matrix) with Z4
    vectors lands within 4.5 sigma of the dense trace, which is real and far from tr(D^{-1})."""
    D, _ = small
    A = np.linalg.inv(D.toarray())
    g5 = osch.gamma5(16).diagonal()
    exact = np.sum(g5 * np.diag(A))
    z = rng.noise(rng.NOISE_Z4, 3, 0, rng.PHASE_HUTCH, 0, 64)
    assert set(np.round(z, 12).tolist()) == {1, 1j, -1, -1j}       # kind Z4 draws fourth roots of unity
    tau, V, s, _ = hutchinson(lambda b: A @ b, A.shape[0], 0.5, seed=8, smax=600, noise=rng.NOISE_Z4, weight=g5)
    assert abs(tau - exact) < 4.5 * math.sqrt(V / s)
    assert abs(exact - np.trace(A)) > 20 * math.sqrt(V / s)


@pytest.mark.parametrize("form", ["accumulated", "reduced"])
def test_gamma5_telescoping_and_unbiased(small3_g5, form):
    """With gamma5 weighting the exact level traces telescope to tr(gamma5 D^{-1}) (the gamma5 signs of the
    fine and coarse levels agree through the chirality-preserving aggregation), and the projected
    Algorithm 2 estimate (Z4 vectors) lands within 4.5 sigma of it."""
    H = small3_g5
    ld = LevelDifference(H, form, gamma5=True)
    diffs, tL = ld.exact_traces()
    exact = np.trace(osch.gamma5(32).toarray() @ np.linalg.inv(H.D[0].toarray()))
    assert abs(sum(diffs) + tL - exact) < 1e-9 * abs(exact)
    # tr(gamma5 D^{-1}) is small against the sample spread, so the relative target is loose and capped
    r = mgmlmc_pp(ld, 0.5, 6, 2, seed=5, noise=rng.NOISE_Z4, max_samples=600)
    assert abs(r["tau"] - exact) < 4.5 * r["sigma"]
    assert r["sigma"] <= 0.5 * abs(r["tau"]) * 1.0000001 or max(r["N"]) == 600


@pytest.fixture(scope="module")
def small3_g5():
    U = gauge.links(gauge.field(32, 3.0, 3, sweeps=40))
    return mg.Hierarchy(osch.dirac_sparse(U, -0.05), 32, levels=3, agg=2, ntv=2, setup_sweeps=2, seed=1)
