"""Pins of the oracle's multigrid hierarchy: orthonormal aggregation
prolongators (R = P^H, P^H P = I, Section 3.1), their sparsity, the Galerkin
definition D_{l+1} = R_l D_l P_l, gamma5-structure of the coarse operators,
the SAP smoother's defining property, and the telescoping identity of
eq. mlmc_decomp_trace."""
import numpy as np
import pytest

from oracle import multigrid as mg
from oracle import schwinger as osch
from oracle.linalg import trace_inverse_dense
from synthetic import gauge


@pytest.fixture(scope="module")
def hier():
    U = gauge.links(gauge.field(64, 3.0, 0, sweeps=40))
    D = osch.dirac_sparse(U, -0.05)
    return mg.Hierarchy(D, 64, ntv=4, setup_sweeps=3, seed=5)


def test_level_rule():
    assert [mg.default_levels(L) for L in (16, 32, 64, 128, 256, 512, 1024)] == [2, 2, 3, 3, 4, 4, 5]


def test_sizes(hier):
    assert hier.levels == 3
    assert hier.n == [2 * 64 * 64, 8 * 16 * 16, 8 * 4 * 4]


def test_orthonormal_and_aggregate_support(hier):
    for l, P in enumerate(hier.P):
        PhP = (P.conj().T @ P).toarray()
        assert np.abs(PhP - np.eye(P.shape[1])).max() < 1e-13
        Ls, d = hier.side[l], hier.dof[l]
        Lc, dc = Ls // 4, hier.dof[l + 1]
        Pc = P.tocoo()
        fs = Pc.row // d
        fk = Pc.row % d
        cs = Pc.col // dc
        ck = Pc.col % dc
        ft, fx = fs // Ls, fs % Ls
        ct, cx = cs // Lc, cs % Lc
        assert np.all(ft // 4 == ct) and np.all(fx // 4 == cx)           # aggregate support
        assert np.all(mg.chirality(fk, d) == mg.chirality(ck, dc))      # chirality blocks


@pytest.fixture(scope="module")
def small3():
    """A 3-level hierarchy small enough for dense checks (2x2 aggregates)."""
    U = gauge.links(gauge.field(32, 3.0, 3, sweeps=40))
    return mg.Hierarchy(osch.dirac_sparse(U, -0.05), 32, levels=3, agg=2, ntv=2,
                        setup_sweeps=2, seed=1)


def test_galerkin_dense(small3):
    for l in range(small3.levels - 1):
        P, D = small3.P[l].toarray(), small3.D[l].toarray()
        assert np.abs(P.conj().T @ D @ P - small3.D[l + 1].toarray()).max() < 1e-13


def test_galerkin_on_vectors(hier):
    rng = np.random.default_rng(2)
    for l in range(hier.levels - 1):
        x = rng.standard_normal((hier.n[l + 1], 3)) + 1j * rng.standard_normal((hier.n[l + 1], 3))
        P = hier.P[l]
        ref = P.conj().T @ (hier.D[l] @ (P @ x))
        assert np.abs(hier.D[l + 1] @ x - ref).max() < 1e-12 * np.abs(ref).max()


def test_gamma5_coarse(hier):
    for l in range(hier.levels):
        g5 = hier.gamma5(l)
        Dl = hier.D[l]
        assert abs(g5 @ Dl @ g5 - Dl.conj().T).max() < 1e-13
        assert np.allclose(g5.diagonal() ** 2, 1.0)


def test_coarse_operator_is_nearest_neighbour(hier):
    Dc = hier.D[1]
    S = mg.stencil_blocks(Dc, hier.side[1], hier.dof[1])
    rebuilt = sum(np.abs(S[..., k, :, :]).sum() for k in range(5))
    assert abs(rebuilt - np.abs(Dc).sum()) < 1e-9 * np.abs(Dc).sum()


def test_sap_residual_vanishes_on_updated_colour():
    L = 16
    U = gauge.links(gauge.field(L, 3.0, 1, sweeps=30))
    D = osch.dirac_sparse(U, 0.1)
    sap = mg.SAP(D, L, 2, 4)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    x = np.zeros_like(f)
    for c, (I, inv) in enumerate(sap.sets):
        r = f - D @ x
        x[I] += np.einsum("bij,bj->bi", inv, r[I])
        assert np.abs((f - D @ x)[I]).max() < 1e-12
    # the class's sweep is exactly these two half steps
    x2 = sap.sweep(f, np.zeros_like(f))
    assert np.abs(x2 - x).max() < 1e-14
    # fixed point: the exact solution is not moved
    xs = np.linalg.solve(D.toarray(), f)
    assert np.abs(sap.sweep(f, xs.copy()) - xs).max() < 1e-11
    # and iterating converges to it
    y = np.zeros_like(f)
    for _ in range(60):
        sap.sweep(f, y)
    assert np.linalg.norm(y - xs) < 1e-8 * np.linalg.norm(xs)


def test_coarse_sap_blocks():
    U = gauge.links(gauge.field(32, 3.0, 2, sweeps=30))
    H = mg.Hierarchy(osch.dirac_sparse(U, 0.1), 32, ntv=2, setup_sweeps=1)
    sap = mg.SAP(H.D[1], H.side[1], H.dof[1], 2)
    f = np.random.default_rng(1).standard_normal(H.n[1]).astype(complex)
    x = np.zeros_like(f)
    I0, inv0 = sap.sets[0]
    x[I0] += np.einsum("bij,bj->bi", inv0, f[I0])
    assert np.abs((f - H.D[1] @ x)[I0]).max() < 1e-12


def test_telescoping_sum_equals_trace(small3):
    from oracle.estimators import LevelDifference
    for form in ("accumulated", "reduced"):
        ld = LevelDifference(small3, form)
        # traces of the level differences from their explicit matrices
        diffs = [complex(np.trace(ld.apply(l, np.eye(ld.vec_size(l))))) for l in range(2)]
        tL = complex(np.trace(np.linalg.inv(small3.D[2].toarray())))
        total = sum(diffs) + tL
        assert abs(total - trace_inverse_dense(small3.D[0].toarray())) < 1e-10 * abs(total)


def _sap_iteration_matrix(sap, n):
    """I - M D of one SAP sweep, built from the block inverses as dense matrices (the two colours in order)."""
    D = sap.D.toarray()
    S = np.eye(n, dtype=complex)
    for I, inv in sap.sets:
        M = np.zeros((n, n), dtype=complex)
        for b in range(len(I)):
            M[np.ix_(I[b], I[b])] = inv[b]
        S = (np.eye(n) - M @ D) @ S
    return S


def test_vcycle_two_level_without_smoothing_is_coarse_correction(small3):
    """V(0,0) on a two-level hierarchy is the coarse-grid correction P D_c^{-1} P^H exactly."""
    H = mg.Hierarchy.from_prolongators(small3.D[0], 32, small3.P[:1], agg=2, sap_block=(4, 2))
    P, Dc = H.P[0].toarray(), H.D[1].toarray()
    r = np.random.default_rng(4).standard_normal((H.n[0], 2)) + 0j
    ref = P @ np.linalg.solve(Dc, P.conj().T @ r)
    assert np.abs(H.vcycle(0, r, 0, 0) - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("pre,post", [(1, 1), (2, 1)])
def test_vcycle_error_propagator(small3, pre, post):
    """Three-level V(pre, post) cycle: with B_l the cycle as a linear map, the error propagator
    I - B_l D_l equals S^post (I - P_l B_{l+1} P_l^H D_l) S^pre, S the SAP sweep's iteration matrix,
    and B_L = D_L^{-1} on the coarsest level (built from dense blocks, independent of vcycle)."""
    H = mg.Hierarchy.from_prolongators(small3.D[0], 32, small3.P, agg=2, sap_block=(4, 2))
    B = [None] * H.levels
    B[-1] = np.linalg.inv(H.D[-1].toarray())
    for l in range(H.levels - 2, -1, -1):
        n = H.n[l]
        S = _sap_iteration_matrix(H.sap(l), n)
        P, D = H.P[l].toarray(), H.D[l].toarray()
        C = np.eye(n) - P @ B[l + 1] @ P.conj().T @ D
        E = np.linalg.matrix_power(S, post) @ C @ np.linalg.matrix_power(S, pre)
        B[l] = (np.eye(n) - E) @ np.linalg.inv(D)
    r = np.random.default_rng(5).standard_normal((H.n[0], 3)) + 1j * np.random.default_rng(6).standard_normal(
        (H.n[0], 3))
    got = H.vcycle(0, r, pre, post)
    ref = B[0] @ r
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    # the cycle contracts the error of the fine system
    D0 = H.D[0].toarray()
    assert np.linalg.norm(np.eye(H.n[0]) - B[0] @ D0, 2) < 1.0


def test_imported_prolongators_rebuild_the_hierarchy(hier):
    """from_prolongators with the oracle's own P gives back its Galerkin operators; check_prolongator
    accepts them; the GPU block layout round-trips; a row moved into another aggregate is caught."""
    H2 = mg.Hierarchy.from_prolongators(hier.D[0], 64, hier.P, agg=4)
    for l in range(hier.levels):
        assert abs(H2.D[l] - hier.D[l]).max() < 1e-13
    for l, P in enumerate(hier.P):
        c = mg.check_prolongator(P, hier.side[l], hier.dof[l], 4)
        assert c["orth"] < 1e-13 and c["support"] and c["chirality"]
        Ls, d, Lc = hier.side[l], hier.dof[l], hier.side[l + 1]
        ntv = hier.dof[l + 1] // 2
        blocks = mg.aggregate_blocks(Ls, d, 4)
        Pr = P.tocsr()
        B = np.empty((Lc * Lc, 2, blocks.shape[-1], ntv), dtype=complex)
        for T in range(Lc):
            for X in range(Lc):
                for ch in range(2):
                    cols = (T * Lc + X) * 2 * ntv + ch * ntv + np.arange(ntv)
                    B[T * Lc + X, ch] = Pr[blocks[X, T, ch]][:, cols].toarray()
        assert abs(mg.prolongator_from_blocks(B, Ls, d, 4, ntv) - P).max() == 0
    # planted mistake: swap one fine row of aggregate (0, 0) with a row of aggregate (1, 0)
    P = hier.P[0].tolil()
    i, j = 0, 2 * 4 + 0          # fine dof of site (0,0) and of site (4,0)
    ri, rj = P.getrow(i).copy(), P.getrow(j).copy()
    P[i, :] = rj
    P[j, :] = ri
    assert not mg.check_prolongator(P.tocsr(), 64, 2, 4)["support"]
    # planted mistake: swap the two spin rows (chiralities) of fine site (0, 0): same aggregate, wrong chirality
    P = hier.P[0].tolil()
    r0, r1 = P.getrow(0).copy(), P.getrow(1).copy()
    P[0, :] = r1
    P[1, :] = r0
    c = mg.check_prolongator(P.tocsr(), 64, 2, 4)
    assert c["support"] and not c["chirality"]
    # planted mistake: one column scaled by 1.1 is no longer orthonormal (|P^H P - I| = 0.21 on its diagonal)
    P = hier.P[0].tocsc(copy=True)
    P[:, 3] = P[:, 3] * 1.1
    assert abs(mg.check_prolongator(P.tocsr(), 64, 2, 4)["orth"] - 0.21) < 1e-12


def test_stencil_blocks_direction_convention():
    """stencil_blocks on the fine operator gives the hop blocks of the Wilson formula: S[+x] = -1/2 (1 - sigma_1)
    U_0(x), S[-x] = -1/2 (1 + sigma_1) conj(U_0(x - x^)), S[+t] with the antiperiodic sign on the last time slice."""
    L = 8
    U = gauge.links(gauge.field(L, 3.0, 2, sweeps=20))
    S = mg.stencil_blocks(osch.dirac_sparse(U, 0.1), L, 2)
    e, s1, s2 = np.eye(2), osch.SIGMA[0], osch.SIGMA[1]
    T, X = 3, 5
    assert np.abs(S[T, X, 0] - 2.1 * e).max() < 1e-15
    assert np.abs(S[T, X, 1] + 0.5 * (e - s1) * U[T, X, 0]).max() < 1e-15
    assert np.abs(S[T, X, 2] + 0.5 * (e + s1) * np.conj(U[T, X - 1, 0])).max() < 1e-15
    assert np.abs(S[T, X, 3] + 0.5 * (e - s2) * U[T, X, 1]).max() < 1e-15
    assert np.abs(S[T, X, 4] + 0.5 * (e + s2) * np.conj(U[T - 1, X, 1])).max() < 1e-15
    assert np.abs(S[L - 1, X, 3] - 0.5 * (e - s2) * U[L - 1, X, 1]).max() < 1e-15


def test_sparse_from_stencil_round_trip(hier):
    for l in range(1, hier.levels):
        S = mg.stencil_blocks(hier.D[l], hier.side[l], hier.dof[l])
        back = mg.sparse_from_stencil(S.reshape(-1, 5, hier.dof[l], hier.dof[l]), hier.side[l], hier.dof[l])
        assert abs(back - hier.D[l]).max() < 1e-15 * abs(hier.D[l]).max()
