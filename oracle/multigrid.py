"""Aggregation multigrid hierarchy, oracle form (FP64, scipy.sparse).

The paper builds its hierarchy "with a bootstrap setup and aggregation based
prolongations as in DD-alpha-AMG" (Section 4) and uses R_l = P_l^H with
orthonormal columns, D_{l+1} = R_l D_l P_l (Section 3, eq. mlmc_decomp_matrix
and the text before eq. mlmc_dec_trace_reduced).  It does not print the
set-up.  The set-up written here is this library's reading of it, and the
CUDA path implements the same definition:

Geometry of level l: side L_l, d_l dof per site (2 on the fine level,
2 * ntv on coarse levels), n_l = L_l^2 d_l, dof index (t * L_l + x) * d_l + k.
Chirality of dof k: the fine spin index (gamma5 = sigma_3); on coarse levels
k < ntv is chirality 0 and k >= ntv chirality 1.

Test vectors: ntv complex Rademacher vectors on level l (stream level = l,
phase TESTVEC, sample = m), each smoothed by `setup_sweeps` SAP sweeps for
D_l v = 0 (the initial phase of the DD-alpha-AMG bootstrap set-up).

Aggregates: agg x agg site blocks; in aggregate (X, T) and chirality c the
block of the test vectors is ordered by local site j = (t - agg T) * agg +
(x - agg X) and then by the dof of chirality c at that site.  Each such block
(bs x ntv) is orthonormalised with a QR whose R has a real positive
diagonal; column m becomes coarse dof c * ntv + m of coarse site (X, T).

SAP (Schwarz alternating procedure): blocks of b x b sites, block colour
(BX + BT) mod 2; one sweep for D x = f updates all colour-0 blocks, then all
colour-1 blocks, each by x_B += D_BB^{-1} (f - D x)_B with the exact inverse
of the diagonal block.

Galerkin coarse operator D_{l+1} = P_l^H D_l P_l.

V-cycle (the multigrid solver of Section 4, "done via multigrid"): on level
l < L-1, e = 0; pre_smooth SAP sweeps for D_l e = r; coarse correction
e += P_l V_{l+1}(P_l^H (r - D_l e)); post_smooth SAP sweeps; on the coarsest
level e = D_L^{-1} r exactly.

A hierarchy whose prolongators come from elsewhere (the GPU's adaptive
bootstrap set-up, which has many valid outcomes) is rebuilt from them by
Hierarchy.from_prolongators: the oracle then forms its own Galerkin operators
P^H D P from its own fine operator, and check_prolongator verifies the
defining properties of P (orthonormal columns, aggregate and chirality
support).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import rng
from .linalg import qr_positive


def default_levels(L: int, agg: int = 4) -> int:
    """Coarsen while the side exceeds 8 and the coarse side stays a multiple of 4."""
    lv, side = 1, L
    while side > 8 and side % (4 * agg) == 0:
        side //= agg
        lv += 1
    return lv


def chirality(k: np.ndarray, d: int) -> np.ndarray:
    if d == 2:
        return k
    return (k >= d // 2).astype(int)


def block_indices(Ls: int, d: int, b: int):
    """For each b x b block: colour and its dof indices (block-local order).

    Returns (colors[nb], idx[nb, b*b*d]).  Block order: BT slow, BX fast.
    """
    nbs = Ls // b
    colors, idx = [], []
    jt, jx = np.meshgrid(np.arange(b), np.arange(b), indexing="ij")
    jt = jt.ravel()
    jx = jx.ravel()
    k = np.arange(d)
    for BT in range(nbs):
        for BX in range(nbs):
            sites = (b * BT + jt) * Ls + (b * BX + jx)
            idx.append((sites[:, None] * d + k[None, :]).ravel())
            colors.append((BX + BT) % 2)
    return np.array(colors), np.array(idx)


class SAP:
    """Red-black block Schwarz smoother with exact block inverses."""

    def __init__(self, D: sp.csr_matrix, Ls: int, d: int, b: int):
        if Ls % b or (Ls // b) % 2:
            raise ValueError("SAP needs L/b even")
        self.D = D
        colors, idx = block_indices(Ls, d, b)
        Dd = D.tocsr()
        self.sets = []
        for c in (0, 1):
            I = idx[colors == c]
            inv = np.stack([np.linalg.inv(Dd[i][:, i].toarray()) for i in I])
            self.sets.append((I, inv))

    def sweep(self, f: np.ndarray, x: np.ndarray) -> np.ndarray:
        """One sweep for D x = f (x updated in place and returned).  f, x: (n,) or (n, k)."""
        for I, inv in self.sets:
            r = f - self.D @ x
            if x.ndim == 1:
                x[I] += np.einsum("bij,bj->bi", inv, r[I])
            else:
                x[I] += np.einsum("bij,bjk->bik", inv, r[I])
        return x


def aggregate_blocks(Ls: int, d: int, agg: int):
    """idx[X, T, c] -> fine dof indices of aggregate (X, T), chirality c, in block order."""
    Lc = Ls // agg
    dc = d // 2
    jt, jx = np.meshgrid(np.arange(agg), np.arange(agg), indexing="ij")
    jt = jt.ravel()
    jx = jx.ravel()
    out = np.empty((Lc, Lc, 2, agg * agg * dc), dtype=np.int64)
    for T in range(Lc):
        for X in range(Lc):
            sites = (agg * T + jt) * Ls + (agg * X + jx)
            for c in range(2):
                ks = np.arange(dc) + c * dc if d > 2 else np.array([c])
                out[X, T, c] = (sites[:, None] * d + ks[None, :]).ravel()
    return out


def prolongator(V: np.ndarray, Ls: int, d: int, agg: int, ntv: int) -> sp.csr_matrix:
    """Orthonormal aggregation prolongator from test vectors V (n_l x ntv)."""
    Lc = Ls // agg
    dcoarse = 2 * ntv
    blocks = aggregate_blocks(Ls, d, agg)
    rows, cols, vals = [], [], []
    for T in range(Lc):
        for X in range(Lc):
            for c in range(2):
                I = blocks[X, T, c]
                Q, _ = qr_positive(V[I, :])
                base = (T * Lc + X) * dcoarse + c * ntv
                for m in range(ntv):
                    rows.append(I)
                    cols.append(np.full(I.size, base + m))
                    vals.append(Q[:, m])
    n = Ls * Ls * d
    nc = Lc * Lc * dcoarse
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, nc)).tocsr()


def prolongator_from_blocks(B: np.ndarray, Ls: int, d: int, agg: int, ntv: int) -> sp.csr_matrix:
    """Sparse P (n_l x n_{l+1}) from its aggregate blocks B[T*Lc+X, c, j, m] (row j of block (X, T, c)
    is the j-th fine dof of aggregate_blocks, column m is coarse dof c*ntv+m of coarse site (X, T))."""
    Lc = Ls // agg
    dcoarse = 2 * ntv
    blocks = aggregate_blocks(Ls, d, agg)
    rows, cols, vals = [], [], []
    for T in range(Lc):
        for X in range(Lc):
            for c in range(2):
                I = blocks[X, T, c]
                base = (T * Lc + X) * dcoarse + c * ntv
                for m in range(ntv):
                    rows.append(I)
                    cols.append(np.full(I.size, base + m))
                    vals.append(B[T * Lc + X, c, :, m])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Ls * Ls * d, Lc * Lc * dcoarse)).tocsr()


def check_prolongator(P: sp.spmatrix, Ls: int, d: int, agg: int) -> dict:
    """Defining properties of an aggregation prolongator (Section 3.1): max |P^H P - I| and whether every
    non-zero joins a fine dof to a coarse dof of its own aggregate and of its own chirality."""
    Pc = P.tocoo()
    dc = P.shape[1] // ((Ls // agg) ** 2)
    Lc = Ls // agg
    G = (P.conj().T @ P - sp.identity(P.shape[1], dtype=complex, format="csr")).tocsr()  # sparse: blocks
    orth = float(np.abs(G.data).max()) if G.nnz else 0.0
    fs, fk = Pc.row // d, Pc.row % d
    cs, ck = Pc.col // dc, Pc.col % dc
    ft, fx, ct, cx = fs // Ls, fs % Ls, cs // Lc, cs % Lc
    support = bool(np.all(ft // agg == ct) and np.all(fx // agg == cx))
    chiral = bool(np.all(chirality(fk, d) == chirality(ck, dc)))
    return dict(orth=orth, support=support, chirality=chiral)


def stencil_blocks(Dl: sp.spmatrix, Ls: int, d: int) -> np.ndarray:
    """Blocks of a nearest-neighbour level operator: S[T, X, dir, d, d],
    dir = 0 self, 1 +x, 2 -x, 3 +t, 4 -t; S[B, dir] = D[rows of B, cols of B+dir]."""
    Dd = Dl.tocsr()
    S = np.zeros((Ls, Ls, 5, d, d), dtype=complex)
    k = np.arange(d)
    for T in range(Ls):
        for X in range(Ls):
            r = (T * Ls + X) * d + k
            for di, (dx, dt) in enumerate(((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1))):
                s2 = ((T + dt) % Ls) * Ls + (X + dx) % Ls
                S[T, X, di] = Dd[r][:, s2 * d + k].toarray()
    return S


def sparse_from_stencil(S: np.ndarray, Ls: int, d: int) -> sp.csr_matrix:
    """The level operator from its blocks (inverse of stencil_blocks): S[site T*Ls+X, dir, d, d], dir = self,
    +x, -x, +t, -t, block (s, dir) = D[rows of s, cols of s+dir]; coinciding neighbours add up."""
    S = np.asarray(S).reshape(Ls * Ls, 5, d, d)
    s = np.arange(Ls * Ls)
    T, X = s // Ls, s % Ls
    nbr = [s, T * Ls + (X + 1) % Ls, T * Ls + (X - 1) % Ls, ((T + 1) % Ls) * Ls + X, ((T - 1) % Ls) * Ls + X]
    i, j = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    rows, cols, vals = [], [], []
    for di in range(5):
        rows.append((s[:, None, None] * d + i[None]).ravel())
        cols.append((nbr[di][:, None, None] * d + j[None]).ravel())
        vals.append(S[:, di].ravel())
    n = Ls * Ls * d
    D = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    D.sum_duplicates()
    return D


class Hierarchy:
    """Levels 0..nlev-1 (level 0 = fine).  D[l], P[l] (l < nlev-1), side[l], dof[l]."""

    def __init__(self, D0: sp.csr_matrix, L: int, levels: int | None = None, agg: int = 4,
                 ntv: int = 8, sap_block=(4, 2), setup_sweeps: int = 4, seed: int = 0):
        self.levels = levels or default_levels(L, agg)
        self.agg, self.ntv = agg, ntv
        self.D = [sp.csr_matrix(D0)]
        self.P = []
        self.side = [L]
        self.dof = [2]
        for l in range(self.levels - 1):
            Ls, d = self.side[l], self.dof[l]
            if Ls % agg or (Ls // agg) < 4:
                raise ValueError("level %d side %d cannot be aggregated" % (l, Ls))
            n = Ls * Ls * d
            b = sap_block[0] if l == 0 else sap_block[1]
            V = np.stack([rng.complex_rademacher(seed, l, rng.PHASE_TESTVEC, m, n)
                          for m in range(ntv)], axis=1)
            if setup_sweeps:
                sap = SAP(self.D[l], Ls, d, b)
                f = np.zeros_like(V)
                for _ in range(setup_sweeps):
                    sap.sweep(f, V)
            P = prolongator(V, Ls, d, agg, ntv)
            self.P.append(P)
            Dc = (P.conj().T @ self.D[l] @ P).tocsr()
            self.D.append(Dc)
            self.side.append(Ls // agg)
            self.dof.append(2 * ntv)
        self.n = [Dl.shape[0] for Dl in self.D]
        self.sap_block = tuple(sap_block)
        self._sap = {}

    @classmethod
    def from_prolongators(cls, D0: sp.csr_matrix, L: int, Ps, agg: int = 4, sap_block=(4, 2)) -> "Hierarchy":
        """Hierarchy with the given prolongators P_l (sparse, imported as data) and the oracle's own Galerkin
        operators D_{l+1} = P_l^H D_l P_l built from the oracle's fine operator D0."""
        H = cls.__new__(cls)
        H.levels = len(Ps) + 1
        H.agg = agg
        H.D = [sp.csr_matrix(D0)]
        H.P = []
        H.side = [L]
        H.dof = [2]
        for l, P in enumerate(Ps):
            P = sp.csr_matrix(P)
            if P.shape[0] != H.D[l].shape[0]:
                raise ValueError("prolongator %d has %d rows, level has %d dof" % (l, P.shape[0], H.D[l].shape[0]))
            H.P.append(P)
            H.D.append((P.conj().T @ H.D[l] @ P).tocsr())
            H.side.append(H.side[l] // agg)
            H.dof.append(P.shape[1] // (H.side[l + 1] ** 2))
        H.ntv = H.dof[-1] // 2 if len(Ps) else 0
        H.n = [Dl.shape[0] for Dl in H.D]
        H.sap_block = tuple(sap_block)
        H._sap = {}
        return H

    def sap(self, l: int) -> SAP:
        """The SAP smoother of level l (block side sap_block[0] on the fine level, sap_block[1] above)."""
        if l not in self._sap:
            b = self.sap_block[0] if l == 0 else self.sap_block[1]
            self._sap[l] = SAP(self.D[l], self.side[l], self.dof[l], b)
        return self._sap[l]

    def vcycle(self, l: int, r: np.ndarray, pre: int = 1, post: int = 1) -> np.ndarray:
        """One V(pre, post)-cycle from level l as an approximate solve e ~ D_l^{-1} r (r: (n,) or (n, k))."""
        r = np.asarray(r, dtype=complex)
        if l == self.levels - 1:
            if not hasattr(self, "_coarsest_inv"):
                self._coarsest_inv = np.linalg.inv(self.D[l].toarray())
            return self._coarsest_inv @ r
        S = self.sap(l)
        e = np.zeros_like(r)
        for _ in range(pre):
            S.sweep(r, e)
        res = r - self.D[l] @ e
        P = self.P[l]
        e = e + P @ self.vcycle(l + 1, P.conj().T @ res, pre, post)
        for _ in range(post):
            S.sweep(r, e)
        return e

    def Phat(self, l: int) -> sp.csr_matrix:
        """Accumulated prolongation P_1 ... P_{l-1} (fine x n_l); identity at l = 0."""
        M = sp.identity(self.n[0], dtype=complex, format="csr")
        for j in range(l):
            M = M @ self.P[j]
        return M.tocsr()

    def gamma5(self, l: int) -> sp.dia_matrix:
        d = self.dof[l]
        sgn = 1.0 - 2.0 * chirality(np.arange(d), d)
        return sp.diags(np.tile(sgn, self.side[l] ** 2))
