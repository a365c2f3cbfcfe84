"""Optimal IBF, sweep-out stage (Sec. 4.1-4.2), in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the product path never
imports it.  It starts from the oracle's own explicit preliminary IBF
(``ExplicitIBF``: V^0, H^l, M^h, G^l, U^L of Sec. 3) and compresses it:

* middle level (eq. KeqUCMRV): every switch block M~_p (r x r) is replaced by
  a rank-r0 factorisation M~_p = C_p (R_p)^*, the identity as middle factor;
* toward U^L (eq. GC): for every output pair p of level l = h+1..L the pencil
  [G_{p,0} C_{q0}, G_{p,1} C_{q1}] (r x 2 r0) is factored as
  C'_p [Gbar_{p,0}, Gbar_{p,1}]; finally Ubar = U^L C^L (per point, its leaf);
* toward V^0 (eq. HR): for every input pair q of level l-1 (l = h..1) the
  stacked pencil [R_{p0}^* H_{p0,c}; R_{p1}^* H_{p1,c}] (2 r0 x r) of the two
  outputs p_a it feeds is factored as [Hbar_{p0,c}; Hbar_{p1,c}] R'_q^*;
  finally Vbar = V^0 R^0 (per frequency, its leaf).

Every rank-r0 factorisation is the truncated SVD written as in eq.
lowrankSVD: Z = (U0 S0^(1/2)) (S0^(1/2) V0^*), so both factors carry the
singular values.  The paper computes these SVDs by random sampling for large
blocks and notes that a direct truncated SVD is as good when r is small, as
here; the direct SVD makes the factorisation deterministic.  Ranks are the
same r0 for every block (the paper's simplification r0 = r0(eps, l, i, j) ->
r0); a block of lower rank is padded with zero columns.

The compressed factors have the preliminary IBF's block structure with r
replaced by r0, so ``OptimalIBF.apply`` is the same sequence of block
products: Lambda^0 = Vbar g, Hbar levels 1..h, identity switch, Gbar levels
h+1..L, u = Ubar Lambda^L.

With ``sweep_in=True`` the sweep-in stage (Sec. 4.3, eq. IBFin) follows,
from the outer factors toward the middle:

* Ubar = Udot C^L, per leaf: the rows of Ubar at the leaf's points
  (n_i x r0) split as (n_i x K) (K x r0);
* for l = L..h+1, per input pair q of level l-1, the stacked pencil
  [C_{p0} Gbar_{p0,c}; C_{p1} Gbar_{p1,c}] = [Gdot_{p0,c}; Gdot_{p1,c}] C_q;
* Vbar^* = R^0^* Vdot^*, per frequency leaf: the column Vbar_j (r0 x 1)
  splits as (r0 x K) (K x 1);
* for l = 1..h, per output pair p, the pencil
  [Hbar_{p,0} R_{q0}^*, Hbar_{p,1} R_{q1}^*] = R_p^* [Hdot_{p,0}, Hdot_{p,1}];
* Mdot = C^h Mbar R^h^* (Mbar is the identity after the sweep-out).

The rank of each split is the number of points the boxes hold, capped at
r0: an X box at level l holds at most K^G_l = min(max count, r0) points
and an Omega box at level L-l holds 2^l frequencies, K^H_l = min(2^l, r0).
A block with fewer points has at most that many independent rows, so every
split is exact and the sweep-in leaves the operator unchanged (to
rounding) while shrinking the outer blocks; with one point per leaf the
leaf factors become 1 x 1.
"""
from __future__ import annotations

import numpy as np

from . import ExplicitIBF


def split_svd(Z: np.ndarray, r0: int) -> tuple[np.ndarray, np.ndarray]:
    """Rank-r0 truncated SVD of Z as (A, B), Z ~ A B, A = U0 S0^(1/2),
    B = S0^(1/2) V0^* (eq. lowrankSVD); zero-padded to r0 if rank(Z) < r0."""
    U, s, Vh = np.linalg.svd(Z, full_matrices=False)
    k = min(r0, s.size)
    sq = np.sqrt(s[:k])
    A = np.zeros((Z.shape[0], r0), np.complex128)
    B = np.zeros((r0, Z.shape[1]), np.complex128)
    A[:, :k] = U[:, :k] * sq
    B[:k] = sq[:, None] * Vh[:k]
    return A, B


class OptimalIBF:
    """Sweep-out compression of the preliminary IBF to rank r0 (Sec. 4.2),
    optionally followed by the sweep-in stage (Sec. 4.3)."""

    def __init__(self, phase_id: int, N: int, r: int, x, r0: int, h: int | None = None, sweep_in: bool = False):
        ex = ExplicitIBF(phase_id, N, r, x, h)
        self.N, self.r, self.r0, self.L, self.h = ex.N, ex.r, int(r0), ex.L, ex.h
        if not 1 <= self.r0 <= r:
            raise ValueError("need 1 <= r0 <= r")
        if not 1 <= self.h < self.L:
            raise ValueError("need 1 <= h < L")
        N, L, h, r0 = self.N, self.L, self.h, self.r0
        self.x = np.asarray(x, np.float64)
        self.leaf = np.clip(np.floor(self.x * N).astype(np.int64), 0, N - 1)
        V, U, M = ex.V(), ex.U(), ex.M()
        blk = {l: ex.blocks(l) for l in range(1, L + 1)}

        # middle level: M~_p = C_p R_p^*
        C = np.zeros((N, r, r0), np.complex128)
        Rs = np.zeros((N, r0, r), np.complex128)          # R_p^*
        for p in range(N):
            C[p], Rs[p] = split_svd(M[p], r0)
        self.blocks = {}
        # toward U^L
        for l in range(h + 1, L + 1):
            nj = 1 << (L - l)
            Cn = np.zeros_like(C)
            B = np.zeros((N, 2, r0, r0), np.complex128)
            for p in range(N):
                i, j = p >> (L - l), p & (nj - 1)
                q0 = (i >> 1) * (2 * nj) + 2 * j
                P = np.hstack([blk[l][p, 0] @ C[q0], blk[l][p, 1] @ C[q0 + 1]])
                Cn[p], Bp = split_svd(P, r0)
                B[p, 0], B[p, 1] = Bp[:, :r0], Bp[:, r0:]
            self.blocks[l] = B
            C = Cn
        self.U = np.einsum("nt,nts->ns", U, C[self.leaf])
        # toward V^0
        for l in range(h, 0, -1):
            nj = 1 << (L - l)
            nC = 2 * nj
            Rn = np.zeros_like(Rs)
            B = np.zeros((N, 2, r0, r0), np.complex128)
            for q in range(N):
                ip, Cq = q // nC, q % nC
                j, c = Cq >> 1, Cq & 1
                p0, p1 = (2 * ip) * nj + j, (2 * ip + 1) * nj + j
                Q = np.vstack([Rs[p0] @ blk[l][p0, c], Rs[p1] @ blk[l][p1, c]])
                A, Rn[q] = split_svd(Q, r0)
                B[p0, c], B[p1, c] = A[:r0], A[r0:]
            self.blocks[l] = B
            Rs = Rn
        self.V = np.einsum("kst,kt->ks", Rs, V)          # Vbar_k = R^0_k^* V_k
        self.M = None                                    # identity middle factor
        self.KG = {l: r0 for l in range(h, L + 1)}
        self.KH = {l: r0 for l in range(0, h + 1)}
        if sweep_in:
            self._sweep_in()

    def _sweep_in(self):
        """Sec. 4.3: sweep from U^L and V^0 toward the middle (module docstring)."""
        N, L, h, r0 = self.N, self.L, self.h, self.r0
        KG = {l: min(int(np.bincount(self.leaf >> (L - l), minlength=1 << l).max()), r0) for l in range(h, L + 1)}
        KH = {l: min(1 << l, r0) for l in range(0, h + 1)}
        # Ubar = Udot C^L, leaf by leaf
        C = np.zeros((N, KG[L], r0), np.complex128)
        Ud = np.zeros((self.x.size, KG[L]), np.complex128)
        for i in range(N):
            rows = np.nonzero(self.leaf == i)[0]
            if rows.size:
                Ud[rows], C[i] = split_svd(self.U[rows], KG[L])
        # C^l Gbar^(l-1 -> l) = Gdot C^(l-1), l = L .. h+1
        for l in range(L, h, -1):
            nj = 1 << (L - l)
            nC = 2 * nj
            Cn = np.zeros((N, KG[l - 1], r0), np.complex128)
            B = np.zeros((N, 2, KG[l], KG[l - 1]), np.complex128)
            for q in range(N):
                ip, Cq = q // nC, q % nC
                j, c = Cq >> 1, Cq & 1
                p0, p1 = (2 * ip) * nj + j, (2 * ip + 1) * nj + j
                Z = np.vstack([C[p0] @ self.blocks[l][p0, c], C[p1] @ self.blocks[l][p1, c]])
                A, Cn[q] = split_svd(Z, KG[l - 1])
                B[p0, c], B[p1, c] = A[:KG[l]], A[KG[l]:]
            self.blocks[l] = B
            C = Cn
        # Vbar^* = R^0^* Vdot^*, leaf by leaf (one frequency per leaf)
        Rs = np.zeros((N, r0, KH[0]), np.complex128)      # R^0_j^*
        Vd = np.zeros((N, KH[0]), np.complex128)
        for j in range(N):
            Rs[j], Bv = split_svd(self.V[j][:, None], KH[0])
            Vd[j] = Bv[:, 0]
        # Hbar^(l-1 -> l) R^(l-1)^* = R^l^* Hdot, l = 1 .. h
        for l in range(1, h + 1):
            nj = 1 << (L - l)
            Rn = np.zeros((N, r0, KH[l]), np.complex128)
            B = np.zeros((N, 2, KH[l], KH[l - 1]), np.complex128)
            for p in range(N):
                i, j = p >> (L - l), p & (nj - 1)
                q0 = (i >> 1) * (2 * nj) + 2 * j
                P = np.hstack([self.blocks[l][p, 0] @ Rs[q0], self.blocks[l][p, 1] @ Rs[q0 + 1]])
                Rn[p], Bp = split_svd(P, KH[l])
                B[p, 0], B[p, 1] = Bp[:, :KH[l - 1]], Bp[:, KH[l - 1]:]
            self.blocks[l] = B
            Rs = Rn
        self.M = np.einsum("pks,pst->pkt", C, Rs)          # Mdot = C^h I R^h^*
        self.U, self.V, self.KG, self.KH = Ud, Vd, KG, KH

    def nnz(self) -> int:
        """Stored entries of the factors (V, the butterfly blocks, the middle
        factor counted as r0 x r0 when it is the identity, U)."""
        mid = self.N * self.r0 * self.r0 if self.M is None else self.M.size
        return self.V.size + sum(b.size for b in self.blocks.values()) + mid + self.U.size

    def apply(self, g) -> np.ndarray:
        """u = Ubar Gbar^{L-1..h} I Hbar^{h..1} Vbar g (after the sweep-in:
        Udot Gdot Mdot Hdot Vdot g), g of shape (N,) or (N, nrhs)."""
        g = np.asarray(g, np.complex128)
        vec = g.ndim == 1
        g2 = g.reshape(self.N, -1)
        N, L = self.N, self.L
        lam = self.V[:, :, None] * g2[:, None, :]               # (pair, t, col)
        for l in range(1, L + 1):
            nj = 1 << (L - l)
            p = np.arange(N)
            i, j = p >> (L - l), p & (nj - 1)
            q0 = (i >> 1) * (2 * nj) + 2 * j
            B = self.blocks[l]
            lam = np.einsum("pts,psk->ptk", B[:, 0], lam[q0]) + np.einsum("pts,psk->ptk", B[:, 1], lam[q0 + 1])
            if l == self.h and self.M is not None:
                lam = np.einsum("pts,psk->ptk", self.M, lam)
        u = np.einsum("nt,ntk->nk", self.U, lam[self.leaf])
        return u[:, 0] if vec else u

    def adjoint(self, y) -> np.ndarray:
        """g = (the compressed product)^* y."""
        y = np.asarray(y, np.complex128)
        vec = y.ndim == 1
        y2 = y.reshape(self.x.size, -1)
        N, L = self.N, self.L
        lam = np.zeros((N, self.U.shape[1], y2.shape[1]), np.complex128)
        np.add.at(lam, self.leaf, np.conj(self.U)[:, :, None] * y2[:, None, :])
        for l in range(L, 0, -1):
            if l == self.h and self.M is not None:
                lam = np.einsum("pts,ptk->psk", np.conj(self.M), lam)
            nj = 1 << (L - l)
            p = np.arange(N)
            i, j = p >> (L - l), p & (nj - 1)
            q0 = (i >> 1) * (2 * nj) + 2 * j
            B = self.blocks[l]
            prev = np.zeros((N, B.shape[3], lam.shape[2]), np.complex128)
            np.add.at(prev, q0, np.einsum("pts,ptk->psk", np.conj(B[:, 0]), lam))
            np.add.at(prev, q0 + 1, np.einsum("pts,ptk->psk", np.conj(B[:, 1]), lam))
            lam = prev
        g = np.einsum("kt,ktc->kc", np.conj(self.V), lam)
        return g[:, 0] if vec else g
