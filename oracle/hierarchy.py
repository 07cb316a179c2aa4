"""Multigrid hierarchy: spin-preserving aggregation and Galerkin coarsening.

Sect. 3.1 builds P_l algebraically by aggregation from a few test vectors
(following the adaptive-aggregation construction it cites, whose details the
paper does not give).  Readings used here:

* Aggregates are ax x at blocks of lattice sites.  Each aggregate carries two
  spin blocks: on the fine level the two spin components, on a coarse level
  the first and second half of a site's dof (the Gamma5 = +1 / -1 halves).
* Column (S, s, j) of P_l is test vector j restricted to aggregate S and spin
  block s, after modified Gram-Schmidt in j order inside that block, so
  P^H P = I (Eq. mgmlmc requires it) and Gamma5^l P_l = P_l Gamma5^{l+1}
  (Sect. 4.2).  Coarse dof order: coarse site major, then s, then j.
* Test vectors: seeded complex Gaussian start vectors, then ``setup_iters``
  rounds of inverse iteration v <- D_l^{-1} v (exact solve), v <- v / ||v||.
* D_{l+1} = P_l^H D_l P_l (Galerkin with R_l = P_l^H, Sect. 3.1/3.2).

Pinned in tests/test_oracle_hierarchy.py: P^H P = I, Gamma5 commutation,
Hermitian Q_l on every level, an eigenvalue of D that lies in range(P)
reappearing in D_{l+1}, a complete P preserving the spectrum, and
convergence of the test-vector iteration to the smallest-|lambda| mode.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import wilson


def aggregate_prolongator(vectors: np.ndarray, lx: int, lt: int, d: int,
                          ax: int, at: int) -> sp.csr_matrix:
    """P of shape (n_fine, n_coarse) from test vectors of shape (nvec, n_fine).

    n_fine = lx * lt * d; the fine dof of site (x, t), component a, is
    (x + lx * t) * d + a, and component a belongs to spin block a // (d // 2).
    """
    nvec, n = vectors.shape
    assert n == lx * lt * d and lx % ax == 0 and lt % at == 0 and d % 2 == 0
    half = d // 2
    cx, ct = lx // ax, lt // at
    rows, cols, vals = [], [], []
    for T in range(ct):
        for X in range(cx):
            S = X + cx * T
            sites = [(X * ax + i) + lx * (T * at + j) for j in range(at) for i in range(ax)]
            for s in range(2):
                idx = np.array([site * d + s * half + a for site in sites for a in range(half)])
                B = vectors[:, idx].T.copy()          # (m, nvec), column j = v_j on the block
                if nvec > B.shape[0]:
                    raise ValueError("more test vectors than rows in an aggregate block")
                Q = np.zeros_like(B)
                for j in range(nvec):                 # modified Gram-Schmidt, j order
                    w = B[:, j].copy()
                    for i in range(j):
                        w -= (np.vdot(Q[:, i], w)) * Q[:, i]
                    nrm = np.linalg.norm(w)
                    if nrm == 0.0:
                        raise ValueError("rank-deficient aggregate block")
                    Q[:, j] = w / nrm
                for j in range(nvec):
                    c = S * 2 * nvec + s * nvec + j
                    rows.extend(idx.tolist())
                    cols.extend([c] * len(idx))
                    vals.extend(Q[:, j].tolist())
    P = sp.coo_matrix((vals, (rows, cols)), shape=(n, cx * ct * 2 * nvec)).tocsr()
    return P


def galerkin(D: sp.spmatrix, P: sp.spmatrix) -> sp.csr_matrix:
    """D_{l+1} = P^H D_l P (Sect. 3.1, Petrov-Galerkin with R = P^H)."""
    Dc = (P.conj().T @ (D @ P)).tocsr()
    Dc.sum_duplicates()
    return Dc


def inverse_iteration(D: sp.spmatrix, v0: np.ndarray, iters: int) -> np.ndarray:
    """Test vectors: ``iters`` rounds of v <- D^{-1} v, v <- v/||v|| (exact sparse LU)."""
    V = np.array(v0, dtype=np.complex128, copy=True)
    if iters == 0:
        return V
    lu = spla.splu(sp.csc_matrix(D))
    for _ in range(iters):
        V = lu.solve(np.ascontiguousarray(V.T)).T
        V = V / np.linalg.norm(V, axis=1, keepdims=True)
    return V


@dataclasses.dataclass
class Hierarchy:
    """Operators of every level l = 1..L (index 0 is level 1)."""
    dims: list            # [(lx, lt, d)]
    D: list               # sparse D_l
    P: list               # sparse P_l, l = 1..L-1
    g5: list              # diagonal of Gamma5^l
    nvec: list
    test_vectors: list    # (nvec_l, n_l) after the setup iteration

    @property
    def nlevels(self) -> int:
        return len(self.D)

    def prolongator(self, a: int, b: int) -> sp.csr_matrix:
        """P_{a->b} = P_a P_{a+1} ... P_{b-1} (1-based levels, a < b)."""
        M = self.P[a - 1]
        for lev in range(a + 1, b):
            M = (M @ self.P[lev - 1]).tocsr()
        return M


def build_hierarchy(theta: np.ndarray, m0: float, agg, nvec, start_vectors,
                    setup_iters: int) -> Hierarchy:
    """Levels 1..L from the gauge field, top-down (Sect. 3.1)."""
    Lt, Lx, _ = theta.shape
    D = [wilson.wilson_dirac(theta, m0)]
    dims = [(Lx, Lt, 2)]
    g5 = [wilson.gamma5_fine(Lx * Lt)]
    Ps, tvs = [], []
    for (ax, at), nv, v0 in zip(agg, nvec, start_vectors):
        lx, lt, d = dims[-1]
        V = inverse_iteration(D[-1], v0, setup_iters)
        P = aggregate_prolongator(V, lx, lt, d, ax, at)
        Ps.append(P)
        tvs.append(V)
        D.append(galerkin(D[-1], P))
        dims.append((lx // ax, lt // at, 2 * nv))
        g5.append(wilson.gamma5_coarse((lx // ax) * (lt // at), nv))
    return Hierarchy(dims=dims, D=D, P=Ps, g5=g5, nvec=list(nvec), test_vectors=tvs)
