"""Exact deflation (Sect. 2).

The k smallest singular triplets of a Gamma5-Hermitian D come from the
eigenpairs of the Hermitian Q = Gamma5 D = X Lambda X^H: the left singular
vectors are U = Gamma5 X sign(Lambda), the singular values Sigma = |Lambda|
and the right singular vectors V = X; the k smallest |lambda| give the k
smallest sigma.  The deflated trace term is (Eq. small_trace_term)

    tr(D^{-1} U_k U_k^H) = tr(U_k^H V_k Sigma_k^{-1}) = sum_i (u_i^H v_i) / sigma_i.

Deflation data are held in the generic form used by the estimator: for the
traced operator A = D^{-1} = V Sigma^{-1} U^H, left vectors L = V, right
vectors R = U and values a = 1/sigma, so that A's deflated part is
L diag(a) R^H and its trace is sum_i a_i r_i^H l_i.

Pinned in tests/test_oracle_deflation.py: the singular values equal a direct
SVD's, D V = U Sigma, the trace term equals tr(D^{-1} U U^H) from a dense
inverse, and k = n removes the whole operator (zero-variance samples).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Deflation:
    L: np.ndarray      # (n, k) left vectors of the traced operator
    R: np.ndarray      # (n, k) right vectors
    a: np.ndarray      # (k,) singular values of the traced operator
    lam: np.ndarray    # (k,) eigenvalues of the Hermitian operator they came from

    @property
    def k(self) -> int:
        return self.a.shape[0]

    def trace_term(self) -> complex:
        """sum_i a_i r_i^H l_i (Eq. small_trace_term)."""
        return complex(np.sum(self.a * np.einsum("ik,ik->k", self.R.conj(), self.L)))


def smallest_triplets(D, g5: np.ndarray, k: int):
    """(sigma, U, V, lam): the k smallest singular triplets of D via eig(Gamma5 D).

    Ordered by increasing |lambda|; dense Hermitian eigensolver (numpy eigh).
    """
    Dd = D.toarray() if sp.issparse(D) else np.asarray(D)
    Q = g5[:, None] * Dd
    Q = 0.5 * (Q + Q.conj().T)           # exact Hermitian part (Q is Hermitian up to rounding)
    lam, X = np.linalg.eigh(Q)
    order = np.argsort(np.abs(lam), kind="stable")[:k]
    lam, X = lam[order], X[:, order]
    sigma = np.abs(lam)
    U = g5[:, None] * X * np.sign(lam)[None, :]
    V = X
    return sigma, U, V, lam


def smallest_triplets_sparse(D, g5: np.ndarray, k: int):
    """smallest_triplets for operators too large for a dense eigensolver: the k
    eigenvalues of Q = Gamma5 D nearest zero (the smallest |lambda|) by shift-invert
    Lanczos at sigma = 0 (scipy's eigsh, which factors Q once with a sparse LU), the
    same ordering and the same (U, Sigma, V) as smallest_triplets."""
    import scipy.sparse.linalg as spla
    Q = sp.diags(g5) @ sp.csr_matrix(D)
    Q = (0.5 * (Q + Q.conj().T)).tocsc()
    lam, X = spla.eigsh(Q, k=k, sigma=0.0, which="LM", tol=1e-14, ncv=min(Q.shape[0], max(2 * k + 1, k + 40)))
    order = np.argsort(np.abs(lam), kind="stable")
    lam, X = lam[order], X[:, order]
    sigma = np.abs(lam)
    U = g5[:, None] * X * np.sign(lam)[None, :]
    return sigma, U, X, lam


def coarsest_deflation(D, g5: np.ndarray, k: int, sparse: bool = False) -> Deflation:
    """Deflation of the traced operator D^{-1} by D's k smallest triplets (dense
    eigensolver, or shift-invert Lanczos with sparse=True)."""
    sigma, U, V, lam = (smallest_triplets_sparse if sparse else smallest_triplets)(D, g5, k)
    return Deflation(L=V, R=U, a=1.0 / sigma, lam=lam)


def hermitian_difference_operator(hier, term) -> np.ndarray:
    """J = M Gamma5^a = Q_a^{-1} - P Q_b^{-1} P^H for the term (a, b) (Sect. 4.2).

    M = D_a^{-1} - P D_b^{-1} P^H with P = P_{a->b}; Gamma5^a P = P Gamma5^b and
    Q_l = Gamma5^l D_l Hermitian make J Hermitian.  Dense; small lattices only.
    """
    a, b = term
    g_a, g_b = hier.g5[a - 1], hier.g5[b - 1]
    Qa = g_a[:, None] * hier.D[a - 1].toarray()
    Qb = g_b[:, None] * hier.D[b - 1].toarray()
    P = hier.prolongator(a, b).toarray()
    J = np.linalg.inv(Qa) - P @ np.linalg.inv(Qb) @ P.conj().T
    return 0.5 * (J + J.conj().T)


def difference_deflation(hier, term, k: int) -> Deflation:
    """Exact deflation of the difference-level operator M by its k largest
    singular triplets, from the eigenpairs of J (Eq. hermitian_diff_lev_op):
    J = X Lambda X^H gives M = U S V^H with U = X sign(Lambda), S = |Lambda|,
    V = Gamma5^a X.  For the traced operator A = M: L = U, R = V, a = S.
    Ordered by decreasing |lambda|; dense Hermitian eigensolver (numpy eigh).
    """
    J = hermitian_difference_operator(hier, term)
    lam, X = np.linalg.eigh(J)
    order = np.argsort(-np.abs(lam), kind="stable")[:k]
    lam, X = lam[order], X[:, order]
    g = hier.g5[term[0] - 1]
    U = X * np.sign(lam)[None, :]
    V = g[:, None] * X
    return Deflation(L=U, R=V, a=np.abs(lam), lam=lam)


def vector_deflation(hier, term, V: np.ndarray, solvers=None) -> Deflation:
    """Deflation of a term by given vectors V (n_a x k): the orthogonal projector
    V V^H (Sect. 2's Pi, Sect. 3.2's inexact deflation with approximate vectors),
    whose deflated part A V V^H needs the k extra applications A V of the traced
    operator A (D_a^{-1}, or D_a^{-1} - P D_b^{-1} P^H).  L = A V, R = V, a = 1:
    samples subtract x^H (A V)(V^H x), the estimate adds tr(V^H A V).  The
    estimator stays unbiased for any V.
    """
    from .estimator import DirectSolvers
    a, b = term
    S = solvers if solvers is not None else DirectSolvers(hier)
    V = np.asarray(V, dtype=np.complex128)
    W = S.solve(a, V)
    if b is not None:
        P = hier.prolongator(a, b)
        W = W - P @ S.solve(b, P.conj().T @ V)
    return Deflation(L=W, R=V, a=np.ones(V.shape[1]), lam=np.zeros(V.shape[1]))


def bf16_factors(d: Deflation) -> Deflation:
    """The same deflation with its factors L and R rounded to BF16 (oracle.rounding),
    the form the tensor-core projections use; trace_term() of the result is the
    deflated part over the rounded factors."""
    from .rounding import bf16
    return Deflation(L=bf16(d.L), R=bf16(d.R), a=d.a.copy(), lam=d.lam.copy())

