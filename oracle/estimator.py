"""Per-sample values, exact traces and the MLMC stopping rule.

Telescoping sum (Eq. mgmlmc, Sect. 3.2), with M_l = D_l^{-1} - P_l D_{l+1}^{-1} P_l^H:

    tr(D^{-1}) = sum_{l=1}^{L-1} tr(M_l) + tr(D_L^{-1}).

A *term* is a pair (a, b) of levels: (a, a+1) for a difference level,
(a, b) with b > a+1 when levels are skipped (Eq. skip_level, Sect. 4.1, with
P_{a->b} = P_a ... P_{b-1}), and (L, None) for the coarsest level.  Sample j
of a term uses the Z2 vector x_j on level a (Hutchinson, Eq.
Hutchinson_estimator):

    s_j = x_j^H D_a^{-1} x_j - (P_{a->b}^H x_j)^H D_b^{-1} (P_{a->b}^H x_j)

and, when the term's operator A is deflated with A ~ L diag(a) R^H
(Sect. 2, Eq. splitting_defl_trace),

    s_j -= x_j^H L diag(a) R^H x_j,   estimate = mean_j s_j + tr(L diag(a) R^H).

For real Z2 noise the variance of s_j is (Eq. variance_in_terms_of_frob_norm)
1/2 ||offdiag(A + A^T)||_F^2 with the *transpose* (not the adjoint), read
that way because x is real: s = sum_i A_ii + sum_{i<j} (A_ij + A_ji) x_i x_j.

Pinned in tests/test_oracle_estimator.py by brute force over all 2^n Z2
vectors (mean = trace and variance = closed form, exactly), the telescoping
and skip identities of the exact traces, and zero variance at full deflation.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .noise import z2_noise


def term_list(nlevels: int, skip=()) -> list:
    """Terms of the telescoping sum over the levels not in ``skip``."""
    levels = [lev for lev in range(1, nlevels + 1) if lev not in set(skip)]
    assert levels[0] == 1, "the finest level cannot be skipped"
    return [(levels[i], levels[i + 1]) for i in range(len(levels) - 1)] + [(levels[-1], None)]


class DirectSolvers:
    """Sparse LU factorisations of D_l, built on first use."""

    def __init__(self, hier):
        self.hier = hier
        self._lu = {}

    def solve(self, level: int, B: np.ndarray) -> np.ndarray:
        """D_level^{-1} B for B of shape (n_level, m)."""
        if level not in self._lu:
            self._lu[level] = spla.splu(sp.csc_matrix(self.hier.D[level - 1]))
        return self._lu[level].solve(np.ascontiguousarray(B, dtype=np.complex128))


def term_samples(hier, term, X: np.ndarray, solvers: DirectSolvers, defl=None) -> np.ndarray:
    """Complex samples s_j for the rows x_j of X (shape (nsamples, n_a))."""
    a, b = term
    Xt = np.ascontiguousarray(X.T).astype(np.complex128)           # (n_a, m)
    Z = solvers.solve(a, Xt)
    s = np.einsum("ij,ij->j", Xt.conj(), Z)
    if b is not None:
        Y = hier.prolongator(a, b).conj().T @ Xt
        W = solvers.solve(b, Y)
        s = s - np.einsum("ij,ij->j", Y.conj(), W)
    if defl is not None:
        A = defl.R.conj().T @ Xt                                    # R^H x
        B = defl.L.conj().T @ Xt                                    # L^H x
        s = s - np.einsum("k,kj,kj->j", defl.a, B.conj(), A)
    return s


def noise_samples(hier, term, seed: int, first: int, count: int, solvers, defl=None):
    """Samples first .. first+count-1 of a term on the counter-based Z2 noise."""
    a = term[0]
    n_a = hier.D[a - 1].shape[0]
    X = z2_noise(seed, a, first, count, n_a)
    return term_samples(hier, term, X, solvers, defl)


def term_operator(hier, term) -> np.ndarray:
    """Dense traced operator of a term: D_a^{-1} - P D_b^{-1} P^H, or D_a^{-1}."""
    a, b = term
    A = np.linalg.inv(hier.D[a - 1].toarray())
    if b is not None:
        P = hier.prolongator(a, b).toarray()
        A = A - P @ np.linalg.inv(hier.D[b - 1].toarray()) @ P.conj().T
    return A


def exact_trace(A: np.ndarray) -> complex:
    return complex(np.trace(A))


def z2_variance(A: np.ndarray) -> float:
    """1/2 ||offdiag(A + A^T)||_F^2 (Eq. variance_in_terms_of_frob_norm)."""
    S = A + A.T
    off = S - np.diag(np.diag(S))
    return 0.5 * float(np.sum(np.abs(off) ** 2))


def deflated_operator(A: np.ndarray, defl) -> np.ndarray:
    """A - L diag(a) R^H: the operator whose trace the deflated samples estimate."""
    return A - (defl.L * defl.a[None, :]) @ defl.R.conj().T


def sample_stats(s: np.ndarray):
    """(mean, unbiased variance E|s - mean|^2) of complex samples."""
    m = s.mean()
    v = float(np.sum(np.abs(s - m) ** 2) / max(len(s) - 1, 1))
    return complex(m), v


def mlmc_allocation(V, C, N, abs_tol):
    """Giles-style sample targets, growth capped at x2 per round.

    The MLMC allocation minimising total cost at total variance abs_tol^2 is
    N_l = abs_tol^-2 sqrt(V_l / C_l) sum_m sqrt(V_m C_m) (the general MLMC
    approach Sect. 3.2 builds on; the paper gives no rule of its own).
    """
    V = np.maximum(np.asarray(V, dtype=np.float64), 0.0)
    C = np.asarray(C, dtype=np.float64)
    N = np.asarray(N, dtype=np.int64)
    total = float(np.sum(np.sqrt(V * C)))
    target = np.ceil(np.sqrt(V / C) * total / abs_tol ** 2).astype(np.int64)
    new = np.minimum(np.maximum(target, N), 2 * N)
    if np.all(new == N):                         # guarantee progress
        worst = int(np.argmax(V / N))
        new[worst] = 2 * N[worst]
    return new


def mlmc_estimate(sample_fn, nterms: int, rel_tol: float, max_samples: int,
                  costs, tau: complex = 0.0, pilot: int = 16):
    """Estimate sum of term traces + tau until sqrt(sum V_l/N_l) <= rel_tol |estimate|.

    ``sample_fn(t, first, count)`` returns samples first..first+count-1 of term t
    (0-based).  ``costs`` are the per-sample costs C_l.  Returns a dict with the
    estimate, per-term sample counts, means and variances, and ``converged``.
    """
    samples = [np.asarray(sample_fn(t, 0, pilot)) for t in range(nterms)]
    rounds = 0
    while True:
        N = np.array([len(s) for s in samples])
        stats = [sample_stats(s) for s in samples]
        means = np.array([m for m, _ in stats])
        V = np.array([v for _, v in stats])
        est = complex(np.sum(means) + tau)
        err = math.sqrt(float(np.sum(V / N)))
        rel = err / abs(est) if est != 0 else math.inf
        if rel <= rel_tol or int(N.sum()) >= max_samples:
            return dict(estimate=est, rel_err=rel, N=N.tolist(), means=means.tolist(),
                        variances=V.tolist(), rounds=rounds, converged=rel <= rel_tol)
        target = mlmc_allocation(V, costs, N, rel_tol * abs(est))
        for t in range(nterms):
            extra = int(target[t] - N[t])
            if extra > 0:
                samples[t] = np.concatenate([samples[t], sample_fn(t, int(N[t]), extra)])
        rounds += 1
