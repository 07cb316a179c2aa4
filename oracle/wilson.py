"""The 2D Wilson-Schwinger operator (paper Sect. 1 names it; the form is the
standard Wilson discretisation, read as follows because the paper is silent).

    (D psi)(x) = (m0 + 2) psi(x)
                 - 1/2 sum_{mu=0,1} [ (1 - s_mu) U_mu(x)         psi(x + mu)
                                     + (1 + s_mu) conj(U_mu(x-mu)) psi(x - mu) ]

with U_mu(x) = exp(i theta_mu(x)), s_0 = sigma_1 (space), s_1 = sigma_2 (time),
Gamma5 = sigma_3, periodic in space and antiperiodic in time (every hop across
the t = Lt-1 <-> 0 boundary carries a factor -1).  Degrees of freedom are
ordered site-major, spin-minor: index = 2 * (x + Lx * t) + spin.

With this choice Gamma5 D Gamma5 = D^H (the Gamma5-hermiticity of Sect. 2).
Pinned by the free-field spectrum (closed form), gauge covariance and
Gamma5-hermiticity in tests/test_oracle_wilson.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),        # sigma_1, mu = 0 (x)
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),     # sigma_2, mu = 1 (t)
)
SIGMA3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def wilson_dirac(theta: np.ndarray, m0: float, antiperiodic_t: bool = True) -> sp.csr_matrix:
    """Sparse D for link angles theta[t, x, mu]; returns an (n, n) complex CSR, n = 2 Lx Lt."""
    Lt, Lx, _ = theta.shape
    V = Lx * Lt
    eye2 = np.eye(2, dtype=np.complex128)
    rows, cols, vals = [], [], []

    def add_block(site_a, site_b, block):
        for a in range(2):
            for b in range(2):
                if block[a, b] != 0:
                    rows.append(2 * site_a + a)
                    cols.append(2 * site_b + b)
                    vals.append(block[a, b])

    for t in range(Lt):
        for x in range(Lx):
            s = x + Lx * t
            add_block(s, s, (m0 + 2.0) * eye2)
            for mu in range(2):
                if mu == 0:
                    xf, tf, xb, tb = (x + 1) % Lx, t, (x - 1) % Lx, t
                    sign_f = sign_b = 1.0
                else:
                    xf, tf, xb, tb = x, (t + 1) % Lt, x, (t - 1) % Lt
                    sign_f = -1.0 if (antiperiodic_t and t == Lt - 1) else 1.0
                    sign_b = -1.0 if (antiperiodic_t and t == 0) else 1.0
                u_fwd = np.exp(1j * theta[t, x, mu])
                u_bwd = np.conj(np.exp(1j * theta[tb, xb, mu]))
                add_block(s, xf + Lx * tf, -0.5 * sign_f * u_fwd * (eye2 - SIGMA[mu]))
                add_block(s, xb + Lx * tb, -0.5 * sign_b * u_bwd * (eye2 + SIGMA[mu]))
    n = 2 * V
    D = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    D.sum_duplicates()
    return D


def gamma5_fine(n_sites: int) -> np.ndarray:
    """Diagonal of Gamma5 = sigma_3 on every site (length 2 * n_sites)."""
    return np.tile(np.array([1.0, -1.0]), n_sites)


def gamma5_coarse(n_sites: int, nvec: int) -> np.ndarray:
    """Diagonal of Gamma5 on a coarse level: +1 on the first nvec dof of a site
    (spin block 0), -1 on the next nvec (spin block 1) -- Sect. 4.2."""
    return np.tile(np.concatenate([np.ones(nvec), -np.ones(nvec)]), n_sites)
