"""Pins of the oracle's Wilson-Schwinger operator against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import wilson


def free_field_eigs(Lx, Lt, m0, cx=0.0, ct=0.0, antiperiodic=True):
    """Closed-form spectrum of the free (or constant-background) Wilson operator.

    A plane wave e^{i p.x} chi diagonalises D; the 2x2 symbol is
    m0 + sum_mu (1 - cos q_mu) + i sum_mu sigma_mu sin q_mu with q = p + c,
    whose eigenvalues are a +- i sqrt(sum_mu sin^2 q_mu).
    """
    out = []
    for kx in range(Lx):
        for kt in range(Lt):
            px = 2 * math.pi * kx / Lx + cx
            pt = (2 * kt + (1 if antiperiodic else 0)) * math.pi / Lt + ct
            a = m0 + (1 - math.cos(px)) + (1 - math.cos(pt))
            b = math.sqrt(math.sin(px) ** 2 + math.sin(pt) ** 2)
            out += [complex(a, b), complex(a, -b)]
    return np.array(out)


def match_spectra(e1, e2, tol=1e-10):
    e1 = list(e1)
    for z in e2:
        i = int(np.argmin(np.abs(np.array(e1) - z)))
        assert abs(e1[i] - z) < tol, (z, e1[i])
        e1.pop(i)


@pytest.mark.parametrize("Lx,Lt,m0,ap", [(4, 6, 0.1, True), (6, 4, -0.3, True), (4, 4, 0.2, False)])
def test_free_field_spectrum(Lx, Lt, m0, ap):
    th = np.zeros((Lt, Lx, 2))
    D = wilson.wilson_dirac(th, m0, antiperiodic_t=ap).toarray()
    match_spectra(np.linalg.eigvals(D), free_field_eigs(Lx, Lt, m0, antiperiodic=ap))


def test_constant_background_shifts_momenta():
    # theta_mu = c_mu everywhere shifts p_mu -> p_mu + c_mu (forward hop carries e^{+i c}).
    Lx, Lt, m0, cx, ct = 4, 6, 0.05, 0.3, -0.2
    th = np.zeros((Lt, Lx, 2))
    th[..., 0], th[..., 1] = cx, ct
    D = wilson.wilson_dirac(th, m0).toarray()
    match_spectra(np.linalg.eigvals(D), free_field_eigs(Lx, Lt, m0, cx, ct))


def test_free_field_trace_closed_form():
    Lx, Lt, m0 = 8, 8, -0.1
    D = wilson.wilson_dirac(np.zeros((Lt, Lx, 2)), m0).toarray()
    tr = np.trace(np.linalg.inv(D))
    closed = 0.0
    for kx in range(Lx):
        for kt in range(Lt):
            px, pt = 2 * math.pi * kx / Lx, (2 * kt + 1) * math.pi / Lt
            a = m0 + 2 - math.cos(px) - math.cos(pt)
            closed += 2 * a / (a * a + math.sin(px) ** 2 + math.sin(pt) ** 2)
    assert abs(tr - closed) < 1e-11 * abs(closed)


def test_gauge_covariance_and_gamma5_hermiticity():
    rng = np.random.default_rng(0)
    Lx, Lt = 6, 4
    th = rng.uniform(-math.pi, math.pi, (Lt, Lx, 2))
    phi = rng.uniform(-math.pi, math.pi, (Lt, Lx))
    th2 = th.copy()
    th2[..., 0] += phi - np.roll(phi, -1, axis=1)
    th2[..., 1] += phi - np.roll(phi, -1, axis=0)
    D = wilson.wilson_dirac(th, 0.1).toarray()
    D2 = wilson.wilson_dirac(th2, 0.1).toarray()
    g = np.repeat(np.exp(1j * phi.reshape(-1)), 2)          # G = diag(e^{i phi(x)}) x I_2
    assert np.abs(D2 - (g[:, None] * D * g.conj()[None, :])).max() < 1e-13
    g5 = wilson.gamma5_fine(Lx * Lt)
    assert np.abs(g5[:, None] * D * g5[None, :] - D.conj().T).max() < 1e-14


def test_nonzeros_per_row():
    # 2 spin dof on the site + 4 neighbours x 2 spins: nnz(D1) = n (1 + 8) / 2 ... per row <= 9.
    th = np.random.default_rng(1).uniform(-3, 3, (8, 8, 2))
    D = wilson.wilson_dirac(th, 0.0)
    assert D.nnz == 2 * 64 * 9
