"""Pins of oracle.tune_mass.sigma_min, the function that fixes the Wilson mass of
the 128^2 workload (its sigma_min(D) ~ 1e-3; Sect. 2 ties the variance of the
deflated estimator to the smallest singular values, Eq.
relation_frob_norm_and_singvalues).

sigma_min runs inverse iteration on (D^H D)^{-1} with a sparse LU of D.  It is
checked here against the smallest singular value of a dense SVD (a library
routine that shares nothing with it) on small Metropolis fields, including
masses close to the critical one, where the smallest singular value is small
and the iteration converges slowly.
"""
import numpy as np
import pytest

import inputs
from oracle import tune_mass, wilson


def svd_min(D):
    return float(np.linalg.svd(D.toarray(), compute_uv=False).min())


@pytest.mark.parametrize("L,beta,m0,seed", [
    (4, 3.0, -0.10, 11),
    (4, 5.0, 0.05, 12),
    (8, 3.0, -0.10, 13),
    (8, 3.0, -0.25, 14),
    (8, 5.0, -0.05, 15),
])
def test_sigma_min_matches_svd(L, beta, m0, seed):
    D = wilson.wilson_dirac(inputs.metropolis_u1(L, L, beta, 40, seed), m0)
    ref = svd_min(D)
    got = tune_mass.sigma_min(D)
    assert abs(got - ref) <= 1e-8 * ref, (got, ref)


def test_sigma_min_near_critical_mass():
    # scan m0 on an 8x8 field down to a mass where sigma_min is ~1e-2 or smaller,
    # the regime the 128^2 workload is tuned into (1e-3 there)
    th = inputs.metropolis_u1(8, 8, 3.0, 40, 21)
    vals = []
    for m0 in np.linspace(0.0, -0.6, 13):
        D = wilson.wilson_dirac(th, float(m0))
        vals.append((svd_min(D), D))
    smallest, D = min(vals, key=lambda v: v[0])
    assert smallest < 5e-2
    got = tune_mass.sigma_min(D)
    assert abs(got - smallest) <= 1e-8 * smallest, (got, smallest)


def test_sigma_min_is_not_the_smallest_eigenvalue_modulus():
    # D is not normal for a non-trivial gauge field: min |lambda(D)| differs from
    # sigma_min(D), so an iteration on D^{-1} alone (instead of D^{-1} D^{-H}) would
    # be caught by the SVD comparison above
    D = wilson.wilson_dirac(inputs.metropolis_u1(8, 8, 3.0, 40, 13), -0.10)
    lam = np.abs(np.linalg.eigvals(D.toarray())).min()
    assert abs(lam - svd_min(D)) > 1e-4 * svd_min(D)
