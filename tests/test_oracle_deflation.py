"""Pins of the oracle's exact deflation (Sect. 2)."""
import numpy as np

import inputs
from oracle import deflation, estimator, wilson


def gauge_D(Lx=4, Lt=4, m0=0.05, seed=11):
    th = inputs.metropolis_u1(Lx, Lt, 2.0, 20, seed)
    return wilson.wilson_dirac(th, m0), wilson.gamma5_fine(Lx * Lt)


def test_singular_values_match_direct_svd():
    D, g5 = gauge_D()
    k = 7
    sigma, U, V, lam = deflation.smallest_triplets(D, g5, k)
    sv = np.sort(np.linalg.svd(D.toarray(), compute_uv=False))[:k]
    assert np.abs(sigma - sv).max() < 1e-12


def test_triplets_satisfy_dv_equals_u_sigma():
    D, g5 = gauge_D()
    sigma, U, V, lam = deflation.smallest_triplets(D, g5, 10)
    Dd = D.toarray()
    assert np.abs(Dd @ V - U * sigma[None, :]).max() < 1e-12
    assert np.abs(U.conj().T @ U - np.eye(10)).max() < 1e-12
    assert np.abs(V.conj().T @ V - np.eye(10)).max() < 1e-12


def test_trace_term_equals_projected_inverse_trace():
    # tr(D^{-1} U U^H) = sum_i u_i^H v_i / sigma_i   (Eq. small_trace_term)
    D, g5 = gauge_D()
    defl = deflation.coarsest_deflation(D, g5, 6)
    U = defl.R
    Dinv = np.linalg.inv(D.toarray())
    ref = np.trace(Dinv @ U @ U.conj().T)
    assert abs(defl.trace_term() - ref) < 1e-12 * abs(ref)


def test_full_deflation_removes_everything():
    D, g5 = gauge_D(Lx=2, Lt=4)
    n = D.shape[0]
    defl = deflation.coarsest_deflation(D, g5, n)
    Dinv = np.linalg.inv(D.toarray())
    assert np.abs(estimator.deflated_operator(Dinv, defl)).max() < 1e-11 * np.abs(Dinv).max()
    assert abs(defl.trace_term() - np.trace(Dinv)) < 1e-11 * abs(np.trace(Dinv))


def test_deflation_lowers_variance():
    D, g5 = gauge_D(m0=-0.05)
    Dinv = np.linalg.inv(D.toarray())
    v0 = estimator.z2_variance(Dinv)
    v1 = estimator.z2_variance(estimator.deflated_operator(Dinv, deflation.coarsest_deflation(D, g5, 8)))
    assert v1 < v0
