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


def _three_level(seed=31):
    from oracle import hierarchy
    th = inputs.metropolis_u1(8, 8, 2.0, 10, seed)
    sv = [inputs.start_vectors(seed, 1, 128, 2), inputs.start_vectors(seed, 2, 64, 2)]
    return hierarchy.build_hierarchy(th, 0.05, ((2, 2), (2, 2)), (2, 2), sv, 1)


def test_difference_operator_hermitian_and_svd():
    # J = M Gamma5 is Hermitian and |eig(J)| are the singular values of M (Sect. 4.2)
    H = _three_level()
    for term in [(1, 2), (2, 3), (1, 3)]:
        J = deflation.hermitian_difference_operator(H, term)
        g = H.g5[term[0] - 1]
        M = estimator.term_operator(H, term)
        assert np.abs(M * g[None, :] - J).max() < 1e-11 * np.abs(J).max()
        sv = np.sort(np.linalg.svd(M, compute_uv=False))[::-1]
        ev = np.sort(np.abs(np.linalg.eigvalsh(J)))[::-1]
        assert np.abs(sv - ev).max() < 1e-10 * sv[0]


def test_difference_deflation_triplets_and_trace():
    H = _three_level()
    term = (1, 2)
    M = estimator.term_operator(H, term)
    k = 12
    d = deflation.difference_deflation(H, term, k)
    # M R = L diag(a)  (M V = U S), and the deflated trace term equals tr(U S V^H)
    assert np.abs(M @ d.R - d.L * d.a[None, :]).max() < 1e-10 * d.a.max()
    sv = np.sort(np.linalg.svd(M, compute_uv=False))[::-1][:k]
    assert np.abs(np.sort(d.a)[::-1] - sv).max() < 1e-10 * sv[0]
    low = (d.L * d.a[None, :]) @ d.R.conj().T
    assert abs(d.trace_term() - np.trace(low)) < 1e-10 * max(1.0, abs(np.trace(low)))
    # deflation removes the largest singular values: the Frobenius norm drops accordingly
    rest = M - low
    assert abs(np.linalg.norm(rest) ** 2 - (np.linalg.norm(M) ** 2 - np.sum(d.a ** 2))) < 1e-8 * np.linalg.norm(M) ** 2


def test_full_difference_deflation_is_exact():
    H = _three_level()
    term = (2, 3)
    n = H.D[1].shape[0]
    d = deflation.difference_deflation(H, term, n)
    M = estimator.term_operator(H, term)
    assert np.abs(estimator.deflated_operator(M, d)).max() < 1e-10 * np.abs(M).max()
    assert abs(d.trace_term() - np.trace(M)) < 1e-10 * max(1.0, abs(np.trace(M)))


def test_vector_deflation_unbiased_and_exact_limit():
    # any V: mean over all Z2 vectors + tr(V^H A V) = tr(A); V = exact right singular
    # vectors: identical to exact deflation
    import itertools
    from oracle import hierarchy
    th = inputs.metropolis_u1(2, 4, 2.0, 10, 3)
    sv = [inputs.start_vectors(3, 1, 16, 1)]
    H = hierarchy.build_hierarchy(th, 0.1, ((1, 2),), (1,), sv, 1)
    solvers = estimator.DirectSolvers(H)
    X = np.array(list(itertools.product([1.0, -1.0], repeat=16)))
    term = (1, 2)
    A = estimator.term_operator(H, term)
    V, _ = np.linalg.qr(inputs.gaussian_complex(5, 5, (16, 3)))
    d = deflation.vector_deflation(H, term, V, solvers)
    s = estimator.term_samples(H, term, X, solvers, d)
    assert abs(s.mean() + d.trace_term() - np.trace(A)) < 1e-11 * max(1.0, abs(np.trace(A)))
    ex = deflation.difference_deflation(H, term, 3)
    dv = deflation.vector_deflation(H, term, ex.R, solvers)
    assert np.abs(estimator.deflated_operator(A, dv) - estimator.deflated_operator(A, ex)).max() < 1e-10 * np.abs(A).max()


def test_sparse_triplets_match_dense_eigensolver():
    # shift-invert Lanczos (eigsh at sigma = 0) gives the same k smallest |lambda| and
    # the same deflated part as the dense Hermitian eigensolver
    th = inputs.metropolis_u1(8, 8, 2.0, 20, 31)
    D = wilson.wilson_dirac(th, 0.05)
    g5 = np.tile([1.0, -1.0], D.shape[0] // 2)
    for k in (4, 12):
        dd = deflation.coarsest_deflation(D, g5, k)
        ds = deflation.coarsest_deflation(D, g5, k, sparse=True)
        assert np.allclose(np.sort(1 / dd.a), np.sort(1 / ds.a), rtol=1e-10, atol=0)
        assert abs(dd.trace_term() - ds.trace_term()) < 1e-10 * abs(dd.trace_term())
        Pd = dd.L @ dd.L.conj().T
        Ps = ds.L @ ds.L.conj().T
        assert np.abs(Pd - Ps).max() < 1e-9

