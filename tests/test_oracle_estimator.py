"""Pins of the oracle's estimator: brute force, closed-form variance, telescoping."""
import itertools
import math

import numpy as np
import pytest

import inputs
from oracle import deflation, estimator, hierarchy, noise


def build(Lx, Lt, m0, agg, nvec, iters=1, seed=21, beta=2.0):
    th = inputs.metropolis_u1(Lx, Lt, beta, 10, seed)
    dims = [(Lx, Lt, 2)]
    for (ax, at), nv in zip(agg, nvec):
        dims.append((dims[-1][0] // ax, dims[-1][1] // at, 2 * nv))
    sv = [inputs.start_vectors(seed, i + 1, lx * lt * d, nv)
          for i, ((lx, lt, d), nv) in enumerate(zip(dims[:-1], nvec))]
    return hierarchy.build_hierarchy(th, m0, agg, nvec, sv, iters)


def all_z2(n):
    return np.array(list(itertools.product([1.0, -1.0], repeat=n)))


@pytest.mark.parametrize("term", [(1, 2), (2, None)])
def test_brute_force_mean_and_variance(term):
    # 2 x 4 lattice, n = 16: all 65536 Z2 vectors; mean = trace, variance = closed form.
    H = build(2, 4, 0.1, ((1, 2),), (1,))
    solvers = estimator.DirectSolvers(H)
    n = H.D[term[0] - 1].shape[0]
    X = all_z2(n)
    defl = None
    if term[1] is None:
        defl = deflation.coarsest_deflation(H.D[-1], H.g5[-1], 2)
    s = estimator.term_samples(H, term, X, solvers, defl)
    A = estimator.term_operator(H, term)
    if defl is not None:
        A = estimator.deflated_operator(A, defl)
    tr = np.trace(A)
    assert abs(s.mean() - tr) < 1e-12 * max(1.0, abs(tr))
    var_pop = float(np.mean(np.abs(s - s.mean()) ** 2))
    assert abs(var_pop - estimator.z2_variance(A)) < 1e-10 * max(1.0, var_pop)


def test_variance_uses_transpose_not_adjoint():
    # For complex non-symmetric A the transpose and adjoint forms differ; brute force decides.
    rng = np.random.default_rng(3)
    A = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
    X = all_z2(10)
    s = np.einsum("mi,ij,mj->m", X, A, X)
    var_pop = float(np.mean(np.abs(s - s.mean()) ** 2))
    assert abs(var_pop - estimator.z2_variance(A)) < 1e-10 * var_pop
    S = A + A.conj().T
    wrong = 0.5 * np.sum(np.abs(S - np.diag(np.diag(S))) ** 2)
    assert abs(var_pop - wrong) > 1e-3 * var_pop


def test_telescoping_identity_three_levels():
    H = build(8, 8, 0.05, ((2, 2), (2, 2)), (2, 2))
    Dinv_tr = np.trace(np.linalg.inv(H.D[0].toarray()))
    terms = estimator.term_list(3)
    assert terms == [(1, 2), (2, 3), (3, None)]
    total = sum(estimator.exact_trace(estimator.term_operator(H, t)) for t in terms)
    assert abs(total - Dinv_tr) < 1e-12 * abs(Dinv_tr)


def test_skip_level_identity_four_levels():
    H = build(8, 8, 0.05, ((2, 2), (2, 1), (1, 2)), (2, 2, 2))
    Dinv_tr = np.trace(np.linalg.inv(H.D[0].toarray()))
    terms = estimator.term_list(4, skip=(2,))
    assert terms == [(1, 3), (3, 4), (4, None)]
    total = sum(estimator.exact_trace(estimator.term_operator(H, t)) for t in terms)
    assert abs(total - Dinv_tr) < 1e-12 * abs(Dinv_tr)


def test_empirical_variance_within_chi2_bounds():
    H = build(8, 8, 0.1, ((2, 2),), (2,))
    solvers = estimator.DirectSolvers(H)
    N = 4000
    s = estimator.noise_samples(H, (1, 2), 77, 0, N, solvers)
    A = estimator.term_operator(H, (1, 2))
    v_exact = estimator.z2_variance(A)
    _, v_emp = estimator.sample_stats(s)
    # the sample variance of N draws has relative spread ~ sqrt(2/N) ~ 0.022 for near-Gaussian s
    assert abs(v_emp / v_exact - 1) < 6 * math.sqrt(2.0 / N)
    mean_err = abs(s.mean() - np.trace(A))
    assert mean_err < 5 * math.sqrt(v_exact / N)


def test_full_deflation_gives_zero_variance_samples():
    H = build(2, 4, 0.1, ((1, 2),), (1,))
    solvers = estimator.DirectSolvers(H)
    n = H.D[-1].shape[0]
    defl = deflation.coarsest_deflation(H.D[-1], H.g5[-1], n)
    s = estimator.noise_samples(H, (2, None), 5, 0, 32, solvers, defl)
    assert np.abs(s).max() < 1e-11
    tr = np.trace(np.linalg.inv(H.D[-1].toarray()))
    assert abs(defl.trace_term() - tr) < 1e-11 * abs(tr)


def test_sparse_solves_have_small_residual():
    H = build(8, 8, -0.05, ((2, 2),), (2,))
    solvers = estimator.DirectSolvers(H)
    X = noise.z2_noise(1, 1, 0, 4, H.D[0].shape[0]).T.astype(complex)
    Z = solvers.solve(1, X)
    assert np.linalg.norm(H.D[0] @ Z - X) < 1e-12 * np.linalg.norm(X)


def test_mlmc_allocation_and_stopping():
    # Synthetic terms with known variances and costs: the allocation follows
    # N_l ~ sqrt(V_l / C_l), and the loop stops once sqrt(sum V_l/N_l) <= tol |est|.
    rng = np.random.default_rng(0)
    sd = [3.0, 1.0, 0.3]
    mu = [1.0, 2.0, 7.0]
    C = [4.0, 1.0, 0.25]

    def fn(t, first, count):
        r = np.random.default_rng(1000 * t + first)
        return mu[t] + sd[t] * r.standard_normal(count)

    res = estimator.mlmc_estimate(fn, 3, 1e-2, 10 ** 7, C)
    assert res["converged"]
    N = np.array(res["N"], dtype=float)
    err = math.sqrt(sum(v / n for v, n in zip(res["variances"], N)))
    assert err <= 1e-2 * abs(res["estimate"])
    assert abs(res["estimate"] - 10.0) < 5 * err
    ratio = (N / np.sqrt(np.array(res["variances"]) / np.array(C)))
    assert ratio.max() / ratio.min() < 2.5
    new = estimator.mlmc_allocation([1.0, 1.0], [1.0, 1.0], [10, 10], 1e-3)
    assert list(new) == [20, 20]
    del rng


def test_brute_force_deflated_difference_term():
    # all 2^16 Z2 vectors on a 2x4 lattice: deflated difference samples average to
    # tr(M) - tr(L a R^H), and adding the deflated trace term gives tr(M) exactly
    H = build(2, 4, 0.1, ((1, 2),), (1,))
    solvers = estimator.DirectSolvers(H)
    term = (1, 2)
    d = deflation.difference_deflation(H, term, 3)
    X = all_z2(H.D[0].shape[0])
    s = estimator.term_samples(H, term, X, solvers, d)
    M = estimator.term_operator(H, term)
    assert abs(s.mean() + d.trace_term() - np.trace(M)) < 1e-11 * max(1.0, abs(np.trace(M)))
    var_pop = float(np.mean(np.abs(s - s.mean()) ** 2))
    assert abs(var_pop - estimator.z2_variance(estimator.deflated_operator(M, d))) < 1e-9 * max(1.0, var_pop)
