"""Pins of the oracle's aggregation hierarchy (Sect. 3.1, Sect. 4.2)."""
import math

import numpy as np
import pytest

import inputs
from oracle import hierarchy, wilson


def small_hierarchy(Lx=8, Lt=8, m0=0.1, agg=((2, 2), (2, 2)), nvec=(2, 2), iters=2, seed=5):
    th = inputs.metropolis_u1(Lx, Lt, 2.0, 10, seed)
    dims = [(Lx, Lt, 2)]
    for (ax, at), nv in zip(agg, nvec):
        dims.append((dims[-1][0] // ax, dims[-1][1] // at, 2 * nv))
    sv = [inputs.start_vectors(seed, i + 1, lx * lt * d, nv)
          for i, ((lx, lt, d), nv) in enumerate(zip(dims[:-1], nvec))]
    return hierarchy.build_hierarchy(th, m0, agg, nvec, sv, iters)


def test_orthonormal_columns_and_gamma5_commutation():
    H = small_hierarchy()
    for lev, P in enumerate(H.P):
        Pd = P.toarray()
        assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-13
        g_f, g_c = H.g5[lev], H.g5[lev + 1]
        assert np.abs(g_f[:, None] * Pd - Pd * g_c[None, :]).max() == 0.0


def test_q_hermitian_on_every_level():
    H = small_hierarchy()
    for D, g5 in zip(H.D, H.g5):
        Q = g5[:, None] * D.toarray()
        assert np.abs(Q - Q.conj().T).max() < 1e-13 * np.abs(Q).max()


def test_coarse_operator_is_nearest_neighbour():
    H = small_hierarchy()
    for lev in (1, 2):
        lx, lt, d = H.dims[lev]
        Dd = H.D[lev].toarray()
        for s1 in range(lx * lt):
            for s2 in range(lx * lt):
                x1, t1, x2, t2 = s1 % lx, s1 // lx, s2 % lx, s2 // lx
                dx = min((x1 - x2) % lx, (x2 - x1) % lx)
                dt = min((t1 - t2) % lt, (t2 - t1) % lt)
                if dx + dt > 1:
                    assert np.abs(Dd[s1 * d:(s1 + 1) * d, s2 * d:(s2 + 1) * d]).max() == 0.0


def test_complete_prolongator_preserves_spectrum():
    # 1x1 aggregates with nvec = d/2 make P a unitary change of basis: D_2 ~ D_1.
    th = inputs.metropolis_u1(4, 4, 2.0, 5, 9)
    D = wilson.wilson_dirac(th, 0.1)
    v = inputs.start_vectors(9, 1, 32, 1)
    P = hierarchy.aggregate_prolongator(v, 4, 4, 2, 1, 1)
    D2 = hierarchy.galerkin(D, P).toarray()
    e1 = list(np.linalg.eigvals(D.toarray()))
    for z in np.linalg.eigvals(D2):
        i = int(np.argmin(np.abs(np.array(e1) - z)))
        assert abs(e1.pop(i) - z) < 1e-12


def test_eigenvector_in_range_of_p_keeps_its_eigenvalue():
    # Free field: the plane wave v = e^{ip.x} chi is an eigenvector of D; with v among
    # the test vectors v lies in range(P), so D_2 = P^H D P has the same eigenvalue.
    Lx, Lt, m0 = 8, 8, 0.05
    D = wilson.wilson_dirac(np.zeros((Lt, Lx, 2)), m0)
    px, pt = 2 * math.pi * 1 / Lx, 3 * math.pi / Lt
    sym = (m0 + 2 - math.cos(px) - math.cos(pt)) * np.eye(2) + 1j * (
        math.sin(px) * wilson.SIGMA[0] + math.sin(pt) * wilson.SIGMA[1])
    lam, chi = np.linalg.eig(sym)
    x = np.arange(Lx)[None, :] * np.ones((Lt, 1))
    t = np.arange(Lt)[:, None] * np.ones((1, Lx))
    phase = np.exp(1j * (px * x + pt * t)).reshape(-1)
    v = (phase[:, None] * chi[:, 0][None, :]).reshape(-1)
    assert np.abs(D @ v - lam[0] * v).max() < 1e-12
    V = np.stack([v, inputs.start_vectors(4, 1, 2 * Lx * Lt, 1)[0]])
    P = hierarchy.aggregate_prolongator(V, Lx, Lt, 2, 2, 2)
    D2 = hierarchy.galerkin(D, P).toarray()
    assert np.min(np.abs(np.linalg.eigvals(D2) - lam[0])) < 1e-11


def test_inverse_iteration_finds_smallest_mode():
    th = inputs.metropolis_u1(4, 4, 2.0, 10, 3)
    D = wilson.wilson_dirac(th, 0.2)
    lam, X = np.linalg.eig(D.toarray())
    order = np.argsort(np.abs(lam))
    assert abs(lam[order[1]]) / abs(lam[order[0]]) > 1.0  # distinct smallest |lambda|
    # inverse iteration converges to the eigenvector(s) of the smallest |lambda|
    # (a conjugate pair when it is complex: check the projection onto their span)
    v = hierarchy.inverse_iteration(D, inputs.start_vectors(3, 1, 32, 1), 200)[0]
    small = [i for i in order if abs(abs(lam[i]) - abs(lam[order[0]])) < 1e-12]
    Qb, _ = np.linalg.qr(X[:, small])
    assert np.linalg.norm(Qb.conj().T @ v) > 1 - 1e-8


def test_hierarchy_levels_shapes():
    H = small_hierarchy()
    assert [D.shape[0] for D in H.D] == [128, 16 * 4, 4 * 4]


def test_too_many_test_vectors_rejected():
    v = inputs.start_vectors(1, 1, 32, 5)
    with pytest.raises(ValueError):
        hierarchy.aggregate_prolongator(v, 4, 4, 2, 2, 2)   # 4-row blocks, 5 vectors
