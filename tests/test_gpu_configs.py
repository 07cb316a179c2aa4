"""The two large configurations at their full sizes.

256^2 ("Precision": beta 5, a 3-term sum over levels of 131072 / 65536 / 16384
unknowns with one solver-only level of 4096 below, the last term deflated by the
128 smallest singular vectors of the level-3 operator (the oracle's, given as
vectors), 512 Z2 vectors in one block): sampled per-sample parity with the
oracle's sparse-LU solves in the benchmark's precision (mg_precision 16, BF16
deflation projections: within the bound their rounding allows) and, undeflated, in
FP64.  The hierarchy is built from the seeded start vectors (no inverse-iteration
setup) so that the oracle's own setup stays within a test's time; the setup
iteration itself is checked against the oracle at 128^2 (test_gpu_full_size).

1024^2 ("Scale": 2097152 fine unknowns, three solver-only levels): the oracle
cannot solve it, so the oracle checks the operators that define the samples (D_1,
P_2^H and the level-3 operator D_3, built by the oracle from the same start
vectors), and the mixed-precision path is checked against the FP64 GPU path on the
same hierarchy, sample by sample.
"""
import numpy as np
import pytest

import inputs
from oracle import deflation as odefl
from oracle import estimator as oest
from oracle import hierarchy as ohier
from oracle import noise as onoise

from gpu_common import bf16_deflation_bound, rand_complex, rel_sample_error, require_gpu, within_bound

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
NCHK = 8


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.fixture(scope="module")
def c3():
    w = inputs.workload("schwinger-256x256")
    theta = w.gauge()
    sv = w.start_vectors()
    H = ohier.build_hierarchy(theta, w.m0, w.agg, w.nvec, sv, 0)
    terms = oest.term_list(w.nlevels, w.skip)
    assert terms == [(1, 2), (2, 3), (3, None)]
    defl = odefl.coarsest_deflation(H.D[2], H.g5[2], w.k, sparse=True)
    solvers = oest.DirectSolvers(H)
    # the last term deflated by the oracle's 128 smallest singular vectors of D_3 given
    # as vectors (R = V, L = D_3^{-1} V, a = 1): the deflated samples do not depend on
    # how well an eigensolver converged on this level's clustered spectrum
    defl = odefl.vector_deflation(H, (3, None), defl.L, solvers)
    refs = {term: oest.noise_samples(H, term, w.noise_seed, 0, NCHK, solvers, defl if term[1] is None else None)
            for term in terms}
    plain3 = oest.noise_samples(H, (3, None), w.noise_seed, 0, NCHK, solvers, None)
    X3 = onoise.z2_noise(w.noise_seed, 3, 0, NCHK, H.D[2].shape[0])
    return w, theta, sv, terms, defl, refs, plain3, X3


def _c3_ctx(pkg, w, theta, sv, prec, nrhs):
    ctx = pkg.Context(mg_precision=prec, max_block_rhs=nrhs)
    ctx.set_gauge(theta)
    ctx.set_mass(w.m0)
    ctx.set_hierarchy(w.agg, w.nvec, sv, setup_iters=0)
    ctx.set_terms(list(w.skip))
    return ctx


def test_c3_sampled_parity_benchmark_precision(pkg, c3):
    w, theta, sv, terms, defl, refs, plain3, X3 = c3
    with _c3_ctx(pkg, w, theta, sv, 16, w.nrhs) as ctx:
        assert ctx.num_terms() == (3, [1, 2, 3])
        ctx.set_term_deflation_vectors(2, defl.R.T)
        _, L, R, tau = ctx.get_term_deflation(2, w.k)
        assert abs(tau - defl.trace_term()) < 1e-9 * abs(defl.trace_term())
        assert np.abs(L.T - defl.L).max() < 1e-9 * np.abs(defl.L).max()
        for t, term in enumerate(terms):
            got, st = ctx.estimate_level(t, 0, w.nrhs, w.noise_seed)
            assert st["nsamples"] == w.nrhs and np.all(np.isfinite(got))
            if term[1] is None:
                assert within_bound(got[:NCHK], refs[term], bf16_deflation_bound(defl, X3)), term
            else:
                assert rel_sample_error(got[:NCHK], refs[term]) < 1e-9, term


def test_c3_sampled_parity_fp64(pkg, c3):
    w, theta, sv, terms, defl, refs, plain3, X3 = c3
    with _c3_ctx(pkg, w, theta, sv, 64, 64) as ctx:
        for t, term in enumerate(terms):
            got, _ = ctx.estimate_level(t, 0, NCHK, w.noise_seed)
            ref = plain3 if term[1] is None else refs[term]
            assert rel_sample_error(got, ref) < 1e-9, term


def test_c4_operators_and_precisions(pkg):
    w = inputs.workload("schwinger-1024x1024")
    theta = w.gauge()
    sv = w.start_vectors()
    # the oracle's first three levels from the same start vectors
    H = ohier.build_hierarchy(theta, w.m0, w.agg[:2], w.nvec[:2], sv[:2], 0)
    rng = np.random.default_rng(4)
    with pkg.Context(mg_precision=16, max_block_rhs=32) as ctx:
        ctx.set_gauge(theta)
        ctx.set_mass(w.m0)
        ctx.set_hierarchy(w.agg, w.nvec, sv, setup_iters=0)
        for lev, n in ((1, 2097152), (3, 262144)):
            x = rand_complex(rng, (2, n))
            y = ctx.apply(pkg.OP_D, lev, x, n)
            ref = (H.D[lev - 1] @ x.T).T
            assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max(), lev
        x = rand_complex(rng, (2, 1048576))
        y = ctx.apply(pkg.OP_PH, 2, x, 262144)
        ref = (H.prolongator(2, 3).conj().T @ x.T).T
        assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()
    # mixed against FP64 on one hierarchy: the FP64 context takes the mixed one's test
    # vectors as its start vectors without further iteration, so P and D_l are the same
    w4 = dict(agg=w.agg, nvec=w.nvec)
    with pkg.Context(mg_precision=16, max_block_rhs=32) as c16:
        c16.set_gauge(theta)
        c16.set_mass(w.m0)
        c16.set_hierarchy(w4["agg"], w4["nvec"], sv, setup_iters=w.setup_iters, setup_tol=1e-12)
        c16.set_terms(list(w.skip))
        tv = [c16.get_test_vectors(l + 1, w.nvec[l]) for l in range(len(w.agg))]
        s16 = [c16.estimate_level(t, 0, 16, w.noise_seed)[0] for t in range(3)]
    with pkg.Context(mg_precision=64, max_block_rhs=16) as c64:
        c64.set_gauge(theta)
        c64.set_mass(w.m0)
        c64.set_hierarchy(w4["agg"], w4["nvec"], tv, setup_iters=0)
        c64.set_terms(list(w.skip))
        for t in range(3):
            s64 = c64.estimate_level(t, 0, 16, w.noise_seed)[0]
            assert rel_sample_error(s16[t], s64) < 1e-9, t
