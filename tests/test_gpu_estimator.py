"""Per-sample parity of the GPU estimator with the oracle on identical seeded
noise (FP64 bar 1e-9 relative), deflation triplets, ragged blocks, the
probe-vector entry, mixed precision, skip-a-level terms and the MLMC loop."""
import numpy as np
import pytest

import inputs
from oracle import deflation as odefl
from oracle import estimator as oest
from oracle import hierarchy as ohier

from gpu_common import bf16_deflation_bound, make_ctx, rel_sample_error, require_gpu, small_problem, within_bound
from oracle import noise as onoise

pytestmark = pytest.mark.gpu
TOL64 = 1e-9


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.fixture(scope="module")
def c1():
    """The 16x16 workload: 2 levels, 4x4 aggregates, 4 test vectors per spin, k = 16."""
    w = inputs.workload("schwinger-16x16")
    theta = w.gauge()
    sv = w.start_vectors()
    H = ohier.build_hierarchy(theta, w.m0, w.agg, w.nvec, sv, w.setup_iters)
    defl = odefl.coarsest_deflation(H.D[-1], H.g5[-1], w.k)
    return w, theta, sv, H, defl


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_c1_samples_match_oracle(pkg, c1, prec):
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=prec) as ctx:
        # test vectors after the setup iteration agree with the oracle's exact inverse iteration
        tv = ctx.get_test_vectors(1, w.nvec[0])
        assert np.abs(tv - H.test_vectors[0]).max() < 1e-9
        ctx.compute_deflation(w.k, 1e-10, 500)
        lam, sig, U, V, tau = ctx.get_deflation(w.k, 2)
        assert np.abs(sig - 1.0 / defl.a).max() < 1e-10 * sig.max()
        assert abs(tau - defl.trace_term()) < 1e-9 * abs(defl.trace_term())
        Pg = V.T @ V.conj()
        Po = defl.L @ defl.L.conj().T
        assert np.abs(Pg - Po).max() < 1e-8
        for t, term in enumerate(oest.term_list(2)):
            got, st = ctx.estimate_level(t, 0, w.nrhs, w.noise_seed)
            ref = oest.noise_samples(H, term, w.noise_seed, 0, w.nrhs, solvers,
                                     defl if term[1] is None else None)
            if prec == 16 and term[1] is None:
                # deflation projections on the tensor cores: BF16 factors, FP32 sums
                X = onoise.z2_noise(w.noise_seed, term[0], 0, w.nrhs, H.D[term[0] - 1].shape[0])
                assert within_bound(got, ref, bf16_deflation_bound(defl, X)), (prec, term)
                assert rel_sample_error(got, ref) < 1e-2
                continue
            assert rel_sample_error(got, ref) < TOL64, (prec, term)
            assert st["nsamples"] == w.nrhs
            assert abs(st["mean_re"] - ref.mean().real) < 1e-9 * max(1, abs(ref.mean()))


def test_ragged_blocks_and_probes(pkg, c1):
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, max_block_rhs=16) as ctx:
        got, _ = ctx.estimate_level(0, 7, 37, 99)
        ref = oest.noise_samples(H, (1, 2), 99, 7, 37, solvers)
        assert rel_sample_error(got, ref) < TOL64
        # caller-supplied probes: random signs from the shared input generator
        n = H.D[0].shape[0]
        probes = np.where(inputs.uniform(4, 4, 5 * n).reshape(5, n) < 0.5, 1, -1).astype(np.int8)
        gp, _ = ctx.estimate_level_probes(0, probes)
        rp = oest.term_samples(H, (1, 2), probes.astype(float), solvers)
        assert rel_sample_error(gp, rp) < TOL64


def test_setup_without_iterations_and_single_rhs(pkg):
    theta, sv = small_problem(agg=((2, 2), (2, 2)), nvec=(2, 2))
    H = ohier.build_hierarchy(theta, 0.05, ((2, 2), (2, 2)), (2, 2), sv, 0)
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, 0.05, ((2, 2), (2, 2)), (2, 2), sv, 0) as ctx:
        for t, term in enumerate(oest.term_list(3)):
            got, _ = ctx.estimate_level(t, 3, 1, 5)
            ref = oest.noise_samples(H, term, 5, 3, 1, solvers)
            assert rel_sample_error(got, ref) < TOL64


def test_skip_level_terms(pkg):
    agg, nvec = ((2, 2), (2, 1), (1, 2)), (2, 2, 2)
    theta, sv = small_problem(agg=agg, nvec=nvec)
    H = ohier.build_hierarchy(theta, 0.05, agg, nvec, sv, 1)
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, 0.05, agg, nvec, sv, 1) as ctx:
        ctx.set_terms([2])
        nt, levels = ctx.num_terms()
        assert (nt, levels) == (3, [1, 3, 4])
        for t, term in enumerate(oest.term_list(4, skip=(2,))):
            got, _ = ctx.estimate_level(t, 0, 20, 11)
            ref = oest.noise_samples(H, term, 11, 0, 20, solvers)
            assert rel_sample_error(got, ref) < TOL64, term


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("k", [4, 5])
def test_deflation_above_a_solver_only_level(pkg, prec, k):
    # the last term of the sum on level 2 of 3 (level 3 serves only the solver), its
    # operator's k smallest triplets found by the eigensolver (subspace of b = 20 / 21):
    # |lambda| of Q_2 = Gamma5 D_2 has a slow gap after the 21st (0.8107 / 0.8117), so a
    # Rayleigh-Ritz step with Q_2 itself meets spurious Ritz values in the spectral gap
    # around 0; the triplets, tau and the deflated samples must match the oracle's
    agg, nvec, m0 = ((2, 2), (2, 2)), (2, 4), 0.05
    theta = inputs.metropolis_u1(16, 16, 3.0, 20, 91)
    sv = [inputs.start_vectors(91, 1, 16 * 16 * 2, 2), inputs.start_vectors(91, 2, 8 * 8 * 4, 4)]
    H = ohier.build_hierarchy(theta, m0, agg, nvec, sv, 1)
    defl = odefl.coarsest_deflation(H.D[1], H.g5[1], k)
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, m0, agg, nvec, sv, 1, mg_precision=prec) as ctx:
        ctx.set_terms([3])
        ctx.compute_deflation(k, 1e-10, 300)
        lam, L, R, tau = ctx.get_term_deflation(1, k)
        assert np.abs(np.sort(np.abs(lam)) - np.sort(np.abs(defl.lam))).max() < 1e-9
        assert abs(tau - defl.trace_term()) < 1e-9 * abs(defl.trace_term())
        for t, term in enumerate(oest.term_list(3, (3,))):
            got, _ = ctx.estimate_level(t, 0, 24, 6)
            ref = oest.noise_samples(H, term, 6, 0, 24, solvers, defl if term[1] is None else None)
            assert rel_sample_error(got, ref) < TOL64, (prec, k, term)


def test_mlmc_loop_matches_oracle_rule(pkg, c1):
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    costs = [1.0, 0.1]
    terms = oest.term_list(2)
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters) as ctx:
        ctx.compute_deflation(w.k, 1e-10, 500)
        res = ctx.estimate_trace(2e-2, 200000, 31, costs)

    def fn(t, first, count):
        term = terms[t]
        return oest.noise_samples(H, term, 31, first, count, solvers, defl if term[1] is None else None)

    ref = oest.mlmc_estimate(fn, 2, 2e-2, 200000, costs, tau=defl.trace_term())
    assert res["converged"] == 1 and ref["converged"]
    assert [t["nsamples"] for t in res["terms"]] == ref["N"]
    assert abs(res["trace"] - ref["estimate"]) < 1e-9 * abs(ref["estimate"])
    exact = np.trace(np.linalg.inv(H.D[0].toarray()))
    assert abs(res["trace"] - exact) < 5 * res["rel_err"] * abs(exact)


@pytest.mark.parametrize("prec", [64, 32])
def test_difference_level_deflation(pkg, c1, prec):
    # exact deflation on the difference level (Sect. 4.2): k = 5 largest singular
    # triplets of M_1 (a spectral gap follows the 5th), then deflated samples
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    k = 5
    dref = odefl.difference_deflation(H, (1, 2), k)
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=prec) as ctx:
        ctx.compute_term_deflation(0, k, 1e-10, 2000)
        lam, L, R, tau = ctx.get_term_deflation(0, k)
        assert np.abs(np.abs(lam) - dref.a).max() < 1e-9 * dref.a.max()
        assert abs(tau - dref.trace_term()) < 1e-9 * max(1.0, abs(dref.trace_term()))
        Pg = L.T @ L.conj()
        Po = dref.L @ dref.L.conj().T
        assert np.abs(Pg - Po).max() < 1e-8
        got, _ = ctx.estimate_level(0, 0, w.nrhs, w.noise_seed)
        ref = oest.noise_samples(H, (1, 2), w.noise_seed, 0, w.nrhs, solvers, dref)
        assert rel_sample_error(got, ref) < TOL64
        # the coarsest term is unaffected; with both deflations the MLMC estimate adds both traces
        ctx.compute_deflation(w.k, 1e-10, 500)
        res = ctx.estimate_trace(5e-2, 100000, 3, [1.0, 0.1])
        exact = np.trace(np.linalg.inv(H.D[0].toarray()))
        assert abs(res["trace"] - exact) < 5 * res["rel_err"] * abs(exact)
        assert abs(res["deflated_part"] - (dref.trace_term() + defl.trace_term()).real) < 1e-8 * abs(exact)


def test_deflation_by_given_vectors(pkg, c1):
    # inexact-style deflation with the same seeded orthonormal vectors on both sides
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    n = H.D[0].shape[0]
    V, _ = np.linalg.qr(inputs.gaussian_complex(17, 3, (n, 6)))
    dref = odefl.vector_deflation(H, (1, 2), V, solvers)
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters) as ctx:
        ctx.set_term_deflation_vectors(0, V.T)
        _, L, R, tau = ctx.get_term_deflation(0, 6)
        assert np.abs(R.T - V).max() < 1e-15
        assert abs(tau - dref.trace_term()) < 1e-9 * max(1.0, abs(dref.trace_term()))
        got, _ = ctx.estimate_level(0, 0, 40, 8)
        ref = oest.noise_samples(H, (1, 2), 8, 0, 40, solvers, dref)
        assert rel_sample_error(got, ref) < TOL64


def test_tensor_core_deflation_matches_rounded_factors(pkg, c1):
    # mg_precision 16 forms the deflation projections on the tensor cores from the
    # factors rounded to BF16.  With given vectors that are BF16 numbers already
    # (R = V exact) and L = A V rounded on both sides by the same rule, the samples
    # equal the oracle's with the rounded factors up to FP32 accumulation, and the
    # deflated part the estimate adds is the trace over those rounded factors.
    from oracle import rounding
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    term = (2, None)
    n = H.D[1].shape[0]
    V, _ = np.linalg.qr(inputs.gaussian_complex(19, 4, (n, 12)))
    V = rounding.bf16(V)
    dref = odefl.bf16_factors(odefl.vector_deflation(H, term, V, solvers))
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=16) as ctx:
        ctx.set_term_deflation_vectors(1, V.T)
        tau_used = ctx.term_deflated_part(1)
        assert abs(tau_used - dref.trace_term()) < 1e-12 * abs(dref.trace_term())
        got, _ = ctx.estimate_level(1, 0, 96, 21)
        ref = oest.noise_samples(H, term, 21, 0, 96, solvers, dref)
        X = onoise.z2_noise(21, 2, 0, 96, n)
        assert within_bound(got, ref, bf16_deflation_bound(dref, X, factors_rounded=True))
        # and the bound is tight enough to see a wrong factor: without the deflation
        # the samples are far outside it
        plain = oest.noise_samples(H, term, 21, 0, 96, solvers, None)
        assert not within_bound(got, plain, bf16_deflation_bound(dref, X, factors_rounded=True))


def test_tensor_core_deflation_keeps_estimate_unbiased(pkg, c1):
    # exact deflation at mg_precision 16: BF16 projections in the samples, the trace
    # over the same rounded factors in the estimate -> consistent with the exact trace
    w, theta, sv, H, defl = c1
    exact = np.trace(np.linalg.inv(H.D[0].toarray()))
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=16) as ctx:
        ctx.compute_deflation(w.k, 1e-10, 500)
        tau_used = ctx.term_deflated_part(1)
        tau64 = ctx.get_deflation(w.k, 2)[4]
        assert tau_used != tau64 and abs(tau_used - tau64) < 1e-2 * abs(tau64)
        res = ctx.estimate_trace(2e-2, 200000, 77, [1.0, 0.1])
        assert res["converged"] == 1
        assert abs(res["deflated_part"] - tau_used.real) < 1e-12 * abs(tau_used)
        assert abs(res["trace"] - exact) < 5 * res["rel_err"] * abs(exact)


@pytest.mark.parametrize("prec", [64, 32])
def test_inexact_deflation_keeps_estimate_unbiased(pkg, c1, prec):
    # loosely converged vectors (eigensolver 1e-1, inner solves 1e-3, as in the paper's
    # inexact runs): the trace estimate stays consistent with the exact trace
    w, theta, sv, H, defl = c1
    exact = np.trace(np.linalg.inv(H.D[0].toarray()))
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=prec) as ctx:
        ctx.compute_term_deflation_inexact(0, 8, 1e-1, 1e-3, 500)
        ctx.compute_term_deflation_inexact(1, w.k, 1e-1, 1e-3, 500)
        _, L, R, _ = ctx.get_term_deflation(0, 8)
        assert np.abs(R.conj() @ R.T - np.eye(8)).max() < 1e-10          # orthonormal V
        res = ctx.estimate_trace(3e-2, 100000, 5, [1.0, 0.1])
        assert res["converged"] == 1
        assert abs(res["trace"] - exact) < 5 * res["rel_err"] * abs(exact)


def test_deflated_hutchinson_on_the_fine_operator(pkg, c1):
    # skip every coarse level: one term tr(D_1^{-1}) (Sect. 2's deflated Hutchinson),
    # deflated by the 16 smallest triplets of D_1; MG still preconditions the solves
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    dref = odefl.coarsest_deflation(H.D[0], H.g5[0], 16)
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters) as ctx:
        ctx.set_terms([2])
        assert ctx.num_terms() == (1, [1])
        ctx.compute_term_deflation(0, 16, 1e-10, 2000)
        lam, L, R, tau = ctx.get_term_deflation(0, 16)
        assert np.abs(np.abs(lam) - 1.0 / dref.a).max() < 1e-10 * np.abs(lam).max()
        assert abs(tau - dref.trace_term()) < 1e-9 * abs(dref.trace_term())
        got, _ = ctx.estimate_level(0, 0, 48, 12)
        ref = oest.noise_samples(H, (1, None), 12, 0, 48, solvers, dref)
        assert rel_sample_error(got, ref) < TOL64


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_three_levels_with_wide_coarse_blocks(pkg, prec):
    # d = 16 on level 2 (8 x 8 sites) and 3 (4 x 4 sites, n = 256, tensor-core
    # coarsest solve): mg_precision 16 runs the smoother's block stencil on the
    # tensor cores in BF16; the FP64 outer solve keeps every sample at the bar
    agg, nvec = ((4, 4), (2, 2)), (8, 8)
    theta, sv = small_problem(32, 32, beta=3.0, m0=-0.05, agg=agg, nvec=nvec)
    H = ohier.build_hierarchy(theta, -0.05, agg, nvec, sv, 2)
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, -0.05, agg, nvec, sv, 2, mg_precision=prec) as ctx:
        for t, term in enumerate(oest.term_list(3)):
            got, _ = ctx.estimate_level(t, 0, 40, 21)
            ref = oest.noise_samples(H, term, 21, 0, 40, solvers)
            assert rel_sample_error(got, ref) < TOL64, (prec, term)


@pytest.mark.parametrize("prec", [64, 16])
def test_kcycle_coarse_correction(pkg, prec):
    # 4 levels with a K-cycle (two FGMRES steps per coarse-grid correction on the
    # levels above the coarsest): only the preconditioner changes, so every sample
    # still meets the FP64 bar against the oracle's direct solves
    # 16^2 -> 8^2 x 4 -> 4^2 x 8 -> 4 x 2 sites x 8 dof: no aggregation is complete
    agg, nvec, m0 = ((2, 2), (2, 2), (2, 1)), (2, 4, 4), 0.02
    theta, sv = small_problem(16, 16, 3.0, m0, agg, nvec, seed=41)
    H = ohier.build_hierarchy(theta, m0, agg, nvec, sv, 2)
    solvers = oest.DirectSolvers(H)
    with make_ctx(pkg, theta, m0, agg, nvec, sv, 2, mg_precision=prec, kcycle_iters=2) as ctx:
        for t, term in enumerate(oest.term_list(4)):
            got, _ = ctx.estimate_level(t, 0, 40, 9)
            ref = oest.noise_samples(H, term, 9, 0, 40, solvers)
            assert rel_sample_error(got, ref) < TOL64, (prec, term)


def test_concurrent_terms_on_separate_streams(pkg, c1):
    # the two terms of the 16x16 workload at once, each on its own context and CUDA
    # stream (one entry with device noise, one with caller probes): the second context
    # is a device copy of the first (mgmlmc_create_copy), so every sample must equal the
    # first context's bit for bit, and the oracle's within the bar
    import torch
    w, theta, sv, H, defl = c1
    solvers = oest.DirectSolvers(H)
    with torch.cuda.stream(torch.cuda.Stream()):
        src = make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=16)
    src.compute_deflation(w.k, 1e-10, 500)
    with torch.cuda.stream(torch.cuda.Stream()):
        cpy = pkg.Context(copy_of=src)
    assert cpy.get_deflation(w.k, 2)[-1] == src.get_deflation(w.k, 2)[-1]     # tau
    ctxs = [src, cpy]
    try:
        n1 = H.D[-1].shape[0]
        probes = np.where(inputs.uniform(5, 1, 48 * n1).reshape(48, n1) < 0.5, 1, -1).astype(np.int8)
        for rep in range(2):                                     # twice in a row
            outs, stats = pkg.estimate_concurrent(ctxs, [0, 1], 16, 48, w.noise_seed, probes=[None, probes])
            assert [s["nsamples"] for s in stats] == [48, 48]
            seq0, _ = src.estimate_level(0, 16, 48, w.noise_seed)
            seq1, _ = src.estimate_level_probes(1, probes)
            assert np.array_equal(outs[0], seq0) and np.array_equal(outs[1], seq1)
        ref0 = oest.noise_samples(H, (1, 2), w.noise_seed, 16, 48, solvers)
        ref1 = oest.term_samples(H, (2, None), probes.astype(float), solvers, defl)
        assert rel_sample_error(outs[0], ref0) < TOL64
        # mg_precision 16: the deflation projections use BF16 factors on the tensor cores
        assert within_bound(outs[1], ref1, bf16_deflation_bound(defl, probes.astype(float)))
        assert cpy.term_deflated_part(1) == src.term_deflated_part(1)
        with pytest.raises(pkg.MgmlmcError):
            pkg.estimate_concurrent([ctxs[0], ctxs[0]], [0, 1], 0, 8, 1)   # one context twice
    finally:
        for ctx in ctxs:
            ctx.close()


def test_concurrent_mlmc_loop_matches_one_context(pkg, c1):
    # the MLMC loop with each term drawn on its own context and stream: with fixed
    # costs the allocation is deterministic, so every round, sample count and the
    # estimate equal those of the one-context loop
    import torch
    w, theta, sv, H, defl = c1
    src = make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, w.setup_iters, mg_precision=16)
    src.compute_deflation(w.k, 1e-10, 500)
    with torch.cuda.stream(torch.cuda.Stream()):
        cpy = pkg.Context(copy_of=src)
    ctxs = [src, cpy]
    try:
        res = pkg.estimate_trace_concurrent(ctxs, 2e-2, 200000, 31, [1.0, 0.1])
        one = ctxs[0].estimate_trace(2e-2, 200000, 31, [1.0, 0.1])
        assert res["converged"] == 1 and one["converged"] == 1
        assert res["rounds"] == one["rounds"]
        assert [t["nsamples"] for t in res["terms"]] == [t["nsamples"] for t in one["terms"]]
        assert abs(res["trace"] - one["trace"]) <= 1e-12 * abs(one["trace"])
        exact = np.trace(np.linalg.inv(H.D[0].toarray()))
        assert abs(res["trace"] - exact) < 5 * res["rel_err"] * abs(exact)
    finally:
        for ctx in ctxs:
            ctx.close()
