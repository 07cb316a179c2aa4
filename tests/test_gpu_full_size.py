"""Full-size parity on the 128x128 workload in the launch configuration the
benchmark times (one block of 256 right-hand sides per term; every precision of the
multigrid, 16 being the benchmark's): the GPU's
own setup and deflation against the oracle's, and sampled per-sample values
(the first 16 of each 256-sample block, which the oracle computes one by one
with sparse-LU solves)."""
import numpy as np
import pytest

import inputs
from oracle import deflation as odefl
from oracle import estimator as oest
from oracle import hierarchy as ohier

from gpu_common import bf16_deflation_bound, make_ctx, rel_sample_error, require_gpu, within_bound
from oracle import noise as onoise

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.fixture(scope="module")
def c2():
    w = inputs.workload("schwinger-128x128")
    theta = w.gauge()
    sv = w.start_vectors()
    H = ohier.build_hierarchy(theta, w.m0, w.agg, w.nvec, sv, w.setup_iters)
    defl = odefl.coarsest_deflation(H.D[-1], H.g5[-1], w.k)
    return w, theta, sv, H, defl


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_full_size_sampled_parity(pkg, c2, prec):
    w, theta, sv, H, defl = c2
    solvers = oest.DirectSolvers(H)
    nchk = 16
    with pkg.Context(mg_precision=prec, max_block_rhs=w.nrhs) as ctx:
        ctx.set_gauge(theta)
        ctx.set_mass(w.m0)
        ctx.set_hierarchy(w.agg, w.nvec, sv, setup_iters=w.setup_iters, setup_tol=1e-12)
        for lev in (1, 2):
            tv = ctx.get_test_vectors(lev, w.nvec[lev - 1])
            assert np.abs(tv - H.test_vectors[lev - 1]).max() < 1e-8, lev
        ctx.compute_deflation(w.k, 1e-9, 400)
        lam, sig, U, V, tau = ctx.get_deflation(w.k, 3)
        assert np.abs(sig - 1.0 / defl.a).max() < 1e-9 * sig.max()
        assert abs(tau - defl.trace_term()) < 1e-8 * abs(defl.trace_term())
        for t, term in enumerate(oest.term_list(3)):
            got, st = ctx.estimate_level(t, 0, w.nrhs, w.noise_seed)
            ref = oest.noise_samples(H, term, w.noise_seed, 0, nchk, solvers, defl if term[1] is None else None)
            if prec == 16 and term[1] is None:
                # tensor-core deflation projections: BF16 factors, FP32 sums
                X = onoise.z2_noise(w.noise_seed, term[0], 0, nchk, H.D[term[0] - 1].shape[0])
                assert within_bound(got[:nchk], ref, bf16_deflation_bound(defl, X)), (prec, term)
            else:
                err = rel_sample_error(got[:nchk], ref)
                assert err < 1e-9, (prec, term, err)
            # every sample of the block is finite and the block statistics are consistent
            assert np.all(np.isfinite(got)) and st["nsamples"] == w.nrhs
            assert abs(st["mean_re"] - got.mean().real) < 1e-9 * max(1.0, abs(got.mean()))
