"""Shared fixtures of the GPU tests: build the library, build matching oracle
hierarchies from the same seeded inputs."""
import numpy as np
import pytest

import inputs


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_15383_gb300 as pkg
    return pkg


def small_problem(Lx=8, Lt=8, beta=2.0, m0=0.05, agg=((2, 2), (2, 2)), nvec=(2, 2), seed=5, sweeps=20):
    theta = inputs.metropolis_u1(Lx, Lt, beta, sweeps, seed)
    dims = [(Lx, Lt, 2)]
    for (ax, at), nv in zip(agg, nvec):
        dims.append((dims[-1][0] // ax, dims[-1][1] // at, 2 * nv))
    sv = [inputs.start_vectors(seed, i + 1, lx * lt * d, nv)
          for i, ((lx, lt, d), nv) in enumerate(zip(dims[:-1], nvec))]
    return theta, sv


def make_ctx(pkg, theta, m0, agg, nvec, sv, setup_iters, **opts):
    ctx = pkg.Context(**opts)
    ctx.set_gauge(theta)
    ctx.set_mass(m0)
    ctx.set_hierarchy(agg, nvec, sv, setup_iters=setup_iters, setup_tol=1e-13)
    return ctx


def rel_sample_error(got, ref):
    """max_j |s_gpu - s_ref| / max(|s_ref_j|, RMS |s_ref|) (per-sample error, zero-safe)."""
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    den = np.maximum(np.abs(ref), rms)
    return float(np.max(np.abs(got - ref) / den))


def rand_complex(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
