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


def bf16_deflation_bound(defl, X, factors_rounded=False):
    """Per-sample bound on how far the tensor-core deflation correction (factors
    rounded to BF16, FP32 accumulation over n terms) can be from the correction
    sum_m a_m conj(L_m^H x) (R_m^H x) that the oracle forms with defl's factors.

    Rounding a part of a factor moves it by at most u = 2^-8 (+ 2^-24 for the FP32
    step) of itself, so |dA_m| <= u ||R_m||_1 for +-1 entries; the FP32 sum of n
    terms adds at most 2 n 2^-24 ||R_m||_1.  With factors_rounded the oracle already
    uses the rounded factors and only the accumulation remains."""
    n = X.shape[1]
    acc = 2.0 * n * 2.0 ** -24
    u = acc if factors_rounded else 2.0 ** -8 + 2.0 ** -24 + acc
    Xt = np.ascontiguousarray(X.T).astype(np.complex128)
    A = np.abs(defl.R.conj().T @ Xt)
    B = np.abs(defl.L.conj().T @ Xt)
    eA = 1.01 * u * np.abs(defl.R).sum(axis=0)[:, None]
    eB = 1.01 * u * np.abs(defl.L).sum(axis=0)[:, None]
    return np.sum(defl.a[:, None] * (eA * B + eB * A + eA * eB), axis=0)


def within_bound(got, ref, bound, tol=1e-9):
    """|s_gpu - s_ref| <= tol * max(|s_ref|, RMS) + bound, per sample."""
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    return bool(np.all(np.abs(got - ref) <= tol * np.maximum(np.abs(ref), rms) + bound))

