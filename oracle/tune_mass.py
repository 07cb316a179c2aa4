"""Choose the Wilson mass m0 of a workload so that sigma_min(D) reaches a target.

Used once to fix the input parameter m0 of the 128^2 workload (sigma_min ~ 1e-3,
an ill-conditioned case like the small masses of Sect. 3.2 / Fig. 1).  Only the
oracle is used: sigma_min comes from inverse iteration on (D^H D)^{-1} with a
sparse LU of D.  Writes tests/golden/mass_<L>.json.

    python -m oracle.tune_mass schwinger-128x128 1e-3
    python -m oracle.tune_mass schwinger-128x128 1e-3 --at -0.141406
    python -m oracle.tune_mass schwinger-1024x1024 1e-3 --lattice 128

With --at the bisection is skipped: sigma_min is evaluated (to the default,
certified residual) at the given m0, which is recorded with it.  With
--lattice L the workload's gauge recipe (beta, sweeps, seed) is run on an L x L
lattice and the mass is tuned there (a lattice whose sparse LU the oracle can
afford; the additive mass shift is a short-distance effect), written to
tests/golden/mass_<Lx>_at<L>.json.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import inputs
from oracle import wilson


def sigma_min(D, iters: int = 5000, seed: int = 0, tol: float = 1e-13) -> float:
    """Smallest singular value of D by inverse iteration on A = (D^H D)^{-1}.

    A is Hermitian positive definite with largest eigenvalue 1/sigma_min^2.  Each
    step forms w = D^{-H} x and y = D^{-1} w = A x (two solves with one LU of D);
    theta = x^H A x = ||w||^2 is the Rayleigh quotient of the unit vector x.  The
    iteration stops once the residual ||A x - theta x|| is at most tol * theta:
    for Hermitian A an eigenvalue then lies within that distance of theta, so the
    stop certifies the estimate (a stop on the change of successive estimates
    does not: it ends early on nearly degenerate singular values).
    """
    lu = spla.splu(sp.csc_matrix(D))
    x = np.random.default_rng(seed).standard_normal(D.shape[0]).astype(np.complex128)
    x /= np.linalg.norm(x)
    theta = 0.0
    for _ in range(iters):
        w = lu.solve(x, trans="H")                  # D^{-H} x
        y = lu.solve(w)                             # D^{-1} D^{-H} x = (D^H D)^{-1} x
        theta = float(np.vdot(w, w).real)           # x^H (D^H D)^{-1} x
        if np.linalg.norm(y - theta * x) <= tol * theta:
            break
        x = y / np.linalg.norm(y)
    return 1.0 / np.sqrt(theta)


_sigma_min = sigma_min


def tune(theta, target: float, m_hi: float = 0.0, step: float = 0.02, tol: float = 0.02):
    """Largest-sigma side bracket then bisection on m0 (sigma_min decreases towards m_c).

    The bisection needs sigma_min to about 1e-3 relative, so its estimates stop at a
    residual of 1e-3: the Rayleigh quotient's error is of the order of the squared
    residual over the relative gap, and within a cluster of nearly equal singular
    values it lies inside the cluster."""

    def sigma_min(D):
        return _sigma_min(D, tol=1e-3)

    s_hi = sigma_min(wilson.wilson_dirac(theta, m_hi))
    m_lo = m_hi
    while True:
        m_lo -= step
        s_lo = sigma_min(wilson.wilson_dirac(theta, m_lo))
        print(f"scan m0={m_lo:+.5f} sigma_min={s_lo:.3e}", flush=True)
        if s_lo < target or s_lo > s_hi:      # crossed the target, or passed the minimum
            break
        m_hi, s_hi = m_lo, s_lo
    for _ in range(40):
        m = 0.5 * (m_lo + m_hi)
        s = sigma_min(wilson.wilson_dirac(theta, m))
        print(f"bisect m0={m:+.6f} sigma_min={s:.4e}", flush=True)
        if abs(s / target - 1) < tol:
            return m, s
        if s > target:
            m_hi = m
        else:
            m_lo = m
    return m, s


def _option(argv, flag):
    if flag not in argv:
        return argv, None
    i = argv.index(flag)
    return argv[:i] + argv[i + 2:], float(argv[i + 1])


def main(argv):
    argv, at = _option(argv, "--at")
    argv, lat = _option(argv, "--lattice")
    name = argv[1] if len(argv) > 1 else "schwinger-128x128"
    target = float(argv[2]) if len(argv) > 2 else 1e-3
    w = inputs.workload(name)
    if lat is None:
        theta, fname, lattice = w.gauge(), f"mass_{w.Lx}.json", f"{w.Lx}x{w.Lt}"
    else:
        L = int(lat)
        theta = inputs.metropolis_u1(L, L, w.beta, w.sweeps, w.gauge_seed)
        fname, lattice = f"mass_{w.Lx}_at{L}.json", f"{L}x{L}"
    m0 = at if at is not None else tune(theta, target)[0]
    s = sigma_min(wilson.wilson_dirac(theta, m0))
    out = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden", fname)
    with open(out, "w") as f:
        json.dump({"workload": name, "tuned_on": lattice, "target_sigma_min": target, "m0": round(m0, 6),
                   "sigma_min": s, "written_by": "python -m oracle.tune_mass"}, f, indent=1)
    print(out, m0, s)


if __name__ == "__main__":
    main(sys.argv)
