"""Choose the Wilson mass m0 of a workload so that sigma_min(D) reaches a target.

Used once to fix the input parameter m0 of the 128^2 workload (sigma_min ~ 1e-3,
an ill-conditioned case like the small masses of Sect. 3.2 / Fig. 1).  Only the
oracle is used: sigma_min comes from inverse iteration on (D^H D)^{-1} with a
sparse LU of D.  Writes tests/golden/mass_<L>.json.

    python -m oracle.tune_mass schwinger-128x128 1e-3
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


def sigma_min(D, iters: int = 60, seed: int = 0) -> float:
    lu = spla.splu(sp.csc_matrix(D))
    x = np.random.default_rng(seed).standard_normal(D.shape[0]).astype(np.complex128)
    x /= np.linalg.norm(x)
    est = 0.0
    for _ in range(iters):
        y = lu.solve(lu.solve(x, trans="H"))        # (D^H D)^{-1} x = D^{-1} D^{-H} x
        nrm = np.linalg.norm(y)
        new = 1.0 / np.sqrt(nrm)
        x = y / nrm
        if abs(new - est) < 1e-10 * new:
            return new
        est = new
    return est


def tune(theta, target: float, m_hi: float = 0.0, step: float = 0.02, tol: float = 0.02):
    """Largest-sigma side bracket then bisection on m0 (sigma_min decreases towards m_c)."""
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


def main(argv):
    name = argv[1] if len(argv) > 1 else "schwinger-128x128"
    target = float(argv[2]) if len(argv) > 2 else 1e-3
    w = inputs.workload(name)
    m0, s = tune(w.gauge(), target)
    out = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "tests", "golden", f"mass_{w.Lx}.json")
    with open(out, "w") as f:
        json.dump({"workload": name, "target_sigma_min": target, "m0": round(m0, 6),
                   "sigma_min": s, "written_by": "python -m oracle.tune_mass"}, f, indent=1)
    print(out, m0, s)


if __name__ == "__main__":
    main(sys.argv)
