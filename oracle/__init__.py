"""Plain, slow FP64 CPU oracle for deflated multigrid multilevel Monte Carlo.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2211_15383_gb300``); the two meet only in
the seeded input generators of ``inputs``.

What it computes (Frommer & Ramirez-Hidalgo, "Deflated Multigrid Multilevel
Monte Carlo", Lattice 2022):

* ``wilson``     -- the 2D Wilson-Schwinger operator D and Gamma5 (Sect. 1, 2).
* ``hierarchy``  -- spin-preserving aggregation P_l, Galerkin D_{l+1} = P^H D P
                    and the test-vector setup (Sect. 3.1, Sect. 4.2).
* ``deflation``  -- smallest singular triplets of D from the eigenpairs of
                    Q = Gamma5 D, and the deflated trace term (Sect. 2).
* ``noise``      -- the counter-based Z2 noise of the Hutchinson estimator.
* ``rounding``   -- BF16 rounding of the factors of the tensor-core deflation.
* ``tune_mass``  -- sigma_min(D) by inverse iteration, used to choose the masses.
* ``estimator``  -- per-sample values of every term of the telescoping sum
                    (Eq. mgmlmc, Eq. skip_level), exact traces by dense
                    inversion, the closed-form Z2 variance (Eq.
                    variance_in_terms_of_frob_norm) and the MLMC stopping rule.

Every linear solve is a direct one (dense LU or sparse LU); the oracle has no
smoother and no Krylov method: multigrid only accelerates the CUDA path, while
the samples it must reproduce are defined by exact inverses.

Parity status of each function is stated in its docstring; functions with no
independent pin say "parity unpinned".
"""
from . import wilson, hierarchy, deflation, noise, estimator, rounding  # noqa: F401
