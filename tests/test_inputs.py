"""Host-side checks of the seeded input generators (no GPU)."""
import json
import os

import numpy as np

import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_parallel_metropolis_equals_serial():
    # the strip-parallel form updates exactly the links of the serial form, with the
    # same counter-based draws: the fields agree bit for bit
    for (L, beta, sweeps, seed, workers) in [(16, 3.0, 20, 11, 4), (32, 5.0, 30, 12, 3)]:
        a = inputs.metropolis_u1(L, L, beta, sweeps, seed, workers=1)
        b = inputs.metropolis_u1(L, L, beta, sweeps, seed, workers=workers)
        assert np.array_equal(a, b)


def test_workload_masses_come_from_the_oracle_tuning():
    # the masses of the tuned workloads are the ones python -m oracle.tune_mass wrote
    for name, fname in [("schwinger-128x128", "mass_128.json"), ("schwinger-1024x1024", "mass_1024_at256.json")]:
        g = json.load(open(os.path.join(GOLDEN, fname)))
        assert g["workload"] == name
        assert inputs.workload(name).m0 == g["m0"]
        assert abs(g["sigma_min"] / g["target_sigma_min"] - 1) < 0.02


def test_workload_term_levels():
    w = inputs.workload("schwinger-1024x1024")
    assert w.nlevels == 4 and w.term_levels == (1, 2, 3) and w.nterms == 3
    dims = w.level_dims()
    assert [lx * lt * d for lx, lt, d in dims] == [2097152, 1048576, 262144, 16384]
    w3 = inputs.workload("schwinger-256x256")
    assert w3.term_levels == (1, 2, 3) and [lx * lt * d for lx, lt, d in w3.level_dims()] == [131072, 65536, 16384,
                                                                                              4096]
